// Tile-chunk rendering pipeline (Aokana Sec. 3.5, Fig. 7): the paper's own
// organisation of the primary-ray pass, kept beside the per-ray chunk march
// (aok_kernels.cu) as an alternative with identical output.
//
//   1. tile selection: every chunk region selected and visible this frame
//      (select_kernel) projects its AABB of valid voxels to a rectangle of
//      8x8-pixel tiles; each (tile, chunk) in it is a pair, with the distance
//      from the camera to the AABB as the pair's depth (a lower bound of every
//      hit in it, which is what the paper's AABB depth is).
//   2. ray marching, pass 1: every pair whose depth is not beyond the tile's
//      depth in the previous frame's Hi-Z is marched: each pixel ray of the
//      tile is traced through that chunk's DAG only, and its hit goes into a
//      screen-sized 64-bit visibility buffer with an atomic minimum (the
//      paper's InterlockedMax on an inverted depth).
//   3. Hi-Z of this frame from the visibility buffer (per-tile maximum of an
//      upper bound of each pixel's distance so far).
//   4. ray marching, pass 2: the pairs pass 1 culled are tested again
//      against this frame's Hi-Z and the survivors marched.
//   5. resolve: each pixel decodes its visibility record and writes the same
//      output record as the march; the per-tile maximum of the final
//      distances becomes the next frame's Hi-Z.
//
// Pass 2 makes the result independent of the previous frame: a pair it culls
// lies beyond every pixel's current hit in that tile, so it cannot hold a
// nearer one.  With the beam pass (aok_beam.cu) a half tile (8 x 4 pixels,
// one beam tile) also skips the pairs whose chunk AABB lies wholly nearer
// than its bound -- no voxel there can be met -- and its rays start each
// remaining pair at the bound's restart plane, as in the march.  Differences from the paper: the pair list is implicit (a
// prefix sum over the chunks' rectangle areas, searched by the marching warps)
// instead of an appended TileInfo buffer with indirect dispatch; the key is
// widened; each marching warp takes half a tile (32 pixels).
//
// Visibility record: 16 bytes per pixel, a key and a payload installed
// together by a 128-bit compare-and-swap (the paper's 64-bit InterlockedMax
// record of depth | normal | 13-bit chunk ID | 24-bit position cannot address
// 512^3 chunks).  Payload: the hit voxel's world LOD-0 corner x, y, z (17 bits
// each), its LOD (3 bits), the entry axis (2 bits; 3: origin inside) and the
// material (8 bits) -- with the ray, everything the output record needs.
// Key:
//   bits 63..32  top 32 bits of the FP64 ray parameter t of the hit (t >= 0,
//                so the IEEE bits order as integers; truncation keeps order)
//   bits 31..16  place of the chunk region in the march order along the ray:
//                the sum of its mirrored grid coordinates, which grows by one
//                from each region of a ray's march to the next
//   bits 15..0   chunk region index (scenes of at most 65536 regions)
// The minimum key is the hit of the first region along the ray that has one,
// the march's answer: a later region's hit never has a smaller t, and equal
// truncated t falls back to the march order.
#include <cuda_runtime.h>

#include <cstdint>

#include "aok_internal.h"
#include "aok_trace.cuh"

using namespace aok;

namespace {

constexpr unsigned long long kNoKey = ~0ull;
constexpr int kCasLimit = 4096;  // attempts: each failure means another chunk's smaller key went in

// 128-bit compare-and-swap on a 16-byte aligned record (sm_90+): returns the
// previous record.
__device__ __forceinline__ ulonglong2 cas128(unsigned long long* p, ulonglong2 cmp, ulonglong2 val) {
    ulonglong2 old;
    asm volatile("{\n\t.reg .b128 d, c, n;\n\t"
                 "mov.b128 c, {%2, %3};\n\t"
                 "mov.b128 n, {%4, %5};\n\t"
                 "atom.global.cas.b128 d, [%6], c, n;\n\t"
                 "mov.b128 {%0, %1}, d;\n\t}"
                 : "=l"(old.x), "=l"(old.y)
                 : "l"(cmp.x), "l"(cmp.y), "l"(val.x), "l"(val.y), "l"(p)
                 : "memory");
    return old;
}
enum { kStList = 0, kStTraced1, kStCulled1, kStTraced2, kStCulled2, kStPixelTraces, kStPixelSkips, kStCasExhausted };

__device__ __forceinline__ void region_coords(const SceneDev& S, uint32_t chunk, int32_t u[3]) {
    u[0] = (int32_t)(chunk % (uint32_t)S.grid[0]);
    u[1] = (int32_t)((chunk / (uint32_t)S.grid[0]) % (uint32_t)S.grid[1]);
    u[2] = (int32_t)(chunk / ((uint32_t)S.grid[0] * (uint32_t)S.grid[1]));
}

// top 32 bits of t = N / (2^12 |d_e|) in FP64 (N >= 0; exact operands, one rounding)
__device__ __forceinline__ uint32_t t_key(int32_t N, float de) {
    const double t = __ddiv_rn((double)N, __dmul_rn(4096.0, fabs((double)de)));
    return (uint32_t)((unsigned long long)__double_as_longlong(t) >> 32);
}

// How the march enters chunk region u: entry axis e (3: the origin lies in
// it), entry plane numerator Ne, mirrored local origin.  Returns false when
// the march does not visit the region.  A region the ray passes with positive
// length is visited; one it only touches (entry instant = exit instant, an
// edge or corner) is visited when every axis it is left through has a lower
// index than every axis it is entered through, because at a tie the march
// steps the axis of higher index first.  Rays that enter the world box
// exactly on an interior chunk plane are the one case decided differently
// (the march places them past the plane).
struct Entry {
    int e;
    int32_t Ne;
    int32_t Oloc[3];
    int32_t Hi[3];  // exit plane numerators of the region
    uint32_t order;
};

template <bool FAST>
__device__ __forceinline__ bool enter_region(const SceneDev& S, const CamDev& C, const RayState& r,
                                             const int32_t u[3], Entry& en) {
    const int cs = S.mlog + kFix;
    int32_t Lo[3], Hi[3];
    uint32_t order = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const bool m = (r.mir >> a) & 1u;
        const int32_t Wfix = S.grid[a] << cs;
        const int32_t Ow = m ? Wfix - C.O[a] : C.O[a];
        const int32_t cc = m ? S.grid[a] - 1 - u[a] : u[a];
        order += (uint32_t)cc;
        Lo[a] = (cc << cs) - Ow;
        Hi[a] = ((cc + 1) << cs) - Ow;
        en.Oloc[a] = -Lo[a];
        en.Hi[a] = Hi[a];
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (Hi[a] <= 0) return false;                      // behind the origin
        if (r.d[a] == 0.0f && Lo[a] > 0) return false;     // parallel slab missed
    }
    int e = 3;
    int32_t Ne = 0, me = 1, Ee = 0;
#pragma unroll
    for (int a = 0; a < 3; a++)  // latest entry plane; ties keep the lowest axis
        if (Lo[a] > 0 && (e == 3 || tltf<FAST>(Ne, me, Lo[a], r.m[a], r.E[a] - Ee))) {
            e = a; Ne = Lo[a]; me = r.m[a]; Ee = r.E[a];
        }
    if (e < 3) {
        int maxpre = -1;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (r.d[a] == 0.0f) continue;
            if (tltf<FAST>(Hi[a], r.m[a], Ne, me, Ee - r.E[a])) return false;  // left before entered
            if (!tltf<FAST>(Ne, me, Hi[a], r.m[a], r.E[a] - Ee)) maxpre = a;    // left at the entry instant
        }
        if (maxpre > e) return false;
    }
    en.e = e;
    en.Ne = Ne;
    en.order = order;
    return true;
}

// The march's skip of regions whose solid-voxel AABB (grown by 1/16 voxel)
// the ray misses, with the same FP32 arithmetic.
__device__ __forceinline__ bool aabb_pass(const SceneDev& S, const CamDev& C, const RayState& r, const ChunkRef& ref,
                                          const int32_t u[3]) {
    float tn = 0.0f, tf = 3.0e38f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float lo = (float)((u[a] << S.mlog) + ref.aabb[a]) - 0.0625f;
        const float hi = (float)((u[a] << S.mlog) + ref.aabb[3 + a]) + 0.0625f;
        if (r.d[a] == 0.0f) {
            if (C.of[a] < lo || C.of[a] > hi) return false;
        } else {
            const float inv = 1.0f / r.d[a];
            const float t1 = (lo - C.of[a]) * inv, t2 = (hi - C.of[a]) * inv;
            tn = fmaxf(tn, fminf(t1, t2));
            tf = fminf(tf, fmaxf(t1, t2));
        }
    }
    return tn <= tf;
}

// One pixel of a pair: 0 = region not entered, 1 = traced, 2 = skipped (the
// pixel already holds a hit nearer than the region's entry, or the beam
// bound Dn puts every voxel the ray can meet past the region).  Dn > 0: the
// ray starts at the bound's restart plane when that lies later than the
// region's entry (trace_pixel_t's beam restart, within one region).
template <bool FAST, bool BEAM>
__device__ __forceinline__ int pair_pixel(const SceneDev& S, const CamDev& C, const ChunkRef& ref, uint32_t chunk,
                                          const RayState& r, size_t pix, unsigned long long* __restrict__ vis,
                                          int32_t Dn) {
    int32_t u[3];
    region_coords(S, chunk, u);
    Entry en;
    if (!enter_region<FAST>(S, C, r, u, en) || !aabb_pass(S, C, r, ref, u)) return 0;
    unsigned long long* rec = vis + 2 * pix;
    const unsigned long long cur = __ldcg(rec);
    if (cur != kNoKey && en.e < 3 && t_key(en.Ne, r.d[en.e]) > (uint32_t)(cur >> 32)) return 2;
    int e = en.e;
    int32_t Ne = en.Ne;
    if (BEAM && Dn > 0) {
        // the last integer plane of the dominant axis crossed before the ray's
        // L-inf distance reaches Dn; at or past the region's exit: no hit here
        int as = 0;
        if (fabsf(r.d[1]) > fabsf(r.d[as])) as = 1;
        if (fabsf(r.d[2]) > fabsf(r.d[as])) as = 2;
        const int32_t Wf = S.grid[as] << (S.mlog + kFix);
        const int32_t Ow = ((r.mir >> as) & 1u) ? Wf - C.O[as] : C.O[as];
        const long long kp = ((long long)Dn - 1 + Ow) >> kFix;
        const long long Nl = (kp << kFix) - Ow;
        if (Nl >= (long long)en.Hi[as]) return 2;
        const int32_t me = e < 3 ? r.m[e] : 1, Ee = e < 3 ? r.E[e] : 0;
        if (Nl > 0 && (e == 3 || tltf<FAST>(Ne, me, (int32_t)Nl, r.m[as], r.E[as] - Ee))) {
#pragma unroll
            for (int a = 0; a < 3; a++)
                if (a != as && r.d[a] != 0.0f && !tltf<FAST>((int32_t)Nl, r.m[as], en.Hi[a], r.m[a], r.E[a] - r.E[as]))
                    return 2;  // the ray leaves the region no later than the restart point
            e = as;
            Ne = (int32_t)Nl;
        }
    }
    HitRec hit;
    Counters cnt = {0, 0, 0};
    if (trace_chunk<FAST, false, false, BEAM>(S, ref, r, en.Oloc, e, Ne, hit, cnt) &&
        (lowest_entry_face<FAST>(r, en.Oloc, (int)ref.lod, hit), within_view(S, r, hit))) {
        const uint32_t tk = hit.e < 3 ? t_key(hit.Ne, r.d[hit.e]) : 0u;
        const int n = (int)ref.lod;
        const int32_t side = (1 << (S.mlog - n)) - 1;
        unsigned long long pay = 0;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int32_t uv = ((r.mir >> a) & 1u) ? side - hit.c[a] : hit.c[a];
            pay |= (unsigned long long)(uint32_t)((u[a] << S.mlog) + (uv << n)) << (17 * a);
        }
        const uint32_t mat = hit_material(S, ref, hit.idx);
        pay |= (unsigned long long)n << 51 | (unsigned long long)hit.e << 54 | (unsigned long long)mat << 56;
        const ulonglong2 mine = make_ulonglong2(
            ((unsigned long long)tk << 32) | ((unsigned long long)(en.order & 0xFFFFu) << 16) | chunk, pay);
        // install the record if its key is the smallest so far
        ulonglong2 seen = make_ulonglong2(cur, __ldcg(rec + 1));
        int tries = 0;
        while (seen.x > mine.x) {
            if (++tries > kCasLimit) return 3;
            const ulonglong2 old = cas128(rec, seen, mine);
            if (old.x == seen.x && old.y == seen.y) break;
            seen = old;
        }
    }
    return 1;
}

// ---------------------------------------------------------------------------
// 1. tile selection: per chunk region, its tile rectangle and depth
// ---------------------------------------------------------------------------
// Eight lanes per region (lane k projects corner k of its AABB; FP64 is a
// slow pipe on this GPU, so the corners are spread over more SMs).
__global__ void __launch_bounds__(128) tc_rect_kernel(SceneDev S, CamDev C, const ChunkRef* __restrict__ frame,
                                                      TileDev T) {
    const int nch = S.grid[0] * S.grid[1] * S.grid[2];
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = tid >> 3, k = tid & 7;
    const bool valid = chunk < nch;
    const ChunkRef ref = valid ? frame[chunk] : ChunkRef{kNone, 0, 0, {0, 0, 0, 0, 0, 0}, 0};
    uint32_t area = 0;
    int4 rc = make_int4(0, 0, 0, 0);
    float dm = 0.0f;
    int32_t far = 0;
    // the group's lanes agree on every branch below (same region)
    const bool live = valid && ref.root != kNone;
    double lo[3] = {0.0, 0.0, 0.0}, hi[3] = {0.0, 0.0, 0.0};
    if (live) {
        int32_t u[3];
        region_coords(S, (uint32_t)chunk, u);
        double d2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; a++) {  // exact: |values| < 2^30
            const int32_t l = (((u[a] << S.mlog) + (int32_t)ref.aabb[a]) << kFix) - C.O[a];
            const int32_t h = (((u[a] << S.mlog) + (int32_t)ref.aabb[3 + a]) << kFix) - C.O[a];
            far = max(far, max(abs(l), abs(h)));
            lo[a] = (double)((u[a] << S.mlog) + ref.aabb[a]) - (double)C.of[a];
            hi[a] = (double)((u[a] << S.mlog) + ref.aabb[3 + a]) - (double)C.of[a];
            const double q = fmax(fmax(lo[a], -hi[a]), 0.0);
            d2 += q * q;
        }
        // every hit point of the region lies in the AABB: its distance is >= this
        if (k == 0) dm = __double2float_rd(sqrt(d2) * (1.0 - 1e-12));
    }
    dm = __shfl_sync(0xFFFFFFFFu, dm, 0, 8);
    const bool project = live && !(S.view_dist > 0.0f && dm > S.view_dist);
    // screen position of corner k (pixel-centre coordinates); a corner near or
    // behind the camera plane makes the rectangle the whole screen
    double px = 0.0, py = 0.0;
    bool full = false;
    if (project) {
        const double th = C.tan_half, asp = (double)C.W / (double)C.H;
        const double p0 = (k & 1) ? hi[0] : lo[0], p1 = (k & 2) ? hi[1] : lo[1], p2 = (k & 4) ? hi[2] : lo[2];
        const double xc = C.R[0] * p0 + C.R[3] * p1 + C.R[6] * p2;
        const double yc = C.R[1] * p0 + C.R[4] * p1 + C.R[7] * p2;
        const double zc = -(C.R[2] * p0 + C.R[5] * p1 + C.R[8] * p2);
        if (zc < 1e-3 * (fabs(p0) + fabs(p1) + fabs(p2) + 1.0)) {
            full = true;
        } else {
            px = (xc / zc / (th * asp) + 1.0) * 0.5 * C.W - 0.5;
            py = (1.0 - yc / zc / th) * 0.5 * C.H - 0.5;
        }
    }
    double x0 = full ? 1e300 : px, x1 = full ? -1e300 : px, y0 = full ? 1e300 : py, y1 = full ? -1e300 : py;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        x0 = fmin(x0, __shfl_xor_sync(0xFFFFFFFFu, x0, o, 8));
        x1 = fmax(x1, __shfl_xor_sync(0xFFFFFFFFu, x1, o, 8));
        y0 = fmin(y0, __shfl_xor_sync(0xFFFFFFFFu, y0, o, 8));
        y1 = fmax(y1, __shfl_xor_sync(0xFFFFFFFFu, y1, o, 8));
        const int fo = __shfl_xor_sync(0xFFFFFFFFu, (int)full, o, 8);  // every lane shuffles
        full = full || fo;
    }
    if (project) {
        if (full) {
            rc = make_int4(0, 0, T.tiles_x, T.tiles_y);
        } else {  // 2 px margin
            rc.x = (int)fmax(floor((x0 - 2.0) / 8.0), 0.0);
            rc.y = (int)fmax(floor((y0 - 2.0) / 8.0), 0.0);
            rc.z = (int)fmin(floor((x1 + 2.0) / 8.0) + 1.0, (double)T.tiles_x);
            rc.w = (int)fmin(floor((y1 + 2.0) / 8.0) + 1.0, (double)T.tiles_y);
        }
        if (rc.z > rc.x && rc.w > rc.y) area = (uint32_t)(rc.z - rc.x) * (uint32_t)(rc.w - rc.y);
    }
    if (valid && k == 0) {
        T.rect[chunk] = rc;
        T.dmin[chunk] = dm;
        T.dfar[chunk] = far;
        T.area[chunk] = area;
    }
}

// Compacts the regions with pairs (ascending) and their exclusive area prefix
// (one block); zeroes the frame's statistics.
__global__ void __launch_bounds__(1024) tc_scan_kernel(int nch, TileDev T) {
    __shared__ unsigned long long s_sum[1024];
    __shared__ uint32_t s_cnt[1024];
    const int tid = threadIdx.x;
    const int per = (nch + 1023) / 1024;
    const int b = min(tid * per, nch), e = min(b + per, nch);
    unsigned long long sum = 0;
    uint32_t cnt = 0;
    for (int i = b; i < e; i++) {
        const uint32_t a = T.area[i];
        sum += a;
        cnt += a ? 1u : 0u;
    }
    s_sum[tid] = sum;
    s_cnt[tid] = cnt;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned long long vs = tid >= off ? s_sum[tid - off] : 0ull;
        const uint32_t vc = tid >= off ? s_cnt[tid - off] : 0u;
        __syncthreads();
        s_sum[tid] += vs;
        s_cnt[tid] += vc;
        __syncthreads();
    }
    unsigned long long base = s_sum[tid] - sum;
    uint32_t pos = s_cnt[tid] - cnt;
    for (int i = b; i < e; i++) {
        const uint32_t a = T.area[i];
        if (a) {
            T.list[pos] = (uint32_t)i;
            T.offs[pos] = base;
            pos++;
            base += a;
        }
    }
    if (tid == 1023) {
        T.offs[s_cnt[1023]] = s_sum[1023];
        T.stats[kStList] = s_cnt[1023];
    }
    if (tid > 0 && tid < kTileStats) T.stats[tid] = 0ull;
}

// ---------------------------------------------------------------------------
// 2./4. ray marching of the pairs: each warp takes half a tile (8 x 4 pixels)
// of one pair; warps stride over all 2 x pairs items.  PASS 1 marches the
// pairs the previous frame's Hi-Z keeps, PASS 2 those it culled and this
// frame's keeps.
// ---------------------------------------------------------------------------
template <int PASS, bool BEAM>
__global__ void __launch_bounds__(128, 7) tc_cast_kernel(SceneDev S, CamDev C, const ChunkRef* __restrict__ frame,
                                                      TileDev T, const BeamLookup beam) {
    const uint32_t n_list = (uint32_t)T.stats[kStList];
    if (n_list == 0) return;
    const unsigned long long n_items = 2ull * T.offs[n_list];
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    uint32_t traced = 0, culled = 0, pix_traced = 0, pix_skipped = 0;
    for (unsigned long long item = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < n_items;
         item += nw) {
        const unsigned long long pair = item >> 1;
        uint32_t lo = 0, hi = n_list - 1;  // last listed region with offs <= pair
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (T.offs[mid] <= pair) lo = mid;
            else hi = mid - 1;
        }
        const uint32_t chunk = T.list[lo];
        const uint32_t local = (uint32_t)(pair - T.offs[lo]);
        const int4 rc = T.rect[chunk];
        const int rw = rc.z - rc.x;
        const int tx = rc.x + (int)(local % (uint32_t)rw), ty = rc.y + (int)(local / (uint32_t)rw);
        const int tile = ty * T.tiles_x + tx;
        const float dm = T.dmin[chunk];
        if (PASS == 1) {
            if (dm > T.hiz_prev[tile]) { culled++; continue; }
        } else {
            if (dm <= T.hiz_prev[tile]) continue;  // marched in pass 1
            if (dm > T.hiz[tile]) { culled++; continue; }
        }
        const int by = ty * 2 + (int)(item & 1);  // the half tile: one beam tile
        if (by * 4 >= C.H) continue;              // below the last row
        int32_t Dn = 0;
        if (BEAM) {
            Dn = warp_beam_bound(beam, (uint32_t)tx, (uint32_t)by, lane);
            if (Dn > T.dfar[chunk]) { culled++; continue; }  // wholly nearer than every voxel its rays meet
        }
        traced++;
        const int px = tx * 8 + (lane & 7), py = by * 4 + (lane >> 3);
        if (px < C.W && py < C.H) {
            const ChunkRef ref = frame[chunk];
            RayState r;
            const size_t pix = (size_t)py * C.W + px;
            const int res = make_ray(C, px, py, r) ? pair_pixel<true, BEAM>(S, C, ref, chunk, r, pix, T.vis, Dn)
                                                   : pair_pixel<false, BEAM>(S, C, ref, chunk, r, pix, T.vis, Dn);
            pix_traced += res == 1;
            pix_skipped += res == 2;
            if (res == 3) atomicAdd(&T.stats[kStCasExhausted], 1ull);
        }
    }
    pix_traced = __reduce_add_sync(0xFFFFFFFFu, pix_traced);
    pix_skipped = __reduce_add_sync(0xFFFFFFFFu, pix_skipped);
    if (lane == 0) {
        if (traced) atomicAdd(&T.stats[PASS == 1 ? kStTraced1 : kStTraced2], (unsigned long long)traced);
        if (culled) atomicAdd(&T.stats[PASS == 1 ? kStCulled1 : kStCulled2], (unsigned long long)culled);
        if (pix_traced) atomicAdd(&T.stats[kStPixelTraces], (unsigned long long)pix_traced);
        if (pix_skipped) atomicAdd(&T.stats[kStPixelSkips], (unsigned long long)pix_skipped);
    }
}

// ---------------------------------------------------------------------------
// 3. Hi-Z of this frame after pass 1: per tile, the maximum over its pixels of
// an upper bound of the distance of the pixel's hit so far (+inf: none yet).
// One warp per tile.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tc_hiz_kernel(CamDev C, TileDev T) {
    const int lane = threadIdx.x & 31;
    const int tile = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (tile >= T.tiles_x * T.tiles_y) return;
    const int tx = tile % T.tiles_x, ty = tile / T.tiles_x;
    float m = 0.0f;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int px = tx * 8 + (lane & 7), py = ty * 8 + k * 4 + (lane >> 3);
        if (px < C.W && py < C.H) {
            const unsigned long long key = __ldcg(T.vis + 2 * ((size_t)py * C.W + px));
            float dist = __int_as_float(0x7F800000);
            if (key != kNoKey) {
                float d[3];
                ray_dir(C, px, py, d);
                // upper bounds in FP32 with upward rounding: |d| and t (the key's next value)
                const float dn = __fsqrt_ru(__fadd_ru(__fadd_ru(__fmul_ru(d[0], d[0]), __fmul_ru(d[1], d[1])),
                                                      __fmul_ru(d[2], d[2])));
                const float t_up = __double2float_ru(__longlong_as_double((long long)(((key >> 32) + 1ull) << 32)));
                dist = __fmul_ru(t_up, dn);
            }
            m = fmaxf(m, dist);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if (lane == 0) T.hiz[tile] = m;
}

// ---------------------------------------------------------------------------
// 5. resolve: 16 x 8 pixel blocks (two tiles), warps of 8 x 4 pixels
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) tc_resolve_kernel(SceneDev S, CamDev C, const ChunkRef* __restrict__ frame,
                                                         TileDev T, uint4* __restrict__ out_hit,
                                                         float* __restrict__ out_t) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tx = blockIdx.x * 2 + (warp & 1), ty = blockIdx.y;
    const int px = tx * 8 + (lane & 7);
    const int py = ty * 8 + (warp >> 1) * 4 + (lane >> 3);
    float dist_up = 0.0f;
    if (px < C.W && py < C.H) {
        const size_t pix = (size_t)py * C.W + px;
        const ulonglong2 rec = __ldcg(reinterpret_cast<const ulonglong2*>(T.vis) + pix);
        if (rec.x == kNoKey) {
            emit_miss(out_hit, out_t, pix);
            dist_up = __int_as_float(0x7F800000);
        } else {
            // the output record of emit_hit, rebuilt from the payload and the ray
            RayState r;
            ray_dir(C, px, py, r.d);
            r.mir = (r.d[0] < 0.0f ? 1u : 0u) | (r.d[1] < 0.0f ? 2u : 0u) | (r.d[2] < 0.0f ? 4u : 0u);
            const unsigned long long pay = rec.y;
            const uint32_t x = (uint32_t)(pay & 0x1FFFFu), y = (uint32_t)((pay >> 17) & 0x1FFFFu),
                           z = (uint32_t)((pay >> 34) & 0x1FFFFu);
            const int n = (int)((pay >> 51) & 7u), e = (int)((pay >> 54) & 3u);
            const uint32_t mat = (uint32_t)(pay >> 56);
            float dist = 0.0f;
            if (e < 3) {
                // entry plane: the voxel's face the mirrored ray meets first, as a numerator
                const uint32_t w[3] = {x, y, z};
                const bool m = (r.mir >> e) & 1u;
                const int32_t wext = S.grid[e] << S.mlog;
                const int32_t face = m ? wext - (int32_t)w[e] - (1 << n) : (int32_t)w[e];
                const int32_t Ow = m ? (S.grid[e] << (S.mlog + kFix)) - C.O[e] : C.O[e];
                const int32_t Ne = (face << kFix) - Ow;
                dist = __fdiv_rn((float)Ne * (1.0f / 4096.0f), fabsf(r.d[e])) * ray_norm(r);
            }
            const uint32_t normal = e == 3 ? 7u : (uint32_t)(2 * e) + ((r.mir >> e) & 1u);
            out_hit[pix] = make_uint4(x, y, z, (uint32_t)n | (mat << 8) | (normal << 16) | (1u << 19));
            out_t[pix] = dist;
            dist_up = __fmul_ru(dist, 1.000001f);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dist_up = fmaxf(dist_up, __shfl_xor_sync(0xFFFFFFFFu, dist_up, o));
    if (lane == 0 && tx < T.tiles_x && ty < T.tiles_y)
        atomicMax((int*)&T.hiz_next[ty * T.tiles_x + tx], __float_as_int(dist_up));
}

int tiles_status(cudaError_t e) { return aokk_status(e); }

}  // namespace

extern "C" {

int aokk_tiles_frame(const SceneDev* S, const CamDev* C, const ChunkRef* frame, const TileDev* T, uint4* hit, float* t,
                     int sms, void* stream, const BeamRead* beam) {
    const cudaStream_t s = (cudaStream_t)stream;
    const int nch = S->grid[0] * S->grid[1] * S->grid[2];
    const int tiles = T->tiles_x * T->tiles_y;
    static int per_sm[2] = {0, 0};
    if (!per_sm[0]) {
        int a = 0, b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, tc_cast_kernel<1, true>, 128, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tc_cast_kernel<2, true>, 128, 0);
        per_sm[1] = b > 0 ? b : 1;
        per_sm[0] = a > 0 ? a : 1;
    }
    const BeamLookup bl = beam_lookup(beam && beam->bounds ? beam : nullptr, C->W, C->H);
    cudaError_t e = cudaMemsetAsync(T->hiz_next, 0, (size_t)tiles * sizeof(float), s);
    if (e != cudaSuccess) return AOK_E_CUDA;
    tc_rect_kernel<<<(8 * nch + 127) / 128, 128, 0, s>>>(*S, *C, frame, *T);
    tc_scan_kernel<<<1, 1024, 0, s>>>(nch, *T);
    if (bl.bounds) tc_cast_kernel<1, true><<<sms * per_sm[0], 128, 0, s>>>(*S, *C, frame, *T, bl);
    else tc_cast_kernel<1, false><<<sms * per_sm[0], 128, 0, s>>>(*S, *C, frame, *T, bl);
    tc_hiz_kernel<<<(tiles + 7) / 8, 256, 0, s>>>(*C, *T);
    if (bl.bounds) tc_cast_kernel<2, true><<<sms * per_sm[1], 128, 0, s>>>(*S, *C, frame, *T, bl);
    else tc_cast_kernel<2, false><<<sms * per_sm[1], 128, 0, s>>>(*S, *C, frame, *T, bl);
    tc_resolve_kernel<<<dim3((C->W + 15) / 16, (C->H + 7) / 8), 128, 0, s>>>(*S, *C, frame, *T, hit, t);
    e = cudaMemsetAsync(T->vis, 0xFF, (size_t)C->W * C->H * 16, s);  // re-armed for the next frame
    if (e != cudaSuccess) return AOK_E_CUDA;
    return tiles_status(cudaGetLastError());
}

}  // extern "C"
