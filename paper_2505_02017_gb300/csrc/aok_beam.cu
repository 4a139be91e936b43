// Beam pass: the beam optimisation of ESVO (Laine and Karras; Aokana Sec. 2
// names ESVO as the traversal it builds on), recast so that it cannot change
// a single output record.
//
// ESVO casts a coarse ray per pixel block first and starts the block's rays
// near the surface the coarse ray found.  Here the coarse pass computes, for
// every 8 x 4 pixel tile (one casting warp), a lower bound Dn on the
// L-infinity distance from the camera origin of every solid voxel of the
// frame's LOD-cut scene that the tile's rays can meet.  A ray's L-infinity
// distance from the origin at parameter t is t |d|_max, so the casting
// kernel restarts each ray's march at the last integer plane of its dominant
// axis crossed before that distance: every cell the ray passes before it is
// empty for this ray, the cell holding the restart point is empty, and every
// hit is entered later through the planes the full march crosses -- the same
// first hit, entry plane and distance, without the traversal in front of it.
//
// The bound is a minimum over nodes of the selected DAGs, scattered to the
// tiles their screen rectangle covers:
//   * level 0 takes every chunk region of the frame table with its DAG root,
//     the box being the region's AABB of valid voxels;
//   * a node is projected in FP32 to a rectangle of tiles (box_rect, with
//     margins that cover its rounding); if the rectangle spans more tiles
//     than the refinement threshold and the node is not a 4^3 leaf, its
//     children (cell boxes clipped to the AABB) go to the next level's queue;
//     otherwise atomicMin(Dn[tile], its L-inf distance) over the rectangle.
//     A leaf uses the bounding box of its set voxels;
//   * a box that comes closer to the origin than 2/16 of the largest |d|
//     component covers every tile (rays reach it before camera depth 1/16);
//     any other box is projected from its part at depth >= 1/16, and dropped
//     if it has none or it lies beyond the view distance (a hit there is
//     reported as a miss anyway);
//   * a full queue makes the node scatter itself instead of its children.
// Every solid voxel a pixel ray meets lies in one scattered node whose
// rectangle holds that pixel's tile, so Dn[tile] is at most its distance.
//
// The bounds live in a pyramid (level 0: the tiles; level L: cells of
// 2^L x 2^L tiles): a node writes the finest level at which its rectangle
// spans at most 16 cells, and the casting kernel takes each tile's minimum
// over its cells.  Entries are 64-bit, (pass tag << 32) | bound, written by a
// non-returning atomic minimum; the tag counts down from pass to pass, so an
// entry of this pass always beats one left by an earlier pass, and readers
// take entries of another tag as "nothing solid": the pyramid is never reset.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cooperative_groups.h>

#include "aok_internal.h"
#include "aok_select.cuh"

namespace cg = cooperative_groups;
using namespace aok;

namespace {

constexpr int kBeamThreads = 256;      // block size of the cooperative walk
constexpr int kBeamNarrowThreads = 128;  // block size of the walk that shares SMs with a cast
constexpr int kBeamBlocksPerSM = 2;    // blocks per SM of the full grid (walks over many regions)
constexpr uint32_t kWideWalkRegions = 4096;  // above this many regions a pass takes the full grid; below,
                                             // one block per SM, which can start beside a running cast
constexpr double kNearS = 1.0 / 16.0;  // camera-depth plane the projection clips at
constexpr uint32_t kNoItem = 0xFFFFFFFFu;  // an empty queue slot
constexpr int kMaxBeamDevices = 128;

// Screen rectangle [x, z) x [y, w) of tiles a box (relative to the origin)
// can cover from its part at camera depth s >= kNearS; false if none.
// q = Af p in FP32 errs by at most dl = 8 2^-24 max_i sum_j |Af_ij| |p_j|
// (rounding of p, of Af and of the products and sums).  A box wholly in front
// of the plane is bounded by its corners' projections (their hull holds the
// box's), widened by the error that dl and the division carry; a box that
// straddles it by u = q_x / q_s over q_x in [X0, X1] and q_s in [kNearS, S1],
// each widened by dl.  Then a 0.5 pixel margin for the FP32 pixel rays.
__device__ bool box_rect(const BeamView& K, const float lo[3], const float hi[3], int4& rc) {
    float pm[3];
#pragma unroll
    for (int a = 0; a < 3; a++) pm[a] = fmaxf(fabsf(lo[a]), fabsf(hi[a]));
    float M = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; i++)
        M = fmaxf(M, fabsf(K.Af[3 * i]) * pm[0] + fabsf(K.Af[3 * i + 1]) * pm[1] + fabsf(K.Af[3 * i + 2]) * pm[2]);
    const float dl = M * 4.8e-7f + 1e-6f;
    float X0 = 3e38f, X1 = -3e38f, Y0 = 3e38f, Y1 = -3e38f, S0 = 3e38f, S1 = -3e38f;
    float u0 = 3e38f, u1 = -3e38f, v0 = 3e38f, v1 = -3e38f;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const float p0 = (k & 1) ? hi[0] : lo[0], p1 = (k & 2) ? hi[1] : lo[1], p2 = (k & 4) ? hi[2] : lo[2];
        const float qx = K.Af[0] * p0 + K.Af[1] * p1 + K.Af[2] * p2;
        const float qy = K.Af[3] * p0 + K.Af[4] * p1 + K.Af[5] * p2;
        const float qs = K.Af[6] * p0 + K.Af[7] * p1 + K.Af[8] * p2;
        X0 = fminf(X0, qx); X1 = fmaxf(X1, qx);
        Y0 = fminf(Y0, qy); Y1 = fmaxf(Y1, qy);
        S0 = fminf(S0, qs); S1 = fmaxf(S1, qs);
        if (qs > 0.0f) {
            const float r = 1.0f / qs;
            u0 = fminf(u0, qx * r); u1 = fmaxf(u1, qx * r);
            v0 = fminf(v0, qy * r); v1 = fmaxf(v1, qy * r);
        }
    }
    const float near_s = (float)kNearS;
    if (S1 + dl < near_s) return false;  // wholly behind the plane: only the near rule can reach it
    float a0, a1, b0, b1;
    if (S0 - dl >= near_s) {
        const float um = fmaxf(fabsf(u0), fabsf(u1)) * 1.001f, vm = fmaxf(fabsf(v0), fabsf(v1)) * 1.001f;
        const float mu = dl * (1.0f + um) / (S0 - dl) + um * 4.8e-7f;
        const float mv = dl * (1.0f + vm) / (S0 - dl) + vm * 4.8e-7f;
        a0 = u0 - mu; a1 = u1 + mu;
        b0 = v0 - mv; b1 = v1 + mv;
    } else {
        const float Xl = X0 - dl, Xh = X1 + dl, Yl = Y0 - dl, Yh = Y1 + dl, Sh = S1 + dl;
        a0 = fminf(Xl / near_s, Xl / Sh); a1 = fmaxf(Xh / near_s, Xh / Sh);
        b0 = fminf(Yl / near_s, Yl / Sh); b1 = fmaxf(Yh / near_s, Yh / Sh);
        a0 -= fabsf(a0) * 1e-6f; a1 += fabsf(a1) * 1e-6f;
        b0 -= fabsf(b0) * 1e-6f; b1 += fabsf(b1) * 1e-6f;
    }
    // pixel-centre coordinates of the pixel rays (the inverse of ray_dir), 0.5 pixel margin
    const float x0 = (a0 / K.U + 1.0f) * 0.5f * K.W - 1.0f, x1 = (a1 / K.U + 1.0f) * 0.5f * K.W;
    const float y0 = (1.0f - b1 / K.V) * 0.5f * K.H - 1.0f, y1 = (1.0f - b0 / K.V) * 0.5f * K.H;
    if (!(x1 >= 0.0f) || !(y1 >= 0.0f) || !(x0 < (float)K.W) || !(y0 < (float)K.H)) return false;
    rc.x = (int)fmaxf(floorf(x0 * (1.0f / kBeamTileW)), 0.0f);
    rc.y = (int)fmaxf(floorf(y0 * (1.0f / kBeamTileH)), 0.0f);
    rc.z = (int)fminf(floorf(x1 * (1.0f / kBeamTileW)) + 1.0f, (float)K.tiles_x);
    rc.w = (int)fminf(floorf(y1 * (1.0f / kBeamTileH)) + 1.0f, (float)K.tiles_y);
    return rc.z > rc.x && rc.w > rc.y;
}

// Occupied extent [lo, hi) of a 4^3 leaf mask along each axis (bit = x + 4y + 16z).
__device__ __forceinline__ void leaf_extent(uint64_t m, int lo[3], int hi[3]) {
    uint64_t t = m | (m >> 32);
    t |= t >> 16;
    const uint64_t tz = t;  // z folded
    t |= t >> 8;
    t |= t >> 4;
    const uint32_t xo = (uint32_t)(t & 0xFu);
    uint64_t ty = tz | (tz >> 2);
    ty |= ty >> 1;
    const uint32_t yo = (uint32_t)((ty & 1u) | ((ty >> 3) & 2u) | ((ty >> 6) & 4u) | ((ty >> 9) & 8u));
    uint64_t q = m | (m >> 8);
    q |= q >> 4;
    q |= q >> 2;
    q |= q >> 1;
    const uint32_t zo = (uint32_t)((q & 1u) | ((q >> 15) & 2u) | ((q >> 30) & 4u) | ((q >> 45) & 8u));
    const uint32_t o[3] = {xo, yo, zo};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        lo[a] = __ffs(o[a]) - 1;
        hi[a] = 32 - __clz(o[a]);
    }
}

// A node's box (the box of its solid voxels the device header carries, in
// 16ths of the cell, or a leaf's set voxels), its L-inf distance from the
// origin and screen rectangle.  A region root's box is also clipped to the
// region's AABB (clip, ref: the region's entry; below the roots a node's
// solid voxels lie in that AABB already, so the clip would only trim the
// rounding to 16ths).  hdr: the
// interior node's header word, loaded here.  Returns false if the node cannot
// meet any pixel ray.
__device__ __forceinline__ bool node_bound(const BeamView& V, int lod, bool clip, const ChunkRef& ref, uint32_t chunk,
                                           uint32_t node, uint32_t packed_cell, int s, int4& rc, int32_t& D,
                                           uint32_t& hdr) {
    const SceneDev& S = V.scene;
    const bool leaf = s == lod + 2;
    int32_t u[3];
    u[0] = (int32_t)(chunk % (uint32_t)S.grid[0]);
    u[1] = (int32_t)((chunk / (uint32_t)S.grid[0]) % (uint32_t)S.grid[1]);
    u[2] = (int32_t)(chunk / ((uint32_t)S.grid[0] * (uint32_t)S.grid[1]));
    const int32_t cell[3] = {(int32_t)(packed_cell & 1023u), (int32_t)((packed_cell >> 10) & 1023u),
                             (int32_t)((packed_cell >> 20) & 1023u)};
    int32_t blo[3], bhi[3];
    if (leaf) {
        int l[3], h[3];
        leaf_extent(S.leaves[node], l, h);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            blo[a] = cell[a] + (l[a] << lod);
            bhi[a] = cell[a] + (h[a] << lod);
        }
    } else {
        hdr = __ldg(S.nodes + node);
        const uint32_t q = hdr >> 8;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int32_t ql = (int32_t)((q >> (8 * a)) & 15u), qh = (int32_t)((q >> (8 * a + 4)) & 15u) + 1;
            blo[a] = cell[a] + ((ql << s) >> 4);
            bhi[a] = cell[a] + (((qh << s) + 15) >> 4);
            if (clip) {
                blo[a] = max(blo[a], (int32_t)ref.aabb[a]);
                bhi[a] = min(bhi[a], (int32_t)ref.aabb[3 + a]);
            }
        }
    }
    // L-inf distance from the origin (exact, numerator units: |values| < 2^30)
    int32_t wl[3], wh[3];
    int32_t dmax = 0;
    float e2 = 0.0f;
    bool empty = false;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        empty = empty || blo[a] >= bhi[a];
        wl[a] = (((u[a] << S.mlog) + blo[a]) << kFix) - V.O[a];
        wh[a] = (((u[a] << S.mlog) + bhi[a]) << kFix) - V.O[a];
        const int32_t da = wl[a] > 0 ? wl[a] : (wh[a] < 0 ? -wh[a] : 0);
        dmax = max(dmax, da);
        e2 += (float)da * (float)da;
    }
    D = dmax;
    if (empty || (V.view_num > 0.0f && sqrtf(e2) > V.view_num)) return false;
    if ((float)D < V.near_dn) {
        rc = make_int4(0, 0, V.tiles_x, V.tiles_y);
        return true;
    }
    const float sc = 1.0f / (1 << kFix);
    const float lf[3] = {(float)wl[0] * sc, (float)wl[1] * sc, (float)wl[2] * sc};
    const float hf[3] = {(float)wh[0] * sc, (float)wh[1] * sc, (float)wh[2] * sc};
    return box_rect(V, lf, hf, rc);
}

// Atomic minimum without a return value (a reduction the SM does not wait for).
__device__ __forceinline__ void red_min_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.global.min.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// D into the finest level L of the view's bound pyramid (level 0: the tiles;
// level L: cells of 2^L x 2^L tiles) at which the rectangle spans at most 16
// cells (or the coarsest); the casting kernels take each tile's minimum over
// its cells.
__device__ __forceinline__ void scatter_bound(const BeamView& V, uint32_t tag, const int4& rc, int32_t D) {
    int L = 0;
    int x0 = rc.x, y0 = rc.y, x1 = rc.z - 1, y1 = rc.w - 1;
    while (L < kBeamPyr - 1 && (x1 - x0 + 1) * (y1 - y0 + 1) > 16) {
        L++;
        x0 >>= 1; y0 >>= 1; x1 >>= 1; y1 >>= 1;
    }
    unsigned long long* lv = V.bounds + beam_level_offset((uint32_t)V.tiles_x, (uint32_t)V.tiles_y, L);
    const int wl = (V.tiles_x + (1 << L) - 1) >> L;
    const unsigned long long v = ((unsigned long long)tag << 32) | (uint32_t)D;
    for (int y = y0; y <= y1; y++)
        for (int x = x0; x <= x1; x++) red_min_u64(&lv[(size_t)y * wl + x], v);
}

// A checked pass (P.ck.err set) that meets a node or leaf index outside its
// pool: the error code goes into the error word and the view is bounded by 0
// (no ray of it skips anything), in place of the loads.
__device__ __noinline__ void bad_index(const BeamBatch& P, const BeamView& V, uint32_t code) {
    atomicOr(P.ck.err, code);
    scatter_bound(V, P.tag, make_int4(0, 0, V.tiles_x, V.tiles_y), 0);
}

// Children of interior node `node` (side 2^s) at cell c: {pointer, packed cell}.
__device__ __forceinline__ uint32_t node_children(const SceneDev& S, uint32_t node, uint32_t packed_cell, int s,
                                                  uint32_t ch[8], uint32_t cc[8], uint32_t hdr) {
    const uint32_t m0 = hdr & 0xFFu;
    const uint32_t k = (uint32_t)__popc(m0);
    const uint32_t h = 1u << (s - 1);
    const uint32_t cx0 = packed_cell & 1023u, cy0 = (packed_cell >> 10) & 1023u, cz0 = (packed_cell >> 20) & 1023u;
    uint32_t m = m0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        ch[j] = (uint32_t)j < k ? __ldg(S.nodes + node + 2 + 2 * j) : 0u;
        const int oct = m ? __ffs(m) - 1 : 0;
        m &= m - 1;
        cc[j] = (cx0 + ((oct & 1) ? h : 0u)) | ((cy0 + ((oct & 2) ? h : 0u)) << 10) | ((cz0 + ((oct & 4) ? h : 0u)) << 20);
    }
    return k;
}

// The whole pass in one cooperative launch (every block resident): the
// levels of the walk over all views with a grid-wide barrier after each,
// ending at the first level that queued nothing.  Level 0 takes every view's
// chunk regions; every lane of a warp runs the same iterations (the queue
// reservation is warp-wide).  A queued item carries what its node's bound
// needs (region, node, cell, side, view, LOD), so a level's chain of
// dependent loads starts at the item itself; each thread loads its first
// item beside the level's count and the next one while it works on the
// current one.  Queues are read through L2 (written by other SMs before the
// barrier).  Bounds carry the pass's tag, so nothing has to be reset before
// the walk or folded after it.
__device__ __forceinline__ void beam_walk(const BeamBatch& P) {
    cg::grid_group g = cg::this_grid();
    __shared__ uint32_t hist[kBeamLevels];
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    const int lane = (int)(threadIdx.x & 31u);
    if (threadIdx.x < kBeamLevels) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int level = 0; level < kBeamLevels - 1; level++) {
        const uint4* qin = P.q[level & 1];
        uint4* qout = P.q[(level + 1) & 1];
        // level 0 (the regions, few): one warp per block first, so that its
        // selection and root projections spread over the SMs
        const uint32_t first = level == 0 ? (((threadIdx.x >> 5) * gridDim.x + blockIdx.x) << 5) : (gtid & ~31u);
        uint4 nxt = make_uint4(kNoItem, 0u, 0u, 0u);
        if (level > 0 && first + (uint32_t)lane < P.cap) nxt = __ldcg(qin + first + lane);
        const uint32_t n = level == 0 ? P.n_regions : min(*(volatile uint32_t*)&P.cnt[level], P.cap);
        if (n == 0) break;  // the same value in every thread after the barrier
        for (uint32_t base = first; base < n; base += stride) {
            const uint32_t i = base + (uint32_t)lane;
            uint32_t kids = 0, ch[8], cc[8];
            uint4 it = make_uint4(kNoItem, 0u, 0u, 0u);
            bool clip = false;
            ChunkRef ref;
            if (i < n) {
                if (level == 0) {
                    // the view holding region item i: the last with region_begin <= i
                    uint32_t lo = 0, hi = P.n_views - 1;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if (P.v[mid].region_begin <= i) lo = mid;
                        else hi = mid - 1;
                    }
                    const uint32_t r = i - P.v[lo].region_begin;
                    // a pass that selects first writes the region's frame entry here
                    ref = P.select ? select_one(P.v[lo].scene, P.cam, const_cast<ChunkRef*>(P.v[lo].frame), nullptr,
                                                nullptr, nullptr, (int)r)
                                   : P.v[lo].frame[r];
                    if (ref.root != kNone)
                        it = make_uint4(r, ref.root, 0u,
                                        (uint32_t)P.v[lo].scene.mlog | (lo << 8) | ((uint32_t)ref.lod << 16));
                    clip = true;
                } else {
                    it = nxt;
                }
            }
            if (level > 0) {
                const uint32_t j = i + stride;
                nxt = make_uint4(kNoItem, 0u, 0u, 0u);
                if (j < n) nxt = __ldcg(qin + j);
            }
            const uint32_t vi = (it.w >> 8) & 0xFFu;
            const int s = (int)(it.w & 0xFFu), lod = (int)((it.w >> 16) & 0xFFu);
            const BeamView& V = P.v[it.x != kNoItem ? vi : 0u];
            if (it.x != kNoItem) {
                atomicAdd(&hist[min(V.scene.mlog - s, kBeamLevels - 1)], 1u);
                int4 rc;
                int32_t D;
                uint32_t hdr = 0;
                if (P.ck.err && (s == lod + 2 ? it.y >= P.ck.n_leaves : (uint64_t)it.y + 2 > P.ck.n_nodes)) {
                    bad_index(P, V, s == lod + 2 ? 2u : 1u);
                } else if (node_bound(V, lod, clip, ref, it.x, it.y, it.z, s, rc, D, hdr)) {
                    const uint32_t area = (uint32_t)(rc.z - rc.x) * (uint32_t)(rc.w - rc.y);
                    if (s > lod + 2 && area > P.expand && s > P.smin) {
                        if (P.ck.err && (uint64_t)it.y + 2 + 2 * __popc(hdr & 0xFFu) > P.ck.n_nodes)
                            bad_index(P, V, 1u);
                        else
                            kids = node_children(V.scene, it.y, it.z, s, ch, cc, hdr);
                    } else {
                        scatter_bound(V, P.tag, rc, D);
                    }
                }
            }
            // queue the children: one reservation per warp
            uint32_t pre = kids;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, pre, o);
                if (lane >= o) pre += v;
            }
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, pre, 31);
            uint32_t wbase = 0;
            if (total) {
                if (lane == 31) wbase = atomicAdd(&P.cnt[level + 1], total);
                wbase = __shfl_sync(0xFFFFFFFFu, wbase, 31);
            }
            if (kids) {
                const uint32_t at = wbase + pre - kids;
                if (at + kids <= P.cap) {
#pragma unroll
                    for (int q = 0; q < 8; q++)
                        if ((uint32_t)q < kids) qout[at + q] = make_uint4(it.x, ch[q], cc[q], it.w - 1);
                } else {
                    // queue full: this node stands for its children; its slots
                    // below the capacity are marked empty
                    for (uint32_t q = at; q < P.cap && q < at + kids; q++) qout[q] = make_uint4(kNoItem, 0u, 0u, 0u);
                    int4 rc;
                    int32_t D;
                    uint32_t hdr;
                    if (node_bound(V, lod, clip, ref, it.x, it.y, it.z, s, rc, D, hdr)) scatter_bound(V, P.tag, rc, D);
                }
            }
        }
        g.sync();
    }
    __syncthreads();
    if (threadIdx.x < kBeamLevels && hist[threadIdx.x]) atomicAdd(&P.hist[threadIdx.x], hist[threadIdx.x]);
}

__global__ void __launch_bounds__(kBeamThreads) beam_kernel(const __grid_constant__ BeamBatch P) { beam_walk(P); }

// The same walk as one block of kBeamNarrowThreads per SM with at most 80
// registers: it fits beside six blocks of a running cast (7 x 128 threads x
// 72 registers per SM), so a pipelined frame's pass can start on an SM as
// soon as one casting block of the frame before retires there instead of
// after the cast.  Alone it is slower (half the threads).
__global__ void __maxnreg__(80) beam_kernel_narrow(const __grid_constant__ BeamBatch P) { beam_walk(P); }

}  // namespace

extern "C" {

unsigned aokk_beam_grid(int sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, beam_kernel, kBeamThreads, 0) != cudaSuccess ||
        per_sm < 1)
        return 0;
    return (unsigned)(sms > 0 ? sms : 1) * (unsigned)(per_sm < kBeamBlocksPerSM ? per_sm : kBeamBlocksPerSM);
}

bool aokk_beam_view(const SceneDev* S, const CamDev* C, const ChunkRef* frame, unsigned long long* bounds,
                    BeamView* out) {
    // A = [c0, c1, -c2] with d_i = R[3i] u + R[3i+1] v - R[3i+2]
    double A[9];
    for (int i = 0; i < 3; i++) {
        A[3 * i + 0] = C->R[3 * i + 0];
        A[3 * i + 1] = C->R[3 * i + 1];
        A[3 * i + 2] = -(double)C->R[3 * i + 2];
    }
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    double nrm = 0.0;
    for (int i = 0; i < 9; i++) nrm = fmax(nrm, fabs(A[i]));
    if (!(std::isfinite(det) && fabs(det) > 1e-6 * nrm * nrm * nrm)) return false;
    const double id = 1.0 / det;
    double Ai[9];
    Ai[0] = (A[4] * A[8] - A[5] * A[7]) * id;
    Ai[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    Ai[3] = (A[5] * A[6] - A[3] * A[8]) * id;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    Ai[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    Ai[6] = (A[3] * A[7] - A[4] * A[6]) * id;
    Ai[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    BeamView& K = *out;
    std::memset(&K, 0, sizeof(K));
    K.scene = *S;
    K.frame = frame;
    K.bounds = bounds;
    for (int i = 0; i < 9; i++) K.Af[i] = (float)Ai[i];
    const double U = (double)C->tan_half * (double)C->W / (double)C->H, V = (double)C->tan_half;
    K.U = (float)U;
    K.V = (float)V;
    // largest |d| component over the screen, with slack for the FP32 ray arithmetic
    double dmax = 0.0;
    for (int i = 0; i < 3; i++) dmax = fmax(dmax, fabs(A[3 * i]) * U + fabs(A[3 * i + 1]) * V + fabs(A[3 * i + 2]));
    K.near_dn = (float)(2.0 * kNearS * dmax * 1.01 * (double)(1 << kFix));
    K.view_num = S->view_dist > 0.0f ? (float)(((double)S->view_dist * 1.00001 + 1.0) * (double)(1 << kFix)) : 0.0f;
    K.W = C->W;
    K.H = C->H;
    K.tiles_x = (C->W + kBeamTileW - 1) / kBeamTileW;
    K.tiles_y = (C->H + kBeamTileH - 1) / kBeamTileH;
    for (int a = 0; a < 3; a++) K.O[a] = C->O[a];
    return true;
}

// Beam passes of this process run one after another on each device: a pass
// waits for the previous one, whatever stream either was launched on, so that
// two cooperative launches that each fill the GPU never wait for each other's
// blocks.
static std::mutex g_beam_mu;
static cudaEvent_t g_beam_done[kMaxBeamDevices];

// The pass as a node of a CUDA graph (aokk_batch_run): its kernel with the
// launch shape aokk_beam_run uses, and the memset of the counters that
// aokk_beam_run zeroes before it.  argp: one slot, valid until the node is set.
void aokk_beam_node(const BeamBatch* P, unsigned grid, void** argp, cudaKernelNodeParams* kp, cudaMemsetParams* zero) {
    argp[0] = (void*)P;
    kp->func = (void*)beam_kernel;
    kp->gridDim = dim3(P->n_regions > kWideWalkRegions ? grid : (grid + kBeamBlocksPerSM - 1) / kBeamBlocksPerSM);
    kp->blockDim = dim3(kBeamThreads);
    kp->sharedMemBytes = 0;
    kp->kernelParams = argp;
    kp->extra = nullptr;
    zero->dst = P->cnt;
    zero->pitch = 0;
    zero->value = 0;
    zero->elementSize = sizeof(uint32_t);
    zero->width = 2 * kBeamLevels;
    zero->height = 1;
}

// The per-device order of beam passes for work that holds passes but is not
// launched by aokk_beam_run (a graph): before (record = 0) the stream waits
// for the previous pass; after (record = 1) the end of the stream's work so
// far becomes the point the next pass waits for.
int aokk_beam_order(void* stream, int record) {
    const cudaStream_t st = (cudaStream_t)stream;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return aokk_status(e);
    if (dev < 0 || dev >= kMaxBeamDevices) return aokk_status(cudaErrorInvalidDevice);
    std::lock_guard<std::mutex> lk(g_beam_mu);
    if (!g_beam_done[dev]) e = cudaEventCreateWithFlags(&g_beam_done[dev], cudaEventDisableTiming);
    if (e == cudaSuccess) e = record ? cudaEventRecord(g_beam_done[dev], st) : cudaStreamWaitEvent(st, g_beam_done[dev], 0);
    return aokk_status(e);
}

int aokk_beam_run(const BeamBatch* P, unsigned grid, void* stream, int narrow) {
    const cudaStream_t st = (cudaStream_t)stream;
    if (P->n_views == 0) return AOK_OK;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return aokk_status(e);
    if (dev < 0 || dev >= kMaxBeamDevices) return aokk_status(cudaErrorInvalidDevice);
    std::lock_guard<std::mutex> lk(g_beam_mu);
    if (!g_beam_done[dev]) e = cudaEventCreateWithFlags(&g_beam_done[dev], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g_beam_done[dev], 0);
    // queue counts and the walk histogram (cnt and hist are adjacent)
    if (e == cudaSuccess) e = cudaMemsetAsync(P->cnt, 0, 2 * kBeamLevels * sizeof(uint32_t), st);
    void* args[] = {(void*)P};
    const bool wide = P->n_regions > kWideWalkRegions;
    const unsigned g = wide ? grid : (grid + kBeamBlocksPerSM - 1) / kBeamBlocksPerSM;
    if (e == cudaSuccess) {
        if (narrow && !wide)  // one narrow block per SM
            e = cudaLaunchCooperativeKernel((const void*)beam_kernel_narrow, g, kBeamNarrowThreads, args, 0, st);
        else
            e = cudaLaunchCooperativeKernel((const void*)beam_kernel, g, kBeamThreads, args, 0, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(g_beam_done[dev], st);
    return aokk_status(e);
}

}  // extern "C"
