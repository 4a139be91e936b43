// Device-side ray casting shared by the kernels of the per-ray chunk march
// and of the tile-chunk pipeline: exact plane-crossing comparisons, the
// pixel ray, and the first-hit traversal of one chunk's sparse voxel DAG
// (Aokana Sec. 3.4-3.5).
//
// Exactness.  The ray is origin + t d with the origin on a 2^-12 grid and d
// an FP32 vector.  Every ordering decision of the traversal (which face a
// cell is left through, which child octant holds the entry point) compares
// two plane-crossing parameters t_a = (P_a - o_a) / d_a.  The traversal works
// in a frame mirrored so that every d_a >= 0, writes N_a = (P_a - o_a) 2^12 as
// an int32 and |d_a| = m_a 2^E_a (24-bit mantissa), and decides
// t_a < t_b  <=>  N_a m_b 2^(E_b - E_a) < N_b m_a  with 64-bit products and an
// exact shift comparison.  No decision is approximated, so the hit voxel,
// LOD, material and normal equal those of the exact real ray; only the
// reported distance is rounded (FP32, relative error ~1e-7).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "aok_internal.h"

namespace aok {

// ---------------------------------------------------------------------------
// exact comparison of plane-crossing parameters
// ---------------------------------------------------------------------------
// N1 / (m1 2^E1) < N2 / (m2 2^E2), s = E2 - E1, m1, m2 > 0, |N| < 2^31, m < 2^24.
__device__ __forceinline__ bool tlt(int32_t N1, int32_t m1, int32_t N2, int32_t m2, int32_t s) {
    const long long P = (long long)N1 * m2;
    const long long Q = (long long)N2 * m1;
    if (s >= 0) {
        // P 2^s < Q  <=>  P <= floor((Q - 1) / 2^s)
        return P <= ((Q - 1) >> min(s, 63));
    }
    // P 2^s < Q  <=>  floor(P / 2^-s) < Q
    return (P >> min(-s, 63)) < Q;
}

// |d| = m 2^E; a zero component becomes m = 1, E = -400 (crossings at +-infinity).
__device__ __forceinline__ void decompose(float d, int32_t& m, int32_t& E) {
    const uint32_t b = __float_as_uint(d) & 0x7FFFFFFFu;
    const uint32_t ex = b >> 23, man = b & 0x7FFFFFu;
    if (b == 0) { m = 1; E = -400; }
    else if (ex == 0) { m = (int32_t)man; E = -149; }
    else { m = (int32_t)(man | 0x800000u); E = (int32_t)ex - 150; }
}

// floor(x) of a real x from an FP32 estimate p with |p - x| <= err: when no
// integer lies within err of p, floor(p) == floor(x) (p - floor(p) and
// floor(p) + 1 - p are exact for the magnitudes used here).  False when an
// integer is that close: the caller then decides with exact comparisons.
__device__ __forceinline__ bool floor_if_clear(float p, float err, int32_t& f) {
    const float fl = floorf(p);
    if (!(p - fl > err && fl + 1.0f - p > err)) return false;
    f = (int32_t)fl;
    return true;
}

// Ray direction of pixel (px, py): IEEE binary32, one rounding per operation.
__device__ __forceinline__ void ray_dir(const CamDev& c, int px, int py, float d[3]) {
    const float fW = __int2float_rn(c.W), fH = __int2float_rn(c.H);
    const float a = __int2float_rn(2 * px + 1);
    const float b = __fdiv_rn(a, fW);
    const float cc = __fsub_rn(b, 1.0f);
    const float e = __fmul_rn(cc, c.tan_half);
    const float aspect = c.aspect;  // fW / fH, rounded once (on the host)
    const float u = __fmul_rn(e, aspect);
    const float a2 = __int2float_rn(2 * py + 1);
    const float b2 = __fdiv_rn(a2, fH);
    const float c2 = __fsub_rn(1.0f, b2);
    const float v = __fmul_rn(c2, c.tan_half);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float p = __fmul_rn(c.R[3 * i + 0], u);
        const float q = __fmul_rn(c.R[3 * i + 1], v);
        const float s = __fadd_rn(p, q);
        d[i] = __fsub_rn(s, c.R[3 * i + 2]);
    }
}

// ---------------------------------------------------------------------------
// per-chunk DAG traversal in the chunk's mirrored local frame
// ---------------------------------------------------------------------------
// FAST rays: the exponents of the non-zero |d| components span <= 6, so the
// mantissas are shifted to a common exponent (m < 2^30, zero components get
// m = 0, i.e. crossings at +-infinity) and t_a < t_b <=> N_a m_b < N_b m_a;
// other rays keep (m, E) per axis and use tlt().
template <bool FAST>
__device__ __forceinline__ bool tltf(int32_t N1, int32_t m1, int32_t N2, int32_t m2, int32_t s) {
    if (FAST) return (long long)N1 * m2 < (long long)N2 * m1;
    return tlt(N1, m1, N2, m2, s);
}

// Cells are addressed by level k (side 2^k LOD-0 units) and mirrored integer
// coordinates c.  Levels R = log2(M) (root) .. n+3 are interior nodes, n+2 a
// 4x4x4 leaf block, n+1 a 2x2x2 group in it, n a voxel of LOD n.  Leaf bits
// are addressed in stored (unmirrored) order: along a mirrored axis the index
// inside a block is c ^ 3 (group: c ^ 1).
// Colour of DFS index idx in a colour-block array (Sec. 3.3) at base:
// [nt][nt x uint32: block holding entry 128 j][nblocks x uint32 first index]
// [nblocks x uint8 colour].  The block is the last one whose first index is
// <= idx (Sec. 3.5: a binary search), searched between the blocks holding
// entries 128 (idx / 128) and 128 (idx / 128 + 1), so that a hit costs a few
// dependent loads instead of log2(nblocks).
static __device__ __forceinline__ uint32_t block_colour(const uint8_t* __restrict__ base, uint32_t nblocks,
                                                        uint32_t idx) {
    const uint32_t* __restrict__ w = reinterpret_cast<const uint32_t*>(base);
    const uint32_t nt = w[0], j = idx >> 7;
    uint32_t lo = w[1 + j];
    uint32_t hi = j + 1 < nt ? w[2 + j] : nblocks - 1;
    const uint32_t* __restrict__ first = w + 1 + nt;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (first[mid] <= idx) lo = mid;
        else hi = mid - 1;
    }
    return base[4ull * (1 + nt + nblocks) + lo];
}

struct RayState {
    float d[3];
    int32_t m[3], E[3];
    uint32_t mir;
};

struct HitRec {
    int32_t c[3];       // voxel index (mirrored, chunk-local, voxel units of the LOD)
    int e;              // entry axis (3 = origin inside)
    int32_t Ne;         // entry plane numerator
    uint32_t idx;       // depth-first index of the voxel in its DAG (Sec. 3.3)
};

// Material of a hit: the entry of its DFS index in the (chunk, LOD)'s colour
// array or colour blocks (the colour resolve of Sec. 3.5).
__device__ __forceinline__ uint32_t hit_material(const SceneDev& S, const ChunkRef& ref, uint32_t idx) {
    return ref.nblocks == 0 ? S.mats[ref.mat_base + idx] : block_colour(S.mats + ref.mat_base, ref.nblocks, idx);
}

struct Counters {
    uint32_t v_int, v_leaf, rbytes;
};

// Returns true on a hit inside this chunk.  (e, Ne): entry plane into the chunk
// (e = 3: the origin lies inside the chunk).  Oloc: mirrored local origin numerators.
// BEAM: the entry plane (e, Ne) may lie inside the chunk (a restart of the
// march past the beam's bound, trace_pixel_t), so the descent compares it
// with the entry axis' mid planes as well.
// In a checked build (CHECK) every pool index is tested before its load; an
// index out of range ORs its code into *ck.err and ends the chunk's traversal
// as a miss.
template <bool CHECK>
__device__ __forceinline__ bool out_of(uint64_t i, uint64_t n, const CheckDev* ck, uint32_t code) {
    if (CHECK && i >= n) {
        atomicOr(ck->err, code);
        return true;
    }
    return false;
}

// (the per-level stack is written on entering a level, before any read: the
// compiler cannot see that through the level index)
#pragma nv_diag_suppress 549
template <bool FAST, bool COUNT, bool CHECK = false, bool BEAM = false>
__device__ __forceinline__ bool trace_chunk(const SceneDev& S, const ChunkRef& ref, const RayState& r,
                                            const int32_t Oloc[3], int e, int32_t Ne, HitRec& hit, Counters& cnt,
                                            const CheckDev* ck = nullptr) {
    const uint32_t* __restrict__ nodes = S.nodes;
    const int R = S.mlog;
    const int n = (int)ref.lod;
    // per interior level j (3 <= j <= R) on the path: {node word index, child
    // mask} in st[j - 3] (a level is written when the path enters it, before
    // any read); the parent of the current level's cells is also kept in
    // registers (pidx and its mask pm8)
    uint2 st[kMaxLevels - 3];
    uint32_t pidx = 0;
    int k = R;
    int32_t c0 = 0, c1 = 0, c2 = 0;
    int32_t me = 1, Ee = 0;
    if (e < 3) { me = r.m[e]; Ee = r.E[e]; }
    uint64_t lmu = 0;
    const int f1 = (r.mir & 1u) ? 1 : 0, f2 = (r.mir & 2u) ? 1 : 0, f4 = (r.mir & 4u) ? 1 : 0;
    uint32_t pm8 = 0;   // parent's child mask, stored octant order (node mask / leaf groups / group voxels)
    uint32_t g8 = 0;    // group occupancy of the current leaf block
    bool occ = true;
    // Child masks of the occupied cell (k, c) into pm8: its node's mask
    // (interior levels, also pushed on the stack), its leaf block's group
    // occupancy (leaf level) or its 2x2x2 group's voxel bits.  False when a
    // checked build finds a pool index out of range.
    auto fetch = [&]() -> bool {
        if (k >= n + 2) {
            uint32_t idx;
            if (k == R) {
                idx = ref.root;
            } else {
                const uint32_t oct = ((uint32_t)(c0 & 1) | ((uint32_t)(c1 & 1) << 1) | ((uint32_t)(c2 & 1) << 2)) ^ r.mir;
                const uint64_t at = (uint64_t)pidx + 2 + 2 * __popc(pm8 & ((1u << oct) - 1u));
                if (out_of<CHECK>(at, ck ? ck->n_nodes : 0, ck, 1u)) return false;
                idx = nodes[at];
            }
            if (k >= n + 3) {
                if (out_of<CHECK>((uint64_t)idx + 1, ck ? ck->n_nodes : 0, ck, 1u)) return false;
                pm8 = nodes[idx] & 0xFFu;
                st[k - 3] = make_uint2(idx, pm8);
                pidx = idx;
                if (COUNT) cnt.v_int++;
            } else {
                if (out_of<CHECK>(idx, ck ? ck->n_leaves : 0, ck, 2u)) return false;
                lmu = S.leaves[idx];
                uint64_t t = lmu | (lmu >> 1);
                t |= t >> 4;
                t |= t >> 16;
                g8 = (uint32_t)((t & 1) | ((t >> 1) & 2) | ((t >> 6) & 4) | ((t >> 7) & 8) | ((t >> 28) & 16) |
                                ((t >> 29) & 32) | ((t >> 34) & 64) | ((t >> 35) & 128));
                pm8 = g8;
                if (COUNT) cnt.v_leaf++;
            }
        } else {
            // entering a 2x2x2 group of the leaf: its 8 voxel bits in octant order
            const uint64_t v = lmu >> (((c0 & 1) ^ f1) * 2 + ((c1 & 1) ^ f2) * 8 + ((c2 & 1) ^ f4) * 32);
            pm8 = (uint32_t)((v & 3) | ((v >> 2) & 0xC) | ((v >> 12) & 0x30) | ((v >> 14) & 0xC0));
        }
        return true;
    };
    if (FAST) {
        // First descent.  Until the first empty cell, every cell entered is
        // the one holding the entry point, so its coordinates at level j are
        // those of the entry point's voxel (level n) shifted right by j - n:
        // the voxel coordinates F are found once (a float estimate, then the
        // exact plane comparisons of the descent: a plane crossed no later
        // than the entry is passed), and the descent needs no comparison per
        // level.  F is clamped to the chunk as the per-level halving would.
        const int sh = n + kFix;
        const int32_t fmax = (1 << (R - n)) - 1;
        const float te = e < 3 ? __fdividef((float)Ne, (float)me) : 0.0f;
        int32_t F[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            int32_t f;
            if (e == 3 || r.m[a] == 0) {
                f = Oloc[a] >> sh;  // the origin's coordinate
            } else if (a == e) {
                f = (Ne + Oloc[a]) >> sh;  // on the entry plane
            } else {
                // p: the entry point's coordinate in voxels of the LOD.  Its
                // error is below 2^-21 of |Oloc| + |te m| (six roundings, the
                // quotient within 2 ulp): with a margin of 2, the floor of p
                // is exact unless p lies that close to an integer.
                const float fo = (float)Oloc[a], pr = te * (float)r.m[a];
                const float p = (fo + pr) * (1.0f / (float)(1 << sh));
                const float err = (fabsf(fo) + fabsf(pr)) * (1.0f / (float)(1 << sh)) * 0x1p-20f;
                const float pc = fminf(fmaxf(p, -1.0f), (float)fmax + 1.0f);
                if (!floor_if_clear(pc, err, f)) {
                    f = (int32_t)floorf(pc);
                    while (f < fmax && !tltf<FAST>(Ne, me, ((f + 1) << sh) - Oloc[a], r.m[a], 0)) f++;
                    while (f > 0 && tltf<FAST>(Ne, me, (f << sh) - Oloc[a], r.m[a], 0)) f--;
                }
            }
            F[a] = max(0, min(f, fmax));
        }
        for (;;) {
            if (!fetch()) return false;
            k--;
            c0 = F[0] >> (k - n);
            c1 = F[1] >> (k - n);
            c2 = F[2] >> (k - n);
            occ = (pm8 >> (((uint32_t)(c0 & 1) | ((uint32_t)(c1 & 1) << 1) | ((uint32_t)(c2 & 1) << 2)) ^ r.mir)) & 1u;
            if (!occ || k == n) break;
        }
    }
    for (;;) {
        if (occ) {
            if (k == n) break;  // the hit: its index is resolved after the loop
            if (!fetch()) return false;
            // child of cell (k, c) holding the entry point: compare t_entry with the mid planes
            const int kk = k - 1;
            const int32_t mid0 = ((2 * c0 + 1) << (kk + kFix)) - Oloc[0];
            const int32_t mid1 = ((2 * c1 + 1) << (kk + kFix)) - Oloc[1];
            const int32_t mid2 = ((2 * c2 + 1) << (kk + kFix)) - Oloc[2];
            const int32_t b0 = (e != 0) ? !tltf<FAST>(Ne, me, mid0, r.m[0], r.E[0] - Ee) : (BEAM && Ne >= mid0);
            const int32_t b1 = (e != 1) ? !tltf<FAST>(Ne, me, mid1, r.m[1], r.E[1] - Ee) : (BEAM && Ne >= mid1);
            const int32_t b2 = (e != 2) ? !tltf<FAST>(Ne, me, mid2, r.m[2], r.E[2] - Ee) : (BEAM && Ne >= mid2);
            c0 = 2 * c0 + b0;
            c1 = 2 * c1 + b1;
            c2 = 2 * c2 + b2;
            k = kk;
        } else {
            // leave cell (k, c) through its nearest exit face; while the
            // neighbour is an empty sibling in the same parent, keep going
            // (the exit planes of the level, advanced one cell per step)
            const int32_t side = 1 << (k + kFix);
            int32_t N0 = ((c0 + 1) << (k + kFix)) - Oloc[0];
            int32_t N1 = ((c1 + 1) << (k + kFix)) - Oloc[1];
            int32_t N2 = ((c2 + 1) << (k + kFix)) - Oloc[2];
            bool xy = tltf<FAST>(N0, r.m[0], N1, r.m[1], r.E[1] - r.E[0]);
            for (;;) {
                const int32_t Na = xy ? N0 : N1, ma = xy ? r.m[0] : r.m[1], Ea = xy ? r.E[0] : r.E[1];
                const bool az = tltf<FAST>(Na, ma, N2, r.m[2], r.E[2] - Ea);
                int ax;
                if (az) { ax = xy ? 0 : 1; Ne = Na; me = ma; Ee = Ea; }
                else { ax = 2; Ne = N2; me = r.m[2]; Ee = r.E[2]; }
                e = ax;
                int32_t cax;
                if (ax == 0) { cax = ++c0; N0 += side; }
                else if (ax == 1) { cax = ++c1; N1 += side; }
                else { cax = ++c2; N2 += side; }
                if ((cax << k) >= (1 << R)) return false;  // left the chunk
                if ((cax & 1) == 0) {
                    // left the parent: up as many levels as cax has trailing
                    // zero bits (fewer than R - k, as the chunk was not left)
                    const int p = __ffs(cax) - 1;
                    c0 >>= p; c1 >>= p; c2 >>= p;
                    k += p;
                    if (k >= n + 2) {  // popped into a new parent: a node ...
                        const uint2 par = st[k - 2];
                        pidx = par.x;
                        pm8 = par.y;
                    } else {
                        pm8 = g8;  // ... or the leaf block
                    }
                    break;
                }
                if ((pm8 >> (((uint32_t)(c0 & 1) | ((uint32_t)(c1 & 1) << 1) | ((uint32_t)(c2 & 1) << 2)) ^ r.mir)) & 1u)
                    break;  // an occupied sibling
                if (ax != 2) xy = tltf<FAST>(N0, r.m[0], N1, r.m[1], r.E[1] - r.E[0]);  // x against y changed
            }
        }
        // occupancy of cell (k, c) in its parent
        occ = (pm8 >> (((uint32_t)(c0 & 1) | ((uint32_t)(c1 & 1) << 1) | ((uint32_t)(c2 & 1) << 2)) ^ r.mir)) & 1u;
    }
    // The hit (k == n): the lanes that hit in this chunk resolve together.
    hit.c[0] = c0; hit.c[1] = c1; hit.c[2] = c2;
    hit.e = e;
    hit.Ne = Ne;
    // depth-first index (Sec. 3.3): per level of the path the summed counts
    // of the earlier children (the prefix word beside the child pointer in the
    // device layout), then the solid voxels before the hit bit in its leaf
    const int32_t side = (1 << (R - n)) - 1;
    const int32_t u0 = (r.mir & 1u) ? side - c0 : c0;
    const int32_t u1 = (r.mir & 2u) ? side - c1 : c1;
    const int32_t u2 = (r.mir & 4u) ? side - c2 : c2;
    uint32_t idx = 0;
    for (int j = R; j >= n + 3; j--) {
        const int sh = j - 1 - n;
        const int oct = ((u0 >> sh) & 1) | (((u1 >> sh) & 1) << 1) | (((u2 >> sh) & 1) << 2);
        const uint2 sj = st[j - 3];
        const int rk = __popc(sj.y & ((1u << oct) - 1u));
        const uint64_t at = (uint64_t)sj.x + 3 + 2 * rk;
        if (out_of<CHECK>(at, ck ? ck->n_nodes : 0, ck, 1u)) return false;
        idx += nodes[at];
        if (COUNT) cnt.rbytes += rk * ((j - 1 == n + 2) ? 8u : 4u);  // the paper-format resolve
    }
    const int bit = (u0 & 3) + 4 * (u1 & 3) + 16 * (u2 & 3);
    idx += (uint32_t)__popcll(lmu & ((1ull << bit) - 1ull));
    if (COUNT) cnt.rbytes += 1;
    hit.idx = idx;
    if (CHECK) {
        // raw array: the entry; blocks: the whole block structure
        const uint64_t end =
            ref.nblocks == 0 ? ref.mat_base + idx : ref.mat_base + 4ull * (1 + ((uint64_t)idx >> 7) + 1) - 1;
        if (out_of<CHECK>(end, ck->n_mats, ck, 4u)) return false;
        if (ref.nblocks) {
            const uint32_t nt = *reinterpret_cast<const uint32_t*>(S.mats + ref.mat_base);
            if (out_of<CHECK>(ref.mat_base + 4ull * (1 + nt + ref.nblocks) + ref.nblocks - 1, ck->n_mats, ck, 4u) ||
                out_of<CHECK>(idx >> 7, nt, ck, 4u))
                return false;
        }
    }
    return true;
}

#pragma nv_diag_default 549

// Entry face of a hit entered through an edge or a corner of its voxel (the
// voxel's lower faces of several axes crossed at the entry instant): the
// lowest of those axes, with its plane.  n: the hit's LOD; Oloc: the mirrored
// chunk-local origin numerators trace_chunk was given.
template <bool FAST>
__device__ __forceinline__ void lowest_entry_face(const RayState& r, const int32_t Oloc[3], int n, HitRec& hit) {
    const int e = hit.e;
    if (e == 0 || e == 3) return;
    const int32_t Ne = hit.Ne, me = r.m[e], Ee = r.E[e];
#pragma unroll
    for (int b = 1; b >= 0; b--) {
        if (b < e && r.d[b] != 0.0f) {
            const int32_t Nb = (hit.c[b] << (n + kFix)) - Oloc[b];
            if (!tltf<FAST>(Ne, me, Nb, r.m[b], r.E[b] - Ee) && !tltf<FAST>(Nb, r.m[b], Ne, me, Ee - r.E[b])) {
                hit.e = b;
                hit.Ne = Nb;
            }
        }
    }
}

// Exact test that the ray (t >= 0) meets the closed box of the chunk's solid
// voxels (ref.aabb), in the chunk's mirrored frame with origin numerators
// Oloc.  The counting build enters a chunk only then, so that its visit counts
// are the definition's (a chunk is entered iff the ray meets its AABB); the
// casting builds use a cheaper FP32 test with a margin, which may enter a
// chunk the ray passes within 1/16 voxel of without changing any hit.
template <bool FAST>
__device__ __noinline__ bool meets_aabb(const RayState& r, const int32_t Oloc[3], const ChunkRef& ref, int mlog) {
    const int32_t M = 1 << mlog;
    int32_t Nn = 0, mn = 1, En = 0;  // latest entry parameter so far: t = 0
    int32_t Hi[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const bool mir = (r.mir >> a) & 1u;
        const int32_t lo = mir ? M - (int32_t)ref.aabb[3 + a] : (int32_t)ref.aabb[a];
        const int32_t hi = mir ? M - (int32_t)ref.aabb[a] : (int32_t)ref.aabb[3 + a];
        const int32_t Lo = (lo << kFix) - Oloc[a];
        Hi[a] = (hi << kFix) - Oloc[a];
        if (r.d[a] == 0.0f) {
            if (Lo > 0 || Hi[a] < 0) return false;
        } else if (tltf<FAST>(Nn, mn, Lo, r.m[a], r.E[a] - En)) {
            Nn = Lo; mn = r.m[a]; En = r.E[a];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++)
        if (r.d[a] != 0.0f && tltf<FAST>(Hi[a], r.m[a], Nn, mn, En - r.E[a])) return false;
    return true;
}

// With a view distance, a hit farther than it is a miss (FP64, fixed order).
__device__ __forceinline__ bool within_view(const SceneDev& S, const RayState& r, const HitRec& hit) {
    if (S.view_dist <= 0.0f) return true;
    double dd = 0.0;
    if (hit.e < 3) {
        const double d0 = r.d[0], d1 = r.d[1], d2 = r.d[2];
        dd = (double)hit.Ne / (4096.0 * fabs((double)r.d[hit.e])) * sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
    return dd <= (double)S.view_dist;
}

// Write the output record of a hit that trace_chunk found in the chunk region
// u (unmirrored chunk coordinates) of the (chunk, LOD) ref; dn = |d| in FP32.
// Returns false (writes nothing) when the view distance turns the hit into a
// miss.
__device__ __forceinline__ bool emit_hit(const SceneDev& S, const RayState& r, const ChunkRef& ref, const int32_t u[3],
                                         const HitRec& hit, float dn, uint4* __restrict__ out_hit,
                                         float* __restrict__ out_t, size_t pix) {
    if (!within_view(S, r, hit)) return false;
    const uint32_t mat = hit_material(S, ref, hit.idx);
    // un-mirror the voxel index to world LOD-0 units
    const int n = (int)ref.lod;
    const int32_t side = (1 << (S.mlog - n)) - 1;
    int32_t wxyz[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int32_t uv = ((r.mir >> a) & 1u) ? side - hit.c[a] : hit.c[a];
        wxyz[a] = (u[a] << S.mlog) + (uv << n);
    }
    float dist = 0.0f;
    if (hit.e < 3) dist = __fdiv_rn((float)hit.Ne * (1.0f / 4096.0f), fabsf(r.d[hit.e])) * dn;
    const uint32_t normal = hit.e == 3 ? 7u : (uint32_t)(2 * hit.e) + ((r.mir >> hit.e) & 1u);
    out_hit[pix] = make_uint4((uint32_t)wxyz[0], (uint32_t)wxyz[1], (uint32_t)wxyz[2],
                              (uint32_t)n | (mat << 8) | (normal << 16) | (1u << 19));
    out_t[pix] = dist;
    return true;
}

__device__ __forceinline__ void emit_miss(uint4* __restrict__ out_hit, float* __restrict__ out_t, size_t pix) {
    out_hit[pix] = make_uint4(0u, 0u, 0u, 0xFFu | (7u << 16));
    out_t[pix] = __int_as_float(0x7F800000);
}

__device__ __forceinline__ float ray_norm(const RayState& r) {
    return sqrtf(__fadd_rn(__fadd_rn(__fmul_rn(r.d[0], r.d[0]), __fmul_rn(r.d[1], r.d[1])), __fmul_rn(r.d[2], r.d[2])));
}

// The beam-pass bound of pixel (px, py) of a W x H view: the minimum over
// its 8 x 4 tile's cells of the bound pyramid among entries of pass `tag`
// (INT32_MAX if there is none), 0 without bounds.
__device__ __forceinline__ int32_t beam_bound(const unsigned long long* __restrict__ b, uint32_t tag, int W, int H,
                                              int px, int py) {
    if (!b) return 0;
    const uint32_t tx = (uint32_t)(W + kBeamTileW - 1) / kBeamTileW, ty = (uint32_t)(H + kBeamTileH - 1) / kBeamTileH;
    const uint32_t x = (uint32_t)px / kBeamTileW, y = (uint32_t)py / kBeamTileH;
    unsigned long long v = ~0ull;
    uint32_t off = 0;
#pragma unroll
    for (int L = 0; L < kBeamPyr; L++) {
        const uint32_t wl = (tx + (1u << L) - 1) >> L, hl = (ty + (1u << L) - 1) >> L;
        v = min(v, __ldcg(b + off + (y >> L) * wl + (x >> L)));
        off += wl * hl;
    }
    return (uint32_t)(v >> 32) == tag ? (int32_t)(uint32_t)v : INT_MAX;
}

// The same bound for the 8 x 4 tile (x, y) of a warp, called by all 32 lanes
// with the same tile: lane L reads level L of the pyramid through the level
// table and a butterfly takes the minimum.  The tile must lie in the view.
__device__ __forceinline__ int32_t warp_beam_bound(const BeamLookup& b, uint32_t x, uint32_t y, int lane) {
    uint32_t off = 0, wl = 0;
#pragma unroll
    for (int L = 0; L < kBeamPyr; L++)
        if (lane == L) { off = b.off[L]; wl = b.wl[L]; }
    unsigned long long v = lane < kBeamPyr ? __ldcg(b.bounds + off + (y >> lane) * wl + (x >> lane)) : ~0ull;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    v = __shfl_sync(0xFFFFFFFFu, v, 0);  // lanes 0..7 hold the minimum
    return (uint32_t)(v >> 32) == b.tag ? (int32_t)(uint32_t)v : INT_MAX;
}

// Pixel ray in the mirrored frame.  Returns true for a FAST ray: the non-zero
// |d| exponents span <= 6, mantissas shifted to a common exponent (E = 0),
// zero components m = 0.
__device__ __forceinline__ bool make_ray(const CamDev& C, int px, int py, RayState& r) {
    ray_dir(C, px, py, r.d);
    r.mir = 0;
    int emin = 1 << 20, emax = -(1 << 20);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        decompose(r.d[a], r.m[a], r.E[a]);
        if (r.d[a] < 0.0f) r.mir |= 1u << a;
        if (r.d[a] != 0.0f) { emin = min(emin, r.E[a]); emax = max(emax, r.E[a]); }
    }
    if (emax - emin > 6) return false;
#pragma unroll
    for (int a = 0; a < 3; a++) { r.m[a] = r.d[a] != 0.0f ? r.m[a] << (r.E[a] - emin) : 0; r.E[a] = 0; }
    return true;
}

// Chunk cell along axis a of the point where the ray crosses the plane (e, Ne)
// (me, Ee: |d_e| as mantissa and exponent), exactly: cell M <= x_a < (cell+1) M,
// clamped to the grid.  Ow: mirrored world origin numerators; t_num: Ne / |d_e|
// in FP32.  The FP32 estimate's error is below 2^-22 of |Ow| + |t_num d_a|
// (five roundings); with a margin of 4 its floor is used unless it lies that
// close to a chunk plane, where the plane comparisons decide.
template <bool FAST>
__device__ __forceinline__ int32_t chunk_cell(const SceneDev& S, const RayState& r, const int32_t Ow[3], int a,
                                              float t_num, int32_t Ne, int32_t me, int32_t Ee, int cs) {
    const float fo = (float)Ow[a], pr = t_num * fabsf(r.d[a]);
    const float q = (fo + pr) * (1.0f / (float)(1 << cs));
    const float err = (fabsf(fo) + fabsf(pr)) * (1.0f / (float)(1 << cs)) * 0x1p-20f;
    const float qc = fminf(fmaxf(q, -1.0f), (float)S.grid[a]);
    int32_t cell;
    if (floor_if_clear(qc, err, cell)) return max(0, min(cell, S.grid[a] - 1));
    cell = max(0, min((int32_t)floorf(qc), S.grid[a] - 1));
    while (cell + 1 < S.grid[a] && !tltf<FAST>(Ne, me, ((cell + 1) << cs) - Ow[a], r.m[a], r.E[a] - Ee)) cell++;
    while (cell > 0 && tltf<FAST>(Ne, me, (cell << cs) - Ow[a], r.m[a], r.E[a] - Ee)) cell--;
    return cell;
}

// ---------------------------------------------------------------------------
// one pixel: world-grid chunk march + per-chunk DAG traversal
// ---------------------------------------------------------------------------
template <bool FAST, bool COUNT, bool CHECK = false, bool BEAM = false>
__device__ __forceinline__ void trace_pixel_t(const SceneDev& S, const CamDev& C, const ChunkRef* __restrict__ frame,
                                            const RayState& r, uint4* __restrict__ out_hit, float* __restrict__ out_t,
                                            uint32_t* __restrict__ counts, size_t pix, const CheckDev* ck = nullptr,
                                            int32_t Dn = 0) {
    int32_t Ow[3], Wfix[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        Wfix[a] = S.grid[a] << (S.mlog + kFix);
        Ow[a] = ((r.mir >> a) & 1u) ? Wfix[a] - C.O[a] : C.O[a];
    }
    Counters cnt = {0, 0, 0};
    HitRec hit;
    bool found = false;
    const int cs = S.mlog + kFix;  // chunk side as a shift of numerator units
    int e = 3;
    int32_t Ne = 0, me = 1, Ee = 0;
    int32_t cc[3];
    bool alive = true;
    if (Ow[0] >= 0 && Ow[1] >= 0 && Ow[2] >= 0 && Ow[0] < Wfix[0] && Ow[1] < Wfix[1] && Ow[2] < Wfix[2]) {
#pragma unroll
        for (int a = 0; a < 3; a++) cc[a] = Ow[a] >> cs;
    } else {
        // enter the world box: latest entry plane vs earliest exit plane
        e = -1;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (Ow[a] >= Wfix[a] || (r.d[a] == 0.0f && Ow[a] < 0)) alive = false;
            if (Ow[a] < 0) {
                const int32_t Na = -Ow[a];
                if (e < 0 || tltf<FAST>(Ne, me, Na, r.m[a], r.E[a] - Ee)) { e = a; Ne = Na; me = r.m[a]; Ee = r.E[a]; }
            }
        }
        int32_t Nx = Wfix[0] - Ow[0], mx = r.m[0], Ex = r.E[0];
#pragma unroll
        for (int a = 1; a < 3; a++) {
            const int32_t Na = Wfix[a] - Ow[a];
            if (tltf<FAST>(Na, r.m[a], Nx, mx, Ex - r.E[a])) { Nx = Na; mx = r.m[a]; Ex = r.E[a]; }
        }
        if (alive && e >= 0 && tltf<FAST>(Ne, me, Nx, mx, Ex - Ee)) {
            const float te_num = (float)Ne / fabsf(r.d[e]);
#pragma unroll
            for (int a = 0; a < 3; a++) {
                if (a == e) { cc[a] = 0; continue; }
                cc[a] = chunk_cell<FAST>(S, r, Ow, a, te_num, Ne, me, Ee, cs);
            }
        } else {
            alive = false;
        }
    }
    if (BEAM && alive && Dn > 0) {
        // Beam restart.  Dn bounds from below (numerator units) the L-inf
        // distance from the origin of every solid voxel this ray can meet, and
        // the ray's L-inf distance at t is t |d|_max: the march resumes at the
        // last integer plane of the dominant axis crossed strictly before that
        // distance.  The cell holding that point is empty, so every hit is
        // entered later, through the planes the full march would cross.
        int as = 0;
        if (fabsf(r.d[1]) > fabsf(r.d[as])) as = 1;
        if (fabsf(r.d[2]) > fabsf(r.d[as])) as = 2;
        const long long kp = ((long long)Dn - 1 + Ow[as]) >> kFix;  // plane index (floor)
        const long long Nl = (kp << kFix) - Ow[as];
        if (Nl >= (long long)Wfix[as] - Ow[as]) {
            alive = false;  // past the world: nothing to meet
        } else if (Nl > 0 && (e == 3 || tltf<FAST>(Ne, me, (int32_t)Nl, r.m[as], r.E[as] - Ee))) {
            const int32_t Ns = (int32_t)Nl;
#pragma unroll
            for (int a = 0; a < 3; a++)
                if (a != as && r.d[a] != 0.0f && !tltf<FAST>(Ns, r.m[as], Wfix[a] - Ow[a], r.m[a], r.E[a] - r.E[as]))
                    alive = false;  // left the world box before the restart point
            if (alive) {
                e = as; Ne = Ns; me = r.m[as]; Ee = r.E[as];
                cc[as] = (int32_t)(kp >> S.mlog);
                const float ts_num = (float)Ns / fabsf(r.d[as]);
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    if (a == as) continue;
                    cc[a] = chunk_cell<FAST>(S, r, Ow, a, ts_num, Ne, me, Ee, cs);
                }
            }
        }
    }
    const float dn = ray_norm(r);
    float inv[3];
#pragma unroll
    for (int a = 0; a < 3; a++) inv[a] = 1.0f / r.d[a];
    // The march stops at the first hit and keeps what the output needs; the
    // per-hit work (entry-face rule, material, distance, stores) runs after
    // the loop, where the warp's lanes are together again.
    int32_t u[3];
    ChunkRef ref;
    int32_t Oloc[3];
    while (alive) {
#pragma unroll
        for (int a = 0; a < 3; a++) u[a] = ((r.mir >> a) & 1u) ? S.grid[a] - 1 - cc[a] : cc[a];
        ref = frame[(size_t)u[0] + (size_t)S.grid[0] * ((size_t)u[1] + (size_t)S.grid[1] * u[2])];
        if (S.view_dist > 0.0f && e < 3) {
            const float tent = (float)Ne / (4096.0f * fabsf(r.d[e]));
            if (tent * dn > S.view_dist * 1.00001f + 1.0f) break;
        }
        if (ref.root != kNone) {
            // skip chunks whose solid-voxel AABB (grown by 1/16 voxel) the ray misses
            float tn = 0.0f, tf = 3.0e38f;
            bool pass = true;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float lo = (float)((u[a] << S.mlog) + ref.aabb[a]) - 0.0625f;
                const float hi = (float)((u[a] << S.mlog) + ref.aabb[3 + a]) + 0.0625f;
                if (r.d[a] == 0.0f) {
                    if (C.of[a] < lo || C.of[a] > hi) pass = false;
                } else {
                    float t1 = (lo - C.of[a]) * inv[a], t2 = (hi - C.of[a]) * inv[a];
                    tn = fmaxf(tn, fminf(t1, t2));
                    tf = fminf(tf, fmaxf(t1, t2));
                }
            }
#pragma unroll
            for (int a = 0; a < 3; a++) Oloc[a] = Ow[a] - (cc[a] << cs);
            if (pass && tn <= tf && (!COUNT || meets_aabb<FAST>(r, Oloc, ref, S.mlog))) {
                if (trace_chunk<FAST, COUNT, CHECK, BEAM>(S, ref, r, Oloc, e, Ne, hit, cnt, ck)) {
                    found = true;
                    break;
                }
            }
        }
        // next chunk cell
        const int32_t N0 = ((cc[0] + 1) << cs) - Ow[0];
        const int32_t N1 = ((cc[1] + 1) << cs) - Ow[1];
        const int32_t N2 = ((cc[2] + 1) << cs) - Ow[2];
        const bool xy = tltf<FAST>(N0, r.m[0], N1, r.m[1], r.E[1] - r.E[0]);
        const int32_t Na = xy ? N0 : N1, ma = xy ? r.m[0] : r.m[1], Ea = xy ? r.E[0] : r.E[1];
        const bool az = tltf<FAST>(Na, ma, N2, r.m[2], r.E[2] - Ea);
        int ax;
        if (az) { ax = xy ? 0 : 1; Ne = Na; me = ma; Ee = Ea; }
        else { ax = 2; Ne = N2; me = r.m[2]; Ee = r.E[2]; }
        e = ax;
        if (++cc[ax] >= S.grid[ax]) break;
    }
    if (found) {
        lowest_entry_face<FAST>(r, Oloc, (int)ref.lod, hit);
        found = emit_hit(S, r, ref, u, hit, dn, out_hit, out_t, pix);
    }
    if (!found) emit_miss(out_hit, out_t, pix);
    if (COUNT) {
        counts[3 * pix + 0] = cnt.v_int;
        counts[3 * pix + 1] = cnt.v_leaf;
        counts[3 * pix + 2] = cnt.rbytes;
    }
}

template <bool COUNT, bool CHECK = false, bool BEAM = false>
__device__ __forceinline__ void trace_pixel(const SceneDev& S, const CamDev& C, const ChunkRef* __restrict__ frame,
                                            int px, int py, uint4* __restrict__ out_hit, float* __restrict__ out_t,
                                            uint32_t* __restrict__ counts, size_t pix, const CheckDev* ck = nullptr,
                                            int32_t Dn = 0) {
    RayState r;
    if (make_ray(C, px, py, r))
        trace_pixel_t<true, COUNT, CHECK, BEAM>(S, C, frame, r, out_hit, out_t, counts, pix, ck, Dn);
    else
        trace_pixel_t<false, COUNT, CHECK, BEAM>(S, C, frame, r, out_hit, out_t, counts, pix, ck, Dn);
}

}  // namespace aok
