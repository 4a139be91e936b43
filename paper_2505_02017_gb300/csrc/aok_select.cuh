// Chunk LOD selection (Eq. 1, Sec. 3.4) and visibility (Sec. 3.5) of one
// chunk region, shared by the selection kernels and the beam pass that
// selects as its first step.
#pragma once
#include "aok_internal.h"

namespace aok {

// ---------------------------------------------------------------------------
// selection + visibility: one thread per chunk region
// ---------------------------------------------------------------------------
// Eq. 1 for the octree block b at level n: LODError <= 0 (load), squared, FP64, fixed order.
__device__ __forceinline__ bool lod_loads(int n, int bx, int by, int bz, int mlog, const float o[3], double sf) {
    const double S = (double)(1ll << (mlog + n));
    const int b[3] = {bx, by, bz};
    double e2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double c = __dadd_rn(__dmul_rn((double)b[a], S), __dmul_rn(0.5, S));
        const double dd = __dsub_rn(c, (double)o[a]);
        e2 = __dadd_rn(e2, __dmul_rn(dd, dd));
    }
    const double thr = __dmul_rn(S, sf);
    return e2 >= __dmul_rn(thr, thr);
}

__device__ __forceinline__ ChunkRef select_one(const SceneDev& S, const CamDev& C, ChunkRef* __restrict__ frame,
                                               int8_t* __restrict__ lod_out, uint8_t* __restrict__ vis_out,
                                               uint32_t* __restrict__ n_visible, int chunk) {
    const int cx = chunk % S.grid[0], cy = (chunk / S.grid[0]) % S.grid[1], cz = chunk / (S.grid[0] * S.grid[1]);
    int sel = 0;
    for (int n = S.n_lods - 1; n >= 1; n--)
        if (lod_loads(n, cx >> n, cy >> n, cz >> n, S.mlog, C.of, C.sf)) { sel = n; break; }
    const ChunkRef* d = S.desc + (size_t)chunk * S.n_lods;
    ChunkRef ref = d[sel];
    if (ref.root == kNone && !(ref.lod & kResidentBit)) {
        // the selected LOD is not resident (still streaming in): show the
        // nearest resident LOD of the region, coarser ones first (Sec. 3.4
        // loads coarser LODs first)
        for (int n = sel + 1; n < S.n_lods; n++)
            if (d[n].root != kNone) { ref = d[n]; break; }
        for (int n = sel - 1; n >= 0 && ref.root == kNone; n--)
            if (d[n].root != kNone) ref = d[n];
    }
    const int used = ref.root != kNone ? (int)(ref.lod & 0xFFu) : sel;
    bool vis = ref.root != kNone;
    if (vis) {
        // AABB grown by one voxel: culling stays conservative under FP32 rounding
        const int org[3] = {cx << S.mlog, cy << S.mlog, cz << S.mlog};
        float lo[3], hi[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            lo[a] = (float)(org[a] + ref.aabb[a]) - 1.0f - C.of[a];
            hi[a] = (float)(org[a] + ref.aabb[3 + a]) + 1.0f - C.of[a];
        }
#pragma unroll
        for (int p = 0; p < 4; p++) {
            const float* n = C.planes[p];
            const float dmin = n[0] * (n[0] > 0 ? lo[0] : hi[0]) + n[1] * (n[1] > 0 ? lo[1] : hi[1]) +
                               n[2] * (n[2] > 0 ? lo[2] : hi[2]);
            if (dmin > 0.0f) vis = false;
        }
        if (S.view_dist > 0.0f) {
            float d2 = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float q = fminf(fmaxf(0.0f, lo[a]), hi[a]);
                d2 += q * q;
            }
            if (d2 > S.view_dist * S.view_dist * 1.0001f + 4.0f) vis = false;
        }
    }
    if (!vis) ref.root = kNone;
    ref.lod = (uint32_t)used;
    frame[chunk] = ref;
    if (lod_out) lod_out[chunk] = (int8_t)used;
    if (vis_out) vis_out[chunk] = vis ? 1 : 0;
    if (vis && n_visible) atomicAdd(n_visible, 1u);
    return ref;
}

}  // namespace aok
