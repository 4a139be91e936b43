// Internal structures shared by the host runtime and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/aok.h"

namespace aok {

constexpr uint32_t kNone = 0xFFFFFFFFu;
// In a descriptor (not a frame entry): lod | kResidentBit marks an uploaded
// (chunk, LOD) whose DAG is empty (root == kNone), as opposed to one that is
// not resident.
constexpr uint32_t kResidentBit = 0x80000000u;
constexpr int kFix = 12;            // camera origin fixed point: multiples of 2^-12
constexpr int kMaxLevels = 10;      // log2(512) + 1
constexpr int kMaxImageHeight = 65535 * 8;  // 8-row casting blocks, at most 65535 in grid y

// One (chunk, LOD) as resident on the device, and (per frame) the selected
// LOD of a chunk region.  32 bytes: one sector per lookup.
struct ChunkRef {
    uint32_t root;       // global node word index, kNone = empty / not resident / culled
    uint32_t lod;        // LOD of this DAG
    uint64_t mat_base;   // offset of its materials in the scene's material pool
    uint16_t aabb[6];    // chunk-local LOD-0 units: lo x,y,z, hi x,y,z ([lo, hi))
    uint32_t nblocks;    // 0: materials[DFS index] at mat_base; else colour blocks at mat_base:
                         // nt, nt uint32 block-of-entry-128j, nblocks uint32 first indices,
                         // nblocks uint8 colours (Sec. 3.3)
};
static_assert(sizeof(ChunkRef) == 32, "ChunkRef is one 32-byte sector");

struct SceneDev {
    const uint32_t* nodes;
    const uint64_t* leaves;
    const uint8_t* mats;
    const ChunkRef* desc;   // [chunk * n_lods + lod]
    int32_t grid[3];
    int32_t mlog;           // log2(chunk_res)
    int32_t n_lods;
    float view_dist;
};

// Checked traversal (no counterpart in the paper; the stand-in for a memory
// checker): pool sizes every node, leaf and colour index is checked against,
// and the word the kernels OR an error code into instead of reading out of
// bounds (1: node word, 2: leaf, 4: colour byte).
struct CheckDev {
    uint64_t n_nodes, n_leaves, n_mats;
    uint32_t* err;
};

// Camera as the kernels consume it.
struct CamDev {
    float R[9];
    float tan_half;
    int32_t W, H;
    int32_t O[3];           // origin * 2^kFix (exact)
    float of[3];            // origin as float
    float planes[4][4];     // view-pyramid side planes: n . (p - o) <= 0 inside (n, unused)
    double sf;              // StreamingFactor for Eq. 1
    float aspect;           // (float)W / (float)H, one IEEE rounding
    float pad;
};

// Device buffers of the tile-chunk pipeline (Sec. 3.5) for one resolution.
constexpr int kTileStats = 8;
struct TileDev {
    unsigned long long* vis;   // [W*H][2] visibility records: key (distance | march order | chunk), ~0 = none;
                               // payload (hit voxel, LOD, entry axis, material)
    float* hiz_prev;           // [tiles] previous frame's per-tile max hit distance (no culling: huge)
    float* hiz;                // [tiles] per-tile max distance after pass 1 of this frame
    float* hiz_next;           // [tiles] this frame's final per-tile max distance
    int4* rect;                // [chunks] tile rectangle [x0, x1) x [y0, y1) of the chunk's AABB
    float* dmin;               // [chunks] lower bound of the distance from the camera to the AABB
    int32_t* dfar;             // [chunks] largest L-inf distance (2^-12 units) from the camera origin to a
                               // point of the AABB
    uint32_t* area;            // [chunks] tiles in the rectangle (0: no pairs)
    uint32_t* list;            // [chunks] chunks with pairs, ascending
    unsigned long long* offs;  // [chunks + 1] exclusive prefix of their areas; offs[n_list] = pairs
    unsigned long long* stats; // [kTileStats] n_list, items traced / culled per pass, pixel traces ...
    int32_t tiles_x, tiles_y;
};

// The beam pass (ESVO's beam optimisation, Sec. 2; aok_beam.cu): per 8 x 4
// pixel tile (one casting warp) a lower bound on the L-infinity distance from
// the camera origin of every solid voxel the tile's rays can meet, found by a
// level-by-level walk of the selected DAGs.  A view's bounds form a pyramid
// of 64-bit entries (pass tag << 32) | bound, level L (cells of 2^L x 2^L
// tiles) at beam_level_offset(L) from the view's first entry; an entry whose
// tag is not the pass's means "no solid voxel".
constexpr int kBeamTileW = 8, kBeamTileH = 4;
constexpr int kBeamLevels = 16;  // queue counters (node levels of a 512^3 chunk: 8)
constexpr int kBeamPyr = 7;      // bound pyramid levels (level 0: the tiles), at most 8
static_assert(kBeamPyr <= 8, "a warp reads the pyramid levels with one lane each, reduced over 8 lanes");
constexpr int kBeamViews = 128;  // views of one beam pass

__host__ __device__ __forceinline__ uint32_t beam_level_offset(uint32_t tx, uint32_t ty, int L) {
    uint32_t off = 0;
    for (int l = 0; l < L; l++) off += ((tx + (1u << l) - 1) >> l) * ((ty + (1u << l) - 1) >> l);
    return off;
}
__host__ __device__ __forceinline__ uint32_t beam_entries(uint32_t W, uint32_t H) {
    return beam_level_offset((W + kBeamTileW - 1) / kBeamTileW, (H + kBeamTileH - 1) / kBeamTileH, kBeamPyr);
}

// One view of a beam pass.
struct BeamView {
    SceneDev scene;
    const ChunkRef* frame;
    unsigned long long* bounds;  // the view's pyramid (beam_entries(W, H) entries)
    float Af[9];                 // row-major inverse of A = [R col 0, R col 1, -R col 2] (d = A (u, v, 1)), FP32
    float U, V;                  // u and v at the screen edges: tan_half * W / H, tan_half
    float near_dn;               // numerator units: boxes closer than this cover every tile
    float view_num;              // > 0: boxes farther than this (Euclidean, numerator units) are dropped
    int32_t W, H, tiles_x, tiles_y;
    int32_t O[3];                // origin numerators
    uint32_t region_begin;       // first item of this view among the pass's regions
};

// The parameter block of one beam pass over up to kBeamViews views.
struct BeamBatch {
    uint32_t n_views, n_regions;  // views; chunk regions of all views
    uint32_t expand;              // refine nodes whose rectangle spans more tiles than this ...
    int32_t smin;                 // ... and whose side is above 2^smin LOD-0 voxels
    uint32_t tag;                 // the pass's tag: decreases from pass to pass
    uint32_t cap;                 // queue capacity in items
    uint4* q[2];                  // node queues of alternate levels: {chunk, node, cell x | y << 10 | z << 20, log2 size | view << 8 | LOD << 16}
    uint32_t* cnt;                // [kBeamLevels] items queued per level
    uint32_t* hist;               // [kBeamLevels] nodes walked per depth below the region roots
    uint32_t select;              // 1: one view whose frame table the pass selects first (cam)
    CamDev cam;                   // that view's camera (select == 1)
    CheckDev ck;                  // ck.err != nullptr: node and leaf indices tested before their loads
    BeamView v[kBeamViews];
};
static_assert(sizeof(BeamBatch) < 32000, "a beam pass's parameters must fit the kernel parameter space");

// What a casting kernel reads of a view's beam pass (bounds == nullptr: none).
struct BeamRead {
    const unsigned long long* bounds;
    uint32_t tag;
};

// The beam pass's bound pyramid of one W x H view as a casting kernel reads
// it: per level, the offset of its first entry and its row width (computed
// once on the host instead of per pixel).
struct BeamLookup {
    const unsigned long long* bounds;  // nullptr: no bounds
    uint32_t tag;
    uint32_t off[kBeamPyr], wl[kBeamPyr];
};

inline BeamLookup beam_lookup(const BeamRead* b, int W, int H) {
    BeamLookup L;
    std::memset(&L, 0, sizeof(L));
    if (!b) return L;
    L.bounds = b->bounds;
    L.tag = b->tag;
    const uint32_t tx = (uint32_t)(W + kBeamTileW - 1) / kBeamTileW, ty = (uint32_t)(H + kBeamTileH - 1) / kBeamTileH;
    for (int l = 0; l < kBeamPyr; l++) {
        L.off[l] = beam_level_offset(tx, ty, l);
        L.wl[l] = (tx + (1u << l) - 1) >> l;
    }
    return L;
}

// Descriptor updates applied by a kernel on the rendering stream, so that a
// frame sees every (chunk, LOD) change published before it and none after.
struct DescPatch {
    uint64_t index;  // descriptor index chunk * n_lods + lod
    ChunkRef ref;
};
constexpr int kPatchMax = 96;
struct DescPatches {
    uint32_t n;
    uint32_t pad;
    DescPatch p[kPatchMax];
};

// A view of a batch: which scene, which camera, where the pixels go.
struct ViewDev {
    SceneDev scene;
    CamDev cam;
    ChunkRef* frame;        // per-view selected chunk table [chunk]
    uint4* hit;
    float* t;
    uint64_t tile_begin;    // first global warp-tile index of this view in the batch
    const unsigned long long* beam;  // the view's beam-pass bounds (BatchParams::beam_tag), or nullptr
};

// Parameter block of one batched launch (kernel parameters: up to 32 KB).
constexpr int kBatchViews = 128;
struct BatchParams {
    uint32_t n_views;
    uint32_t per_fetch;        // warp tiles taken per queue fetch
    uint32_t tile_w_log;       // warp tile = 2^tile_w_log x 32 / 2^tile_w_log pixels
    uint32_t max_chunks;       // largest chunk grid among the views
    uint64_t total_tiles;      // warp tiles of all views
    unsigned long long* queue; // [0] next warp tile, [1] finished CTAs; zero at launch, re-armed by the last CTA
    uint32_t beam_tag;         // tag of the beam pass the views' bounds come from
    uint32_t pad;
    ViewDev v[kBatchViews];
};
static_assert(sizeof(BatchParams) < 32000, "batched launch parameters must fit the kernel parameter space");

// CUDA graph of one batch shape, rebuilt when the shape changes.
struct GraphCache {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> nodes;  // per group: select, [counter memset, beam pass], cast
    std::vector<uint64_t> key;
};

}  // namespace aok

// Kernel launchers (aok_kernels.cu), called by the runtime.
extern "C" {
// Launch errors.  Reading cudaGetLastError clears a non-sticky launch error
// (an invalid grid, say), so a launcher that finds one keeps its code, per host
// thread, and returns AOK_E_CUDA; aokk_take_launch_error hands the code to the
// runtime (else the thread's last CUDA error, and never cudaSuccess).
int aokk_status(cudaError_t e);
cudaError_t aokk_take_launch_error();
int aokk_select(const aok::SceneDev* s, const aok::CamDev* c, aok::ChunkRef* frame, int8_t* lod_out,
                uint8_t* vis_out, uint32_t* n_visible, void* stream);
int aokk_cast(const aok::SceneDev* s, const aok::CamDev* c, const aok::ChunkRef* frame, uint4* hit, float* t,
              uint32_t* counts, void* stream, const aok::CheckDev* ck, const aok::BeamRead* beam = nullptr);
// Beam pass (aok_beam.cu).  aokk_beam_view fills a view's projection (false:
// the camera matrix has no usable inverse; leave the view out, it casts
// without bounds); aokk_beam_run zeroes P's counters and launches the pass
// (narrow: as one 128-thread block per SM that fits beside a running cast,
// for walks over at most 4096 regions; the pipelined host frames use it).
bool aokk_beam_view(const aok::SceneDev* S, const aok::CamDev* C, const aok::ChunkRef* frame,
                    unsigned long long* bounds, aok::BeamView* out);
int aokk_beam_run(const aok::BeamBatch* P, unsigned grid, void* stream, int narrow = 0);
// The pass as a graph node (kernel + counter memset) and the per-device pass
// order around a graph launch (record = 0: wait for the previous pass before;
// 1: mark the end of the launch as the point the next pass waits for).
void aokk_beam_node(const aok::BeamBatch* P, unsigned grid, void** argp, cudaKernelNodeParams* kp,
                    cudaMemsetParams* zero);
int aokk_beam_order(void* stream, int record);
// Blocks of the beam pass's cooperative launch on `sms` SMs (0 on error).
unsigned aokk_beam_grid(int sms);
int aokk_ray_dirs(const aok::CamDev* c, float* dirs, void* stream);
int aokk_tiles_frame(const aok::SceneDev* S, const aok::CamDev* C, const aok::ChunkRef* frame, const aok::TileDev* T,
                     uint4* hit, float* t, int sms, void* stream, const aok::BeamRead* beam = nullptr);
int aokk_patch_desc(aok::ChunkRef* desc, const aok::DescPatches* p, void* stream);
int aokk_read_bw(const void* buf, size_t n16, int passes, uint32_t* sink, int sms, void* stream);
// Batched: one selection launch over (view, chunk), then one persistent
// casting launch over all views' warp tiles.
int aokk_select_batch(const aok::BatchParams* p, void* stream);
int aokk_cast_batch(const aok::BatchParams* p, uint32_t ctas, uint32_t threads, void* stream);
// A batch's beam passes on a stream of their own: the pass waits for the
// group's selection (event sel), the cast for the pass (event beam).
struct BeamHandoff {
    void* stream;
    cudaEvent_t sel, beam;
};
int aokk_batch_run(const aok::BatchParams* groups, uint32_t n_groups, uint32_t ctas, uint32_t threads, void* stream,
                   const aok::BeamBatch* beams, unsigned beam_grid, const BeamHandoff* handoff,
                   aok::GraphCache* gc);
void aokk_graph_destroy(aok::GraphCache* gc);
int aokk_max_ctas_per_sm(uint32_t threads);
int aokk_sm_count(int device);
// aok_render_noalloc's launcher: chunk table in static device memory; with
// ck, the checked casting kernel (its error word is context memory).
int aokk_render_noalloc(const aok::SceneDev* s, const aok::CamDev* c, uint4* hit, float* t, void* stream,
                        const aok::CheckDev* ck);
}
