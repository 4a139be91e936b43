// Host-side state of the runtime (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "aok_internal.h"

namespace aok {

constexpr uint64_t kNoRange = ~0ull;

struct Pool {  // units of the pool's element type
    uint64_t cap = 0, used = 0;
    std::vector<std::pair<uint64_t, uint64_t>> free_list;  // (offset, count)
    uint64_t alloc(uint64_t n);
    void release(uint64_t off, uint64_t n);
};

struct ChunkAlloc {
    uint64_t node_off = 0, node_n = 0, leaf_off = 0, leaf_n = 0, mat_off = 0, mat_n = 0;
};

struct Scene {
    aok_scene_desc desc{};
    double color_tol = -1.0;  // colour-block tolerance of later uploads (< 0: raw arrays)
    int mlog = 0;
    int64_t n_chunks = 0;
    uint32_t* d_nodes = nullptr;
    uint64_t* d_leaves = nullptr;
    uint8_t* d_mats = nullptr;
    ChunkRef* d_desc = nullptr;   // [chunk * n_lods + lod]
    ChunkRef* d_frame = nullptr;  // per-frame selection of aok_render
    uint64_t select_gen = 0;      // selections written into d_frame so far
    Pool nodes, leaves, mats;
    std::vector<ChunkRef> h_desc;
    std::vector<ChunkAlloc> alloc;
    std::mutex mu;
    std::vector<aok_stream*> streams;  // streamers of this scene (guarded by mu)
};

// Stop a streamer of a scene that is being destroyed: join its workers, free
// its loads and quarantined space; the object stays for aok_stream_destroy.
void stream_detach(aok_stream* s);

// Device arena of aok_render_batch: per-view frame tables, work counters and
// the CUDA graph of the last list shape.
struct BatchArena {
    ChunkRef* d_frames = nullptr;
    size_t frames_cap = 0;
    unsigned long long* beam_bounds = nullptr;  // the views' bound pyramids (grow-only)
    size_t beam_cap = 0;                        // entries
    unsigned long long* d_queue = nullptr;  // 2 per group, zero between launches
    size_t queue_cap = 0;
    GraphCache graph;
};

struct ServeState;

// Frames rendered into host memory through a pipeline: slot k's selection
// and beam pass (on `prep`, the highest stream priority) overlap slot k-1's
// cast (on `render`), which overlaps slot k-2's device-to-host copy (on
// `copy`).  Each slot has its own chunk table and bound pyramid.
constexpr int kHostSlots = 3;
struct HostSlot {
    void* hit = nullptr;
    float* t = nullptr;
    ChunkRef* frame = nullptr;  // the slot's chunk table
    size_t frame_cap = 0;       // entries
    unsigned long long* bounds = nullptr;  // the slot's bound pyramid
    size_t bounds_cap = 0;                 // entries
    cudaEvent_t prepped = nullptr, rendered = nullptr, copied = nullptr;
    uint64_t ticket = 0;  // frame in this slot (0: none yet)
};
struct HostPipe {
    cudaStream_t prep = nullptr, render = nullptr, copy = nullptr;
    HostSlot slot[kHostSlots];
    size_t px = 0;        // pixels each slot holds
    uint64_t next = 0;    // last ticket issued
    std::unique_ptr<BeamBatch> P;  // beam pass parameter block
};

// Buffers of the tile-chunk pipeline for one resolution and grid size (one
// device allocation carved into the TileDev arrays), and the scene whose
// Hi-Z history hiz_prev holds.
struct TileState {
    TileDev dev{};
    void* block = nullptr;
    size_t bytes = 0;
    int32_t W = 0, H = 0;
    int64_t n_chunks = 0;
    uint32_t scene = 0xFFFFFFFFu;
};

// The beam pass: the walk's queues and launch grid (shared by all passes of
// the context), the single-view bound pyramid and what its last pass was
// computed for.
struct BeamState {
    std::mutex mu;  // the queues' allocation and the pass counter (the serving thread shares them)
    void* qblock = nullptr;
    size_t qbytes = 0;
    uint4* q[2] = {nullptr, nullptr};
    uint32_t* cnt = nullptr;   // [kBeamLevels] queue counts, then [kBeamLevels] walk histogram
    uint32_t* hist = nullptr;
    unsigned grid = 0;         // blocks of the cooperative launch
    std::unique_ptr<BeamBatch> P;  // host parameter block (~26 KB)
    unsigned long long* bounds = nullptr;  // single-view pyramid (grow-only)
    size_t bounds_cap = 0;                 // entries
    uint32_t passes = 0;                   // passes run (their tags count down)
    // the last single-view pass: a scene, its selection, a camera
    bool valid = false;
    uint32_t scene = 0xFFFFFFFFu;
    uint64_t gen = 0;
    CamDev cam{};
    BeamRead read{nullptr, 0};
    int32_t W = 0, H = 0;
};

struct aok_ctx_impl;

}  // namespace aok

struct aok_ctx {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0, used = 0;
    std::mutex mem_mu;
    cudaError_t last_cuda = cudaSuccess;
    cudaStream_t copy_stream = nullptr;
    std::mutex scene_mu;
    std::map<uint32_t, aok::Scene*> scenes;
    uint32_t next_scene = 0;
    void* staging = nullptr;
    size_t staging_cap = 0;
    uint32_t* pinned_word = nullptr;
    uint32_t* d_counter = nullptr;
    // persistent casting launch shape (0 = defaults) and single-view kernel choice
    uint32_t ctas_per_sm = 0, threads_per_cta = 0, packet_rays = 0, tile_w_log = 0;
    int single_persistent = 0;
    int batch_persistent = 0;  // 0: batches cast with one grid launch over block tiles
    int batch_graph = 1;       // 1: a batch's launches replay as one CUDA graph
    unsigned long long* d_single_queue = nullptr;  // counters of single-view persistent launches
    aok::BatchParams single_params;
    aok::BatchArena batch;
    // device frame of aok_render_host
    void* host_hit_dev = nullptr;
    float* host_t_dev = nullptr;
    size_t host_frame_px = 0;
    aok::ServeState* serve = nullptr;
    aok::TileState tiles;
    aok::BeamState beam;
    int beam_on = 1;  // single-view renders run the beam pass before casting
    uint32_t beam_refine = 8;  // refine nodes spanning more tiles than this ...
    int beam_min_log2 = 2;     // ... whose side is above 2^this LOD-0 voxels
    uint64_t beam_min_pixels = 1500000;  // smaller frames cast without the pass
    uint32_t beam_queue = 0;             // nodes a queue level may hold (0: the allocated 2^20)
    aok::HostPipe pipe;
    int checked = 0;  // single-view casts check every pool index (error word: d_counter[8])
    std::mutex upload_mu;  // the staging buffer and the copy stream: one upload at a time
};

namespace aok {
int cuda_status(aok_ctx* ctx, cudaError_t e);
// AOK_E_CUDA for a launcher that returned AOK_E_CUDA, with the error code it read.
int launch_failure(aok_ctx* ctx);
int charge(aok_ctx* ctx, size_t bytes);
void uncharge(aok_ctx* ctx, size_t bytes);
int dev_alloc(aok_ctx* ctx, void** p, size_t bytes);
void dev_free(aok_ctx* ctx, void* p, size_t bytes);
Scene* find_scene(aok_ctx* ctx, uint32_t id);
int make_cam(aok_ctx* ctx, const Scene* sc, const aok_camera* cam, double tau, CamDev* out);
SceneDev scene_dev(const Scene* sc);
void batch_release(aok_ctx* ctx);
void free_alloc(Scene* sc, ChunkAlloc& a);
// The beam passes of a batch (one per group) for its views of at least the
// context's beam frame size; sets the views' bounds, in the batch arena or,
// with view_bounds, in view_bounds[view] (nullptr: that view casts without).
// Leaves `out` empty if no view takes the pass.
int beam_for_batch(aok_ctx* ctx, BatchParams* groups, uint32_t ngroups, std::vector<BeamBatch>& out, void* stream,
                   unsigned long long* const* view_bounds = nullptr);
// Whether a frame of W x H pixels takes the beam pass in this context.
bool beam_wanted(const aok_ctx* ctx, int32_t W, int32_t H);
// Pinned staging memory and the stream its copies go on.
struct Staging {
    void* buf = nullptr;
    size_t cap = 0;
    cudaStream_t stream = nullptr;
    size_t min_cap = (size_t)64 << 20;  // smallest buffer allocated when it grows
};
int stage_chunk(aok_ctx* ctx, Scene* sc, int64_t di, uint32_t lod, const aok_chunk_blob* blob, bool evict_old_first,
                Staging* stg, std::mutex* pool_mu, ChunkAlloc* out_a, ChunkRef* out_ref);
int render_persistent(aok_ctx* ctx, Scene* sc, const CamDev& cd, const aok_frame* frame, void* stream, bool select);
}  // namespace aok
