// Batched multi-view rendering (one selection + one persistent casting launch
// per group of up to 128 views, as one CUDA graph per list shape), the launch
// autotuner, and the continuous-batching serving loop.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "aok_runtime.h"

using namespace aok;

namespace aok {

// ---------------------------------------------------------------------------
// launch shape
// ---------------------------------------------------------------------------
struct LaunchShape {
    uint32_t ctas, threads, per_fetch, tile_w_log;  // ctas == 0: grid launch over block tiles
};

static LaunchShape launch_shape(aok_ctx* ctx) {
    LaunchShape L;
    if (!ctx->batch_persistent) {
        L.ctas = 0;
        L.threads = 128;
        L.per_fetch = 1;
        L.tile_w_log = ctx->tile_w_log ? ctx->tile_w_log : 3;
        return L;
    }
    L.threads = ctx->threads_per_cta ? ctx->threads_per_cta : 256;
    int occ = aokk_max_ctas_per_sm(L.threads);
    if (occ < 1) occ = 1;
    uint32_t per_sm = ctx->ctas_per_sm ? std::min<uint32_t>(ctx->ctas_per_sm, (uint32_t)occ) : (uint32_t)occ;
    L.ctas = per_sm * (uint32_t)std::max(1, ctx->sm_count);
    L.per_fetch = ctx->packet_rays ? std::max<uint32_t>(1, ctx->packet_rays / 32) : 1;
    L.tile_w_log = ctx->tile_w_log ? ctx->tile_w_log : 3;
    return L;
}

// Work units of one view: warp tiles (persistent kernel) or block tiles of
// 2x2 warp tiles (grid launch).
static uint64_t view_tiles(const LaunchShape& L, int W, int H) {
    uint32_t tw = 1u << L.tile_w_log, th = 32u >> L.tile_w_log;
    if (!L.ctas) { tw *= 2; th *= 2; }
    return (uint64_t)((W + tw - 1) / tw) * (uint64_t)((H + th - 1) / th);
}

// ---------------------------------------------------------------------------
// batch preparation: validate views, place frame tables, fill parameter blocks
// ---------------------------------------------------------------------------
struct Prepared {
    std::vector<BatchParams> groups;  // heap: each is ~30 KB
    size_t frame_entries = 0;
};

// frames: device ChunkRef array with room for every view's chunk grid (laid out
// view after view); counters: 2 per group, zero.
static int prepare_batch(aok_ctx* ctx, const aok_view* views, uint32_t n, ChunkRef* frames, size_t frames_cap,
                         unsigned long long* counters, const LaunchShape& L, Prepared& out) {
    out.groups.clear();
    out.frame_entries = 0;
    const uint32_t ngroups = (n + kBatchViews - 1) / kBatchViews;
    out.groups.resize(ngroups);
    size_t foff = 0;
    for (uint32_t g = 0; g < ngroups; g++) {
        BatchParams& P = out.groups[g];
        std::memset(&P, 0, sizeof(P));
        P.per_fetch = L.per_fetch;
        P.tile_w_log = L.tile_w_log;
        P.queue = counters + 2 * g;
        const uint32_t v0 = g * kBatchViews, v1 = std::min(n, v0 + kBatchViews);
        P.n_views = v1 - v0;
        uint64_t tiles = 0;
        for (uint32_t i = v0; i < v1; i++) {
            const aok_view& v = views[i];
            if (!v.frame.hit || !v.frame.t || ((uintptr_t)v.frame.hit & 15) || ((uintptr_t)v.frame.t & 3))
                return AOK_E_INVALID;
            Scene* sc = find_scene(ctx, v.scene);
            if (!sc) return AOK_E_NOT_RESIDENT;
            ViewDev& d = P.v[i - v0];
            int st = make_cam(ctx, sc, &v.cam, v.lod_threshold_px, &d.cam);
            if (st) return st;
            d.scene = scene_dev(sc);
            if (frames) {
                if (foff + (size_t)sc->n_chunks > frames_cap) return AOK_E_OOM;
                d.frame = frames + foff;
            }
            foff += (size_t)sc->n_chunks;
            d.hit = (uint4*)v.frame.hit;
            d.t = v.frame.t;
            d.tile_begin = tiles;
            tiles += view_tiles(L, v.cam.width, v.cam.height);
            P.max_chunks = std::max<uint32_t>(P.max_chunks, (uint32_t)sc->n_chunks);
        }
        P.total_tiles = tiles;
    }
    out.frame_entries = foff;
    return AOK_OK;
}

static int ensure_batch_arena(aok_ctx* ctx, size_t frame_entries, uint32_t ngroups) {
    BatchArena& A = ctx->batch;
    if (frame_entries > A.frames_cap) {
        cudaDeviceSynchronize();
        dev_free(ctx, A.d_frames, A.frames_cap * sizeof(ChunkRef));
        A.d_frames = nullptr;
        A.frames_cap = 0;
        size_t cap = std::max<size_t>(frame_entries, 4096);
        int st = dev_alloc(ctx, (void**)&A.d_frames, cap * sizeof(ChunkRef));
        if (st) return st;
        A.frames_cap = cap;
    }
    if (ngroups * 2 > A.queue_cap) {
        cudaDeviceSynchronize();
        dev_free(ctx, A.d_queue, A.queue_cap * sizeof(unsigned long long));
        A.d_queue = nullptr;
        A.queue_cap = 0;
        size_t cap = std::max<size_t>(ngroups * 2, 64);
        int st = dev_alloc(ctx, (void**)&A.d_queue, cap * sizeof(unsigned long long));
        if (st) return st;
        if (cudaMemset(A.d_queue, 0, cap * sizeof(unsigned long long)) != cudaSuccess) return AOK_E_CUDA;
        A.queue_cap = cap;
    }
    return AOK_OK;
}

void batch_release(aok_ctx* ctx) {
    BatchArena& A = ctx->batch;
    aokk_graph_destroy(&A.graph);
    dev_free(ctx, A.d_frames, A.frames_cap * sizeof(ChunkRef));
    dev_free(ctx, A.d_queue, A.queue_cap * sizeof(unsigned long long));
    dev_free(ctx, A.beam_bounds, A.beam_cap * 8);
    A = BatchArena();
}

static int render_batch_impl(aok_ctx* ctx, const aok_view* views, uint32_t n, void* stream, bool use_graph) {
    if (!ctx || !views || n == 0 || n > 4096) return AOK_E_INVALID;
    cudaSetDevice(ctx->device);
    const LaunchShape L = launch_shape(ctx);
    Prepared prep;
    int st = prepare_batch(ctx, views, n, nullptr, 0, nullptr, L, prep);  // sizes only
    if (st) return st;
    st = ensure_batch_arena(ctx, prep.frame_entries, (uint32_t)prep.groups.size());
    if (st) return st;
    st = prepare_batch(ctx, views, n, ctx->batch.d_frames, ctx->batch.frames_cap, ctx->batch.d_queue, L, prep);
    if (st) return st;
    // the beam pass for the views large enough (grid launch only)
    std::vector<BeamBatch> beams;
    if (L.ctas == 0) {
        st = beam_for_batch(ctx, prep.groups.data(), (uint32_t)prep.groups.size(), beams, stream);
        if (st) return st;
    }
    st = aokk_batch_run(prep.groups.data(), (uint32_t)prep.groups.size(), L.ctas, L.threads, stream,
                        beams.empty() ? nullptr : beams.data(), ctx->beam.grid, nullptr,
                        use_graph ? &ctx->batch.graph : nullptr);
    return st == AOK_E_CUDA ? cuda_status(ctx, cudaGetLastError()) : st;
}

// single view through the persistent kernel, using the scene's own frame table
int render_persistent(aok_ctx* ctx, Scene* sc, const CamDev& cd, const aok_frame* frame, void* stream,
                      bool select) {
    const LaunchShape L = launch_shape(ctx);
    int st;
    BatchParams* P = &ctx->single_params;
    std::memset(P, 0, sizeof(BatchParams));
    P->n_views = 1;
    P->per_fetch = L.per_fetch;
    P->tile_w_log = L.tile_w_log;
    P->queue = ctx->d_single_queue;
    P->max_chunks = (uint32_t)sc->n_chunks;
    ViewDev& d = P->v[0];
    d.scene = scene_dev(sc);
    d.cam = cd;
    d.frame = sc->d_frame;
    d.hit = (uint4*)frame->hit;
    d.t = frame->t;
    d.tile_begin = 0;
    P->total_tiles = view_tiles(L, cd.W, cd.H);
    if (select) {
        st = aokk_select_batch(P, stream);
        if (st) return st;
    }
    return aokk_cast_batch(P, L.ctas, L.threads, stream);
}

// ---------------------------------------------------------------------------
// serving
// ---------------------------------------------------------------------------
enum TicketState { kQueued, kRunning, kDone, kFailed };

static uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Ticket {
    aok_request req;
    TicketState state = kQueued;
    uint64_t t_submit = 0, t_done = 0;
    void* hit = nullptr;
    float* t = nullptr;
    ChunkRef* frame = nullptr;
    unsigned long long* bounds = nullptr;  // beam-pass pyramid (large frames with the pass on)
    size_t bytes = 0;
    int status = AOK_OK;
};

struct ServeState;

// Completion record of one launched batch; the stream's host callback marks it
// done and wakes the serving loop (no CUDA calls inside the callback).
struct BatchDone {
    ServeState* S = nullptr;
    std::atomic<int> done{0};
    std::atomic<uint64_t> t_ns{0};
};

struct InFlight {
    cudaEvent_t done;
    BatchDone* flag;
    std::vector<uint64_t> tickets;
    uint32_t stream_slot;
};

struct ServeState {
    uint32_t max_slots = 0, max_batch = 0;
    // wake-ups of the loop: own mutex, never held across a CUDA call
    std::mutex wake_mu;
    std::condition_variable wake_cv;
    int wake = 0;
    std::vector<cudaStream_t> streams;
    cudaStream_t beam_stream = nullptr;  // the batches' beam passes
    std::vector<cudaEvent_t> beam_ev;    // per stream: selection done, beam pass done
    std::vector<unsigned long long*> counters;  // 2 * kBatchViews-group pairs per stream
    std::vector<uint32_t> stream_busy;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::vector<InFlight> inflight;
    std::vector<cudaEvent_t> free_events;
    uint64_t next_ticket = 0;
    uint32_t running = 0;  // tickets admitted and not yet done
    bool stop = false;
    std::thread loop;
    std::vector<BatchParams> params;  // staging
    // request frames come from a memory pool of their own that keeps freed
    // memory mapped (release threshold = the budget), so a burst of arrivals
    // never waits for the driver to map memory again
    cudaMemPool_t pool = nullptr;
};

static void wake_loop(ServeState* S) {
    {
        std::lock_guard<std::mutex> g(S->wake_mu);
        S->wake = 1;
    }
    S->wake_cv.notify_all();
}

static void CUDART_CB on_batch_done(void* p) {
    BatchDone* b = (BatchDone*)p;
    b->t_ns.store(now_ns());
    b->done.store(1);
    wake_loop(b->S);
}

// A request's device memory: frame record, distances, chunk table and, for a
// frame that takes the beam pass, its bound pyramid.
static size_t request_bytes(const aok_ctx* ctx, const Scene* sc, const aok_camera& cam) {
    const size_t px = (size_t)cam.width * cam.height;
    size_t b = ((px * 16 + 255) & ~(size_t)255) + ((px * 4 + 255) & ~(size_t)255) +
               (((size_t)sc->n_chunks * sizeof(ChunkRef) + 255) & ~(size_t)255);
    if (beam_wanted(ctx, cam.width, cam.height)) b += (size_t)beam_entries((uint32_t)cam.width, (uint32_t)cam.height) * 8;
    return b;
}

static void free_ticket_memory(aok_ctx* ctx, Ticket& t, cudaStream_t s) {
    if (t.hit) {
        cudaFreeAsync(t.hit, s);
        uncharge(ctx, t.bytes);
    }
    t.hit = nullptr;
    t.t = nullptr;
    t.frame = nullptr;
    t.bounds = nullptr;
    t.bytes = 0;
}

static void serve_loop(aok_ctx* ctx) {
    ServeState& S = *ctx->serve;
    cudaSetDevice(ctx->device);
    const LaunchShape L = launch_shape(ctx);
    std::vector<uint64_t> batch;
    for (;;) {
        // retire finished batches
        {
            std::vector<InFlight> still;
            std::vector<InFlight> finished;
            {
                std::lock_guard<std::mutex> g(S.mu);
                for (auto& f : S.inflight) {
                    if (f.flag->done.load() && cudaEventQuery(f.done) == cudaSuccess) finished.push_back(f);
                    else still.push_back(f);
                }
                S.inflight.swap(still);
                for (auto& f : finished) {
                    const uint64_t tdone = f.flag->t_ns.load();
                    delete f.flag;
                    for (uint64_t id : f.tickets) {
                        auto it = S.tickets.find(id);
                        if (it != S.tickets.end() && it->second.state == kRunning) {
                            it->second.state = kDone;
                            it->second.t_done = tdone;
                        }
                        S.running--;
                    }
                    S.stream_busy[f.stream_slot]--;
                    S.free_events.push_back(f.done);
                }
            }
            if (!finished.empty()) S.done_cv.notify_all();
        }
        // admit: while slots and HBM allow, take queued requests into one batch
        batch.clear();
        uint32_t slot = 0;
        {
            std::unique_lock<std::mutex> g(S.mu);
            if (S.stop && S.pending.empty() && S.inflight.empty()) break;
            // stream with the fewest batches in flight
            for (uint32_t i = 1; i < S.streams.size(); i++)
                if (S.stream_busy[i] < S.stream_busy[slot]) slot = i;
            while (!S.pending.empty() && batch.size() < S.max_batch && S.running < S.max_slots &&
                   S.stream_busy[slot] < 2) {
                const uint64_t id = S.pending.front();
                auto it = S.tickets.find(id);
                if (it == S.tickets.end()) { S.pending.pop_front(); continue; }  // released while queued
                Ticket& t = it->second;
                Scene* sc = find_scene(ctx, t.req.scene);
                if (!sc) {
                    t.state = kFailed;
                    t.status = AOK_E_NOT_RESIDENT;
                    S.pending.pop_front();
                    continue;
                }
                const size_t bytes = request_bytes(ctx, sc, t.req.cam);
                if (charge(ctx, bytes) != AOK_OK) break;  // wait for memory to free up
                void* mem = nullptr;
                if (cudaMallocFromPoolAsync(&mem, bytes, S.pool, S.streams[slot]) != cudaSuccess) {
                    cudaGetLastError();
                    uncharge(ctx, bytes);
                    break;
                }
                const size_t px = (size_t)t.req.cam.width * t.req.cam.height;
                t.hit = mem;
                t.t = (float*)((char*)mem + ((px * 16 + 255) & ~(size_t)255));
                t.frame = (ChunkRef*)((char*)t.t + ((px * 4 + 255) & ~(size_t)255));
                t.bounds = beam_wanted(ctx, t.req.cam.width, t.req.cam.height)
                               ? (unsigned long long*)((char*)t.frame +
                                                       (((size_t)sc->n_chunks * sizeof(ChunkRef) + 255) & ~(size_t)255))
                               : nullptr;
                t.bytes = bytes;
                t.state = kRunning;
                S.running++;
                S.pending.pop_front();
                batch.push_back(id);
            }
        }
        if (batch.empty()) {
            // sleep until a submission, a release or a batch completion wakes us
            std::unique_lock<std::mutex> w(S.wake_mu);
            if (!S.wake) S.wake_cv.wait_for(w, std::chrono::milliseconds(2));
            S.wake = 0;
            continue;
        }
        // launch the batch on its stream: groups of up to 128 views
        const cudaStream_t st = S.streams[slot];
        const uint32_t ngroups = (uint32_t)((batch.size() + kBatchViews - 1) / kBatchViews);
        S.params.resize(ngroups);
        int rc = AOK_OK;
        {
            std::lock_guard<std::mutex> g(S.mu);
            for (uint32_t gi = 0; gi < ngroups && rc == AOK_OK; gi++) {
                BatchParams& P = S.params[gi];
                std::memset(&P, 0, sizeof(P));
                P.per_fetch = L.per_fetch;
                P.tile_w_log = L.tile_w_log;
                P.queue = S.counters[slot] + 2 * gi;
                const size_t v0 = (size_t)gi * kBatchViews, v1 = std::min(batch.size(), v0 + kBatchViews);
                P.n_views = (uint32_t)(v1 - v0);
                uint64_t tiles = 0;
                for (size_t i = v0; i < v1; i++) {
                    Ticket& t = S.tickets[batch[i]];
                    Scene* sc = find_scene(ctx, t.req.scene);
                    ViewDev& d = P.v[i - v0];
                    rc = sc ? make_cam(ctx, sc, &t.req.cam, t.req.lod_threshold_px, &d.cam) : AOK_E_NOT_RESIDENT;
                    if (rc) break;
                    d.scene = scene_dev(sc);
                    d.frame = t.frame;
                    d.hit = (uint4*)t.hit;
                    d.t = t.t;
                    d.tile_begin = tiles;
                    tiles += view_tiles(L, t.req.cam.width, t.req.cam.height);
                    P.max_chunks = std::max<uint32_t>(P.max_chunks, (uint32_t)sc->n_chunks);
                }
                P.total_tiles = tiles;
            }
        }
        // the beam pass for the large requests (grid launch): their pyramids
        // are fresh pool memory, so every entry is first set to "no tag"
        std::vector<BeamBatch> beams;
        if (rc == AOK_OK && L.ctas == 0) {
            std::vector<unsigned long long*> vb(batch.size(), nullptr);
            {
                std::lock_guard<std::mutex> g(S.mu);
                for (size_t i = 0; i < batch.size(); i++) vb[i] = S.tickets[batch[i]].bounds;
            }
            for (size_t i = 0; i < batch.size() && rc == AOK_OK; i++) {
                if (!vb[i]) continue;
                const ViewDev& d = S.params[i / kBatchViews].v[i % kBatchViews];
                if (cudaMemsetAsync(vb[i], 0xFF, (size_t)beam_entries((uint32_t)d.cam.W, (uint32_t)d.cam.H) * 8, st) !=
                    cudaSuccess)
                    rc = AOK_E_CUDA;
            }
            if (rc == AOK_OK) rc = beam_for_batch(ctx, S.params.data(), ngroups, beams, st, vb.data());
        }
        if (rc == AOK_OK) {
            // the server's passes share one stream: a pass waits only for its
            // batch's selection and for the passes before it
            const BeamHandoff ho{S.beam_stream, S.beam_ev[2 * slot], S.beam_ev[2 * slot + 1]};
            rc = aokk_batch_run(S.params.data(), ngroups, L.ctas, L.threads, st, beams.empty() ? nullptr : beams.data(),
                                ctx->beam.grid, &ho, nullptr);
        }
        std::lock_guard<std::mutex> g(S.mu);
        if (rc != AOK_OK) {
            for (uint64_t id : batch) {
                Ticket& t = S.tickets[id];
                t.state = kFailed;
                t.status = rc;
                S.running--;
            }
            S.done_cv.notify_all();
            continue;
        }
        cudaEvent_t ev;
        if (!S.free_events.empty()) {
            ev = S.free_events.back();
            S.free_events.pop_back();
        } else {
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        }
        cudaEventRecord(ev, st);
        BatchDone* flag = new BatchDone();
        flag->S = &S;
        cudaLaunchHostFunc(st, on_batch_done, flag);
        InFlight f;
        f.done = ev;
        f.flag = flag;
        f.tickets = batch;
        f.stream_slot = slot;
        S.stream_busy[slot]++;
        S.inflight.push_back(std::move(f));
    }
}

}  // namespace aok

extern "C" {

int aok_render_batch(aok_ctx* ctx, const aok_view* views, uint32_t n, void* stream) {
    return render_batch_impl(ctx, views, n, stream, ctx && ctx->batch_graph);
}

int aok_set_launch(aok_ctx* ctx, uint32_t ctas_per_sm, uint32_t threads_per_cta, uint32_t packet_rays) {
    if (!ctx) return AOK_E_INVALID;
    if (threads_per_cta && (threads_per_cta % 32 || threads_per_cta > 256)) return AOK_E_INVALID;
    if (packet_rays && packet_rays % 32) return AOK_E_INVALID;
    if (ctas_per_sm) ctx->ctas_per_sm = ctas_per_sm;
    if (threads_per_cta) ctx->threads_per_cta = threads_per_cta;
    if (packet_rays) ctx->packet_rays = packet_rays;
    return AOK_OK;
}

int aok_get_launch(aok_ctx* ctx, uint32_t* ctas_per_sm, uint32_t* threads_per_cta, uint32_t* packet_rays) {
    if (!ctx) return AOK_E_INVALID;
    const LaunchShape L = launch_shape(ctx);
    if (ctas_per_sm) *ctas_per_sm = L.ctas / (uint32_t)std::max(1, ctx->sm_count);  // 0: grid launch
    if (threads_per_cta) *threads_per_cta = L.threads;
    if (packet_rays) *packet_rays = 32 * L.per_fetch;
    return AOK_OK;
}

int aok_set_tile(aok_ctx* ctx, uint32_t tile_w) {
    if (!ctx || !(tile_w == 4 || tile_w == 8 || tile_w == 16 || tile_w == 32)) return AOK_E_INVALID;
    uint32_t l = 0;
    while ((1u << l) < tile_w) l++;
    ctx->tile_w_log = l;
    return AOK_OK;
}

int aok_set_batch_kernel(aok_ctx* ctx, int persistent) {
    if (!ctx || persistent < 0 || persistent > 1) return AOK_E_INVALID;
    ctx->batch_persistent = persistent;
    return AOK_OK;
}

int aok_set_batch_graph(aok_ctx* ctx, int on) {
    if (!ctx || on < 0 || on > 1) return AOK_E_INVALID;
    ctx->batch_graph = on;
    return AOK_OK;
}

int aok_autotune(aok_ctx* ctx, const aok_view* views, uint32_t n, void* stream, float* best_ms) {
    if (!ctx || !views || !n) return AOK_E_INVALID;
    cudaSetDevice(ctx->device);
    struct Cand { int persistent; uint32_t per_sm, threads, packet, twl; };
    std::vector<Cand> cands;
    for (uint32_t twl : {2u, 3u, 4u}) cands.push_back({0, 0, 128, 32, twl});  // grid launches
    for (uint32_t threads : {128u, 256u}) {
        const int occ = std::max(1, aokk_max_ctas_per_sm(threads));
        for (int per_sm : {occ, std::max(1, occ / 2)})
            for (uint32_t packet : {32u, 128u})
                for (uint32_t twl : {3u}) cands.push_back({1, (uint32_t)per_sm, threads, packet, twl});
    }
    const int keep_p = ctx->batch_persistent;
    const uint32_t keep[4] = {ctx->ctas_per_sm, ctx->threads_per_cta, ctx->packet_rays, ctx->tile_w_log};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const cudaStream_t st = (cudaStream_t)stream;
    float best = 1e30f;
    Cand bc = {keep_p, keep[0], keep[1], keep[2], keep[3]};
    int rc = AOK_OK;
    for (const Cand& c : cands) {
        ctx->batch_persistent = c.persistent;
        ctx->ctas_per_sm = c.per_sm;
        ctx->threads_per_cta = c.threads;
        ctx->packet_rays = c.packet;
        ctx->tile_w_log = c.twl;
        float ms = 1e30f;
        for (int rep = 0; rep < 3 && rc == AOK_OK; rep++) {
            cudaEventRecord(e0, st);
            rc = render_batch_impl(ctx, views, n, stream, false);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms = std::min(ms, t);  // the first run warms caches
        }
        if (rc) break;
        if (ms < best) {
            best = ms;
            bc = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) bc = {keep_p, keep[0], keep[1], keep[2], keep[3]};
    ctx->batch_persistent = bc.persistent;
    ctx->ctas_per_sm = bc.per_sm;
    ctx->threads_per_cta = bc.threads;
    ctx->packet_rays = bc.packet;
    ctx->tile_w_log = bc.twl;
    if (rc) return rc;
    if (best_ms) *best_ms = best;
    return AOK_OK;
}

int aok_serve_start(aok_ctx* ctx, uint32_t max_slots, uint32_t max_batch, uint32_t n_streams) {
    if (!ctx || ctx->serve || !max_slots || !max_batch || !n_streams || n_streams > 16) return AOK_E_INVALID;
    cudaSetDevice(ctx->device);
    auto* S = new ServeState();
    S->max_slots = max_slots;
    S->max_batch = std::min<uint32_t>(max_batch, 4096);
    const uint32_t ngroups = (S->max_batch + kBatchViews - 1) / kBatchViews;
    for (uint32_t i = 0; i < n_streams; i++) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return AOK_E_CUDA;
        S->streams.push_back(s);
        unsigned long long* c = nullptr;
        int st = dev_alloc(ctx, (void**)&c, 2 * ngroups * sizeof(unsigned long long));
        if (st) return st;
        cudaMemset(c, 0, 2 * ngroups * sizeof(unsigned long long));
        S->counters.push_back(c);
        S->stream_busy.push_back(0);
        for (int k = 0; k < 2; k++) {
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return AOK_E_CUDA;
            S->beam_ev.push_back(e);
        }
    }
    if (cudaStreamCreateWithFlags(&S->beam_stream, cudaStreamNonBlocking) != cudaSuccess) return AOK_E_CUDA;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return AOK_E_CUDA;
    }
    uint64_t keep = (uint64_t)ctx->budget;
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaDeviceSynchronize();
    ctx->serve = S;
    S->loop = std::thread(serve_loop, ctx);
    return AOK_OK;
}

int aok_serve_stop(aok_ctx* ctx) {
    if (!ctx || !ctx->serve) return AOK_OK;
    ServeState* S = ctx->serve;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        // requests never admitted are cancelled
        for (uint64_t id : S->pending) {
            auto it = S->tickets.find(id);
            if (it != S->tickets.end() && it->second.state == kQueued) {
                it->second.state = kFailed;
                it->second.status = AOK_E_TIMEOUT;
            }
        }
        S->pending.clear();
    }
    wake_loop(S);
    if (S->loop.joinable()) S->loop.join();
    cudaSetDevice(ctx->device);
    for (auto& kv : S->tickets) free_ticket_memory(ctx, kv.second, S->streams[0]);
    for (cudaStream_t s : S->streams) cudaStreamSynchronize(s);
    if (S->beam_stream) {
        cudaStreamSynchronize(S->beam_stream);
        cudaStreamDestroy(S->beam_stream);
    }
    for (cudaEvent_t e : S->beam_ev) cudaEventDestroy(e);
    for (size_t i = 0; i < S->streams.size(); i++) {
        dev_free(ctx, S->counters[i], 0);
        cudaStreamDestroy(S->streams[i]);
    }
    for (cudaEvent_t e : S->free_events) cudaEventDestroy(e);
    for (auto& f : S->inflight) {
        cudaEventDestroy(f.done);
        delete f.flag;
    }
    if (S->pool) {
        cudaDeviceSynchronize();  // frees of the pool's frames are complete
        cudaMemPoolDestroy(S->pool);
        S->pool = nullptr;
    }
    // counters were charged: give the bytes back
    const uint32_t ngroups = (S->max_batch + kBatchViews - 1) / kBatchViews;
    uncharge(ctx, S->streams.size() * 2 * ngroups * sizeof(unsigned long long));
    delete S;
    ctx->serve = nullptr;
    return AOK_OK;
}

int aok_serve_submit(aok_ctx* ctx, const aok_request* req, uint64_t* ticket) {
    if (!ctx || !req || !ticket) return AOK_E_INVALID;
    ServeState* S = ctx->serve;
    if (!S) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, req->scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    CamDev cd;
    int st = make_cam(ctx, sc, &req->cam, req->lod_threshold_px, &cd);
    if (st) return st;
    if (request_bytes(ctx, sc, req->cam) > ctx->budget) return AOK_E_OOM;  // can never be admitted
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) return AOK_E_INVALID;
        if (S->pending.size() >= 65536) return AOK_E_BUSY;
        const uint64_t id = ++S->next_ticket;
        Ticket t;
        t.req = *req;
        t.t_submit = now_ns();
        S->tickets.emplace(id, t);
        S->pending.push_back(id);
        *ticket = id;
    }
    wake_loop(S);
    return AOK_OK;
}

static int poll_locked(ServeState* S, uint64_t ticket, aok_frame* out) {
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return AOK_E_INVALID;
    const Ticket& t = it->second;
    if (t.state == kFailed) return t.status;
    if (t.state != kDone) return AOK_PENDING;
    if (out) {
        out->hit = t.hit;
        out->t = t.t;
    }
    return AOK_OK;
}

int aok_serve_poll(aok_ctx* ctx, uint64_t ticket, aok_frame* out) {
    if (!ctx || !ctx->serve) return AOK_E_INVALID;
    std::lock_guard<std::mutex> g(ctx->serve->mu);
    return poll_locked(ctx->serve, ticket, out);
}

int aok_serve_wait(aok_ctx* ctx, uint64_t ticket, uint32_t timeout_ms, aok_frame* out) {
    if (!ctx || !ctx->serve) return AOK_E_INVALID;
    ServeState* S = ctx->serve;
    std::unique_lock<std::mutex> g(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        const int r = poll_locked(S, ticket, out);
        if (r != AOK_PENDING) return r;
        if (S->done_cv.wait_until(g, deadline) == std::cv_status::timeout) {
            const int r2 = poll_locked(S, ticket, out);
            return r2 == AOK_PENDING ? AOK_E_TIMEOUT : r2;
        }
    }
}

int aok_serve_times(aok_ctx* ctx, uint64_t ticket, uint64_t* submit_ns, uint64_t* done_ns) {
    if (!ctx || !ctx->serve) return AOK_E_INVALID;
    std::lock_guard<std::mutex> g(ctx->serve->mu);
    auto it = ctx->serve->tickets.find(ticket);
    if (it == ctx->serve->tickets.end()) return AOK_E_INVALID;
    if (submit_ns) *submit_ns = it->second.t_submit;
    if (done_ns) *done_ns = it->second.t_done;
    return AOK_OK;
}

int aok_serve_release(aok_ctx* ctx, uint64_t ticket) {
    if (!ctx || !ctx->serve) return AOK_E_INVALID;
    ServeState* S = ctx->serve;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return AOK_E_INVALID;
    Ticket& t = it->second;
    if (t.state == kRunning) return AOK_E_BUSY;  // still on the GPU
    if (t.state == kQueued) {
        auto p = std::find(S->pending.begin(), S->pending.end(), ticket);
        if (p != S->pending.end()) S->pending.erase(p);
    }
    cudaSetDevice(ctx->device);
    free_ticket_memory(ctx, t, S->streams[0]);
    S->tickets.erase(it);
    wake_loop(S);
    return AOK_OK;
}

}  // extern "C"
