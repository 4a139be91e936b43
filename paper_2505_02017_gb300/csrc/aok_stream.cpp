// Asynchronous chunk streaming (Aokana Sec. 3.4): worker threads load the
// (chunk, LOD)s a camera needs while frames render; loads and evictions are
// installed in the descriptor table at frame boundaries, by a kernel on the
// rendering stream; evicted pool space is reused only after the frames that
// could still read it have finished.  Optionally the plans of the camera
// extrapolated along its last displacement are loaded ahead of need.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_set>
#include <vector>

#include "aok_runtime.h"

using namespace aok;

namespace {

struct Request {
    uint32_t rank;  // 0: the current plan; k > 0: the k-th extrapolated plan (loaded ahead of need)
    uint32_t lod;
    double dist2;   // squared distance from the camera to the region's centre
    int64_t chunk;
};

// Heap order: the current plan before the extrapolated ones (nearest in time
// first); within a plan the paper's order, coarser LODs first, then the
// regions nearest the camera.  std::push_heap keeps the "largest" on top, so
// "less" means "loaded later".
struct LoadsLater {
    bool operator()(const Request& a, const Request& b) const {
        if (a.rank != b.rank) return a.rank > b.rank;
        if (a.lod != b.lod) return a.lod < b.lod;
        if (a.dist2 != b.dist2) return a.dist2 > b.dist2;
        return a.chunk > b.chunk;
    }
};

struct Loaded {
    int64_t chunk;
    uint32_t lod;
    ChunkAlloc alloc;
    ChunkRef ref;
};

struct Quarantined {
    cudaEvent_t done;
    std::vector<ChunkAlloc> allocs;
};

uint64_t alloc_bytes(const ChunkAlloc& a) { return a.node_n * 4 + a.leaf_n * 8 + a.mat_n; }

}  // namespace

struct aok_stream {
    aok_ctx* ctx = nullptr;
    uint32_t scene_id = 0;
    Scene* sc = nullptr;
    aok_chunk_source_fn source = nullptr;
    aok_chunk_release_fn release = nullptr;
    void* user = nullptr;
    int L = 0;
    int64_t n = 0;
    int gx = 0, gy = 0;

    std::mutex mu;
    std::condition_variable work_cv, idle_cv;
    bool stop = false;
    std::atomic<bool> detached{false};  // its scene was destroyed: workers joined, calls refused
    std::vector<uint8_t> want;      // planned LOD per region (0xFF: none)
    std::vector<uint8_t> ahead;     // LODs of the extrapolated plans per region (bitmask)
    std::vector<uint8_t> resident;  // installed LODs per region (bitmask)
    std::vector<uint8_t> pending;   // LODs queued, loading or loaded-not-installed (bitmask)
    std::vector<Request> heap;
    std::vector<Request> deferred;  // loads that did not fit in the pools
    std::vector<Loaded> loaded;
    std::deque<Quarantined> quarantine;
    int running = 0;
    std::vector<std::thread> workers;

    uint64_t res_count = 0, res_bytes = 0, max_count = 0, max_bytes = 0;
    uint64_t n_installed = 0, n_evicted = 0, n_cancelled = 0, n_failed = 0, n_deferred = 0;
    uint64_t n_missing = 0;  // planned regions whose planned LOD was not installed at the last update
    uint64_t n_planned = 0;  // regions the last update planned
    uint64_t n_ahead_installed = 0;  // installs of LODs only the extrapolated plans wanted

    // prefetch along the camera's motion (aok_stream_set_prefetch)
    int ahead_frames = 0, ahead_samples = 0;
    bool have_prev = false;
    double prev_origin[3] = {0, 0, 0};

    // the LODs region c needs: its planned one and those of the extrapolated plans
    uint8_t needed(int64_t c) const { return (uint8_t)((want[c] != 0xFF ? 1u << want[c] : 0u) | ahead[c]); }
    void worker();
};

void aok_stream::worker() {
    cudaSetDevice(ctx->device);
    // each worker stages and copies on its own pinned buffer and stream
    Staging sg;
    sg.min_cap = (size_t)8 << 20;
    if (cudaStreamCreateWithFlags(&sg.stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        sg.stream = nullptr;
    }
    for (;;) {
        Request r;
        {
            std::unique_lock<std::mutex> lk(mu);
            work_cv.wait(lk, [&] { return stop || !heap.empty(); });
            if (stop) break;
            std::pop_heap(heap.begin(), heap.end(), LoadsLater());
            r = heap.back();
            heap.pop_back();
            if (!((needed(r.chunk) >> r.lod) & 1u)) {  // the plan moved on: cancel
                pending[r.chunk] &= (uint8_t)~(1u << r.lod);
                n_cancelled++;
                if (heap.empty() && running == 0) idle_cv.notify_all();
                continue;
            }
            running++;
        }
        const int cx = (int)(r.chunk % gx), cy = (int)((r.chunk / gx) % gy), cz = (int)(r.chunk / ((int64_t)gx * gy));
        aok_chunk_blob blob;
        std::memset(&blob, 0, sizeof(blob));
        void* handle = nullptr;
        int st = source(user, cx, cy, cz, r.lod, &blob, &handle) == 0 ? AOK_OK : AOK_E_INVALID;
        ChunkAlloc a;
        ChunkRef ref;
        if (st == AOK_OK) st = sg.stream ? stage_chunk(ctx, sc, r.chunk * L + r.lod, r.lod, &blob, false, &sg, &sc->mu,
                                                       &a, &ref)
                                         : AOK_E_CUDA;
        if (handle) release(user, handle);
        {
            std::lock_guard<std::mutex> lk(mu);
            running--;
            if (st == AOK_OK) {
                loaded.push_back({r.chunk, r.lod, a, ref});
            } else if (st == AOK_E_OOM) {
                deferred.push_back(r);  // retried after the next evictions
                n_deferred++;
            } else {
                pending[r.chunk] &= (uint8_t)~(1u << r.lod);
                n_failed++;
            }
            if (heap.empty() && running == 0) idle_cv.notify_all();
        }
    }
    if (sg.buf) cudaFreeHost(sg.buf);
    if (sg.stream) cudaStreamDestroy(sg.stream);
}

namespace aok {

void stream_detach(aok_stream* s) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->work_cv.notify_all();
    for (std::thread& t : s->workers) t.join();
    s->workers.clear();
    cudaSetDevice(s->ctx->device);
    {
        std::lock_guard<std::mutex> g(s->sc->mu);
        for (Loaded& ld : s->loaded) free_alloc(s->sc, ld.alloc);
        for (Quarantined& q : s->quarantine) {
            cudaEventSynchronize(q.done);
            for (ChunkAlloc& a : q.allocs) free_alloc(s->sc, a);
            cudaEventDestroy(q.done);
        }
    }
    s->loaded.clear();
    s->quarantine.clear();
    {
        // queued requests are dropped; a thread blocked in aok_stream_wait returns
        std::lock_guard<std::mutex> lk(s->mu);
        s->heap.clear();
        s->deferred.clear();
        s->detached = true;
        s->ctx = nullptr;
        s->sc = nullptr;
    }
    s->idle_cv.notify_all();
}

}  // namespace aok

extern "C" {

int aok_stream_create(aok_ctx* ctx, uint32_t scene, aok_chunk_source_fn source, aok_chunk_release_fn release,
                      void* user, int32_t n_threads, aok_stream** out) {
    if (!ctx || !source || !release || !out || n_threads < 1 || n_threads > 256) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    aok_stream* s = new (std::nothrow) aok_stream();
    if (!s) return AOK_E_OOM;
    s->ctx = ctx;
    s->scene_id = scene;
    s->sc = sc;
    s->source = source;
    s->release = release;
    s->user = user;
    s->L = sc->desc.n_lods;
    s->n = sc->n_chunks;
    s->gx = sc->desc.grid[0];
    s->gy = sc->desc.grid[1];
    s->want.assign((size_t)s->n, 0xFF);
    s->ahead.assign((size_t)s->n, 0);
    s->resident.assign((size_t)s->n, 0);
    s->pending.assign((size_t)s->n, 0);
    {
        // adopt what is already installed
        std::lock_guard<std::mutex> g(sc->mu);
        for (int64_t c = 0; c < s->n; c++)
            for (int l = 0; l < s->L; l++) {
                const ChunkAlloc& a = sc->alloc[(size_t)(c * s->L + l)];
                const ChunkRef& d = sc->h_desc[(size_t)(c * s->L + l)];
                if (d.root != kNone || (d.lod & kResidentBit)) {
                    s->resident[c] |= (uint8_t)(1u << l);
                    s->res_count++;
                    s->res_bytes += alloc_bytes(a);
                }
            }
        s->max_count = s->res_count;
        s->max_bytes = s->res_bytes;
    }
    {
        std::lock_guard<std::mutex> g(sc->mu);
        sc->streams.push_back(s);
    }
    for (int i = 0; i < n_threads; i++) s->workers.emplace_back([s] { s->worker(); });
    *out = s;
    return AOK_OK;
}

int aok_stream_update(aok_stream* s, const aok_camera* cam, double tau, void* stream) {
    if (!s || !cam) return AOK_E_INVALID;
    if (s->detached) return AOK_E_NOT_RESIDENT;
    aok_ctx* ctx = s->ctx;
    Scene* sc = s->sc;
    std::vector<uint8_t> plan((size_t)s->n);
    int st = aok_plan_residency(ctx, s->scene_id, cam, tau, plan.data(), nullptr);
    if (st) return st;
    // extrapolated plans: the camera moved on by its last displacement for
    // frames * k / samples more updates (k = 1 .. samples)
    std::vector<uint8_t> ahead((size_t)s->n, 0), ahead_rank;
    int ahead_frames, ahead_samples;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        ahead_frames = s->ahead_frames;
        ahead_samples = s->ahead_samples;
    }
    if (ahead_frames > 0 && s->have_prev) {
        ahead_rank.assign((size_t)s->n * s->L, 0);
        std::vector<uint8_t> pk((size_t)s->n);
        for (int k = 1; k <= ahead_samples; k++) {
            aok_camera ck = *cam;
            const double f = (double)ahead_frames * k / ahead_samples;
            for (int a = 0; a < 3; a++) {
                // on the 2^-12 grid camera origins take (exact in binary32 after rounding)
                const double o = cam->origin[a] + f * ((double)cam->origin[a] - s->prev_origin[a]);
                ck.origin[a] = (float)(std::nearbyint(std::min(std::max(o, -131000.0), 131000.0) * 4096.0) / 4096.0);
            }
            if (aok_plan_residency(ctx, s->scene_id, &ck, tau, pk.data(), nullptr) != AOK_OK) continue;
            for (int64_t c = 0; c < s->n; c++) {
                const uint8_t l = pk[c];
                if (l == 0xFF || l == plan[c] || ((ahead[c] >> l) & 1u)) continue;
                ahead[c] |= (uint8_t)(1u << l);
                ahead_rank[(size_t)(c * s->L + l)] = (uint8_t)k;
            }
        }
    }
    for (int a = 0; a < 3; a++) s->prev_origin[a] = cam->origin[a];
    s->have_prev = true;
    CamDev cd;
    st = make_cam(ctx, sc, cam, tau, &cd);
    if (st) return st;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_status(ctx, cudaGetLastError());
    const double M = sc->desc.chunk_res;
    std::vector<DescPatch> patches;
    std::vector<ChunkAlloc> dead;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        std::lock_guard<std::mutex> g(sc->mu);
        s->want.swap(plan);
        s->ahead.swap(ahead);
        auto none_ref = [](uint32_t lod) {
            ChunkRef r;
            std::memset(&r, 0, sizeof(r));
            r.root = kNone;
            r.lod = lod;
            return r;
        };
        // 1. install finished loads (one no plan wants any more frees its space at once: never visible)
        for (Loaded& ld : s->loaded) {
            const size_t di = (size_t)(ld.chunk * s->L + ld.lod);
            s->pending[ld.chunk] &= (uint8_t)~(1u << ld.lod);
            if (!((s->needed(ld.chunk) >> ld.lod) & 1u) && s->want[ld.chunk] == 0xFF) {
                free_alloc(sc, ld.alloc);
                s->n_cancelled++;
                continue;
            }
            if (s->want[ld.chunk] != ld.lod && ((s->ahead[ld.chunk] >> ld.lod) & 1u)) s->n_ahead_installed++;
            patches.push_back({(uint64_t)di, ld.ref});
            sc->alloc[di] = ld.alloc;
            sc->h_desc[di] = ld.ref;
            s->resident[ld.chunk] |= (uint8_t)(1u << ld.lod);
            s->res_count++;
            s->res_bytes += alloc_bytes(ld.alloc);
            s->n_installed++;
        }
        s->loaded.clear();
        // 2. evictions: a region's other LODs go once its planned LOD is installed,
        //    all of them once it is no longer planned; LODs an extrapolated plan wants stay
        for (int64_t c = 0; c < s->n; c++) {
            const uint8_t res = s->resident[c];
            if (!res) continue;
            const uint8_t w = s->want[c];
            const bool settled = w == 0xFF || (res >> w) & 1u;
            if (!settled) continue;
            for (int l = 0; l < s->L; l++) {
                if (!((res >> l) & 1u) || l == (int)w || ((s->ahead[c] >> l) & 1u)) continue;
                const size_t di = (size_t)(c * s->L + l);
                patches.push_back({(uint64_t)di, none_ref((uint32_t)l)});
                s->res_bytes -= std::min(s->res_bytes, alloc_bytes(sc->alloc[di]));
                dead.push_back(sc->alloc[di]);
                sc->alloc[di] = ChunkAlloc();
                sc->h_desc[di] = none_ref((uint32_t)l);
                s->resident[c] &= (uint8_t)~(1u << l);
                s->res_count--;
                s->n_evicted++;
            }
        }
        s->max_count = std::max(s->max_count, s->res_count);
        s->max_bytes = std::max(s->max_bytes, s->res_bytes);
        // 3. the load queue, rebuilt from the plans: queued and deferred requests
        //    no plan wants are dropped, the others re-ranked; then the needed LODs
        //    neither installed nor on their way are queued
        for (const Request& r : s->heap) {
            s->pending[r.chunk] &= (uint8_t)~(1u << r.lod);
            if (!((s->needed(r.chunk) >> r.lod) & 1u)) s->n_cancelled++;
        }
        for (const Request& r : s->deferred) {
            s->pending[r.chunk] &= (uint8_t)~(1u << r.lod);
            if (!((s->needed(r.chunk) >> r.lod) & 1u)) s->n_cancelled++;
        }
        s->heap.clear();
        s->deferred.clear();
        s->n_missing = 0;
        s->n_planned = 0;
        for (int64_t c = 0; c < s->n; c++) {
            const uint8_t w = s->want[c];
            if (w != 0xFF) s->n_planned++;
            if (w != 0xFF && !((s->resident[c] >> w) & 1u)) s->n_missing++;
            uint8_t need = (uint8_t)(s->needed(c) & ~(s->resident[c] | s->pending[c]));
            if (!need) continue;
            const int cx = (int)(c % s->gx), cy = (int)((c / s->gx) % s->gy), cz = (int)(c / ((int64_t)s->gx * s->gy));
            const double q[3] = {(cx + 0.5) * M - cd.of[0], (cy + 0.5) * M - cd.of[1], (cz + 0.5) * M - cd.of[2]};
            const double d2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
            for (int l = 0; l < s->L; l++) {
                if (!((need >> l) & 1u)) continue;
                const uint32_t rank = l == (int)w ? 0u : (uint32_t)ahead_rank[(size_t)(c * s->L + l)];
                s->heap.push_back({rank, (uint32_t)l, d2, c});
                s->pending[c] |= (uint8_t)(1u << l);
            }
        }
        std::make_heap(s->heap.begin(), s->heap.end(), LoadsLater());
    }
    s->work_cv.notify_all();
    // 4. the descriptor changes, ordered before every later frame on `stream`;
    //    a descriptor changed twice (a load installed above and evicted at
    //    once because its region settled on another LOD) keeps only its last
    //    change, the eviction: its space is quarantined and must never be
    //    published
    {
        std::unordered_set<uint64_t> seen;
        size_t keep = patches.size();
        for (size_t i = patches.size(); i-- > 0;)
            if (seen.insert(patches[i].index).second) patches[--keep] = patches[i];
        patches.erase(patches.begin(), patches.begin() + (ptrdiff_t)keep);
    }
    for (size_t i = 0; i < patches.size(); i += kPatchMax) {
        DescPatches P;
        P.n = (uint32_t)std::min<size_t>(kPatchMax, patches.size() - i);
        P.pad = 0;
        std::memcpy(P.p, patches.data() + i, P.n * sizeof(DescPatch));
        if (aokk_patch_desc(sc->d_desc, &P, stream)) return cuda_status(ctx, cudaGetLastError());
    }
    // 5. evicted space waits for the frames enqueued before the eviction
    if (!dead.empty()) {
        Quarantined q;
        if (cudaEventCreateWithFlags(&q.done, cudaEventDisableTiming) != cudaSuccess)
            return cuda_status(ctx, cudaGetLastError());
        if (cudaEventRecord(q.done, (cudaStream_t)stream) != cudaSuccess) {
            cudaEventDestroy(q.done);
            return cuda_status(ctx, cudaGetLastError());
        }
        q.allocs.swap(dead);
        std::lock_guard<std::mutex> lk(s->mu);
        s->quarantine.push_back(std::move(q));
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        bool freed = false;
        while (!s->quarantine.empty() && cudaEventQuery(s->quarantine.front().done) == cudaSuccess) {
            std::lock_guard<std::mutex> g(sc->mu);
            for (ChunkAlloc& a : s->quarantine.front().allocs) free_alloc(sc, a);
            cudaEventDestroy(s->quarantine.front().done);
            s->quarantine.pop_front();
            freed = true;
        }
        cudaGetLastError();  // cudaErrorNotReady from the query is not an error
        if (freed && !s->deferred.empty()) {
            for (Request& r : s->deferred) {
                if (!((s->needed(r.chunk) >> r.lod) & 1u)) {
                    s->pending[r.chunk] &= (uint8_t)~(1u << r.lod);
                    s->n_cancelled++;
                    continue;
                }
                s->heap.push_back(r);
                std::push_heap(s->heap.begin(), s->heap.end(), LoadsLater());
            }
            s->deferred.clear();
            s->work_cv.notify_all();
        }
    }
    return AOK_OK;
}

int aok_stream_wait(aok_stream* s, int32_t timeout_ms) {
    if (!s) return AOK_E_INVALID;
    if (s->detached) return AOK_E_NOT_RESIDENT;
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [&] { return s->detached || (s->heap.empty() && s->running == 0); };
    if (timeout_ms < 0) s->idle_cv.wait(lk, idle);
    else if (!s->idle_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle)) return AOK_E_TIMEOUT;
    return s->detached ? AOK_E_NOT_RESIDENT : AOK_OK;
}

int aok_stream_stats(aok_stream* s, uint64_t* st) {
    if (!s || !st) return AOK_E_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t v[15] = {s->res_count, s->res_bytes, s->max_count, s->max_bytes, (uint64_t)s->heap.size(),
                            (uint64_t)s->running, (uint64_t)s->loaded.size(), s->n_installed, s->n_evicted,
                            s->n_cancelled, s->n_failed, s->n_deferred, s->n_missing, s->n_planned,
                            s->n_ahead_installed};
    std::memcpy(st, v, sizeof(v));
    return AOK_OK;
}

int aok_stream_set_prefetch(aok_stream* s, int32_t frames, int32_t samples) {
    if (!s || frames < 0 || frames > 1000 || (frames > 0 && (samples < 1 || samples > 16))) return AOK_E_INVALID;
    if (s->detached) return AOK_E_NOT_RESIDENT;
    std::lock_guard<std::mutex> lk(s->mu);
    s->ahead_frames = frames;
    s->ahead_samples = frames > 0 ? samples : 0;
    return AOK_OK;
}

int aok_stream_resident(aok_stream* s, uint8_t* masks) {
    if (!s || !masks) return AOK_E_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memcpy(masks, s->resident.data(), s->resident.size());
    return AOK_OK;
}

int aok_stream_destroy(aok_stream* s) {
    if (!s) return AOK_E_INVALID;
    if (!s->detached) {
        {
            std::lock_guard<std::mutex> g(s->sc->mu);
            auto& v = s->sc->streams;
            v.erase(std::remove(v.begin(), v.end(), s), v.end());
        }
        stream_detach(s);
    }
    delete s;
    return AOK_OK;
}

}  // extern "C"
