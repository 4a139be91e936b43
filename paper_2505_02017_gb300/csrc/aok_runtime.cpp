// Host runtime of the C ABI (include/aok.h): context and HBM budget, scene
// pools, validating chunk upload with pointer rebasing, camera setup, and the
// per-frame select / render entry points.  Batched rendering and the serving
// loop live in aok_serve.cpp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "aok_runtime.h"

using namespace aok;

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
namespace aok {

int cuda_status(aok_ctx* ctx, cudaError_t e) {
    if (e == cudaSuccess) return AOK_OK;
    ctx->last_cuda = e;
    return AOK_E_CUDA;
}

int launch_failure(aok_ctx* ctx) { return cuda_status(ctx, aokk_take_launch_error()); }

int charge(aok_ctx* ctx, size_t bytes) {
    std::lock_guard<std::mutex> g(ctx->mem_mu);
    if (ctx->used + bytes > ctx->budget) return AOK_E_OOM;
    ctx->used += bytes;
    return AOK_OK;
}

void uncharge(aok_ctx* ctx, size_t bytes) {
    std::lock_guard<std::mutex> g(ctx->mem_mu);
    ctx->used -= std::min(ctx->used, bytes);
}

int dev_alloc(aok_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return AOK_OK;
    int st = charge(ctx, bytes);
    if (st) return st;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        uncharge(ctx, bytes);
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? AOK_E_OOM : cuda_status(ctx, e);
    }
    return AOK_OK;
}

void dev_free(aok_ctx* ctx, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    uncharge(ctx, bytes);
}

Scene* find_scene(aok_ctx* ctx, uint32_t id) {
    std::lock_guard<std::mutex> g(ctx->scene_mu);
    auto it = ctx->scenes.find(id);
    return it == ctx->scenes.end() ? nullptr : it->second;
}

static int ilog2i(int v) {
    int l = 0;
    while ((1 << l) < v) l++;
    return l;
}

// First-fit range allocator over a pool of `cap` units.
uint64_t Pool::alloc(uint64_t n) {
    if (n == 0) return 0;
    for (size_t i = 0; i < free_list.size(); i++) {
        if (free_list[i].second >= n) {
            uint64_t off = free_list[i].first;
            free_list[i].first += n;
            free_list[i].second -= n;
            if (!free_list[i].second) free_list.erase(free_list.begin() + (long)i);
            return off;
        }
    }
    if (used + n > cap) return kNoRange;
    uint64_t off = used;
    used += n;
    return off;
}

// Free ranges stay sorted by offset and merge with their neighbours; a range
// that ends at the bump pointer gives the space back to it.
void Pool::release(uint64_t off, uint64_t n) {
    if (!n) return;
    auto it = std::lower_bound(free_list.begin(), free_list.end(), std::make_pair(off, (uint64_t)0));
    it = free_list.insert(it, std::make_pair(off, n));
    if (it + 1 != free_list.end() && it->first + it->second == (it + 1)->first) {
        it->second += (it + 1)->second;
        free_list.erase(it + 1);
    }
    if (it != free_list.begin() && (it - 1)->first + (it - 1)->second == it->first) {
        (it - 1)->second += it->second;
        it = free_list.erase(it) - 1;
    }
    if (it->first + it->second == used) {
        used = it->first;
        free_list.erase(it);
    }
}

int make_cam(aok_ctx* ctx, const Scene* sc, const aok_camera* cam, double tau, CamDev* out) {
    (void)ctx;
    // the casting grid has (H + 7) / 8 rows of blocks (at most 65535), and pixel
    // indices are computed in int32 by some launches
    if (!cam || cam->width <= 0 || cam->height <= 0 || cam->height > kMaxImageHeight ||
        (int64_t)cam->width * cam->height >= (1ll << 31))
        return AOK_E_INVALID;
    if (!(tau > 0.0) || !std::isfinite(tau)) return AOK_E_INVALID;
    if (!(cam->tan_half_fovy > 0.0f) || !std::isfinite(cam->tan_half_fovy)) return AOK_E_INVALID;
    std::memset(out, 0, sizeof(*out));
    for (int i = 0; i < 9; i++) {
        if (!std::isfinite(cam->R[i])) return AOK_E_INVALID;
        out->R[i] = cam->R[i];
    }
    out->tan_half = cam->tan_half_fovy;
    out->W = cam->width;
    out->H = cam->height;
    out->aspect = (float)cam->width / (float)cam->height;  // the ray's W / H: one IEEE binary32 division
    for (int a = 0; a < 3; a++) {
        const double o = cam->origin[a];
        if (!std::isfinite(o) || std::fabs(o) >= 131072.0) return AOK_E_INVALID;
        const double f = o * (double)(1 << kFix);
        if (f != std::floor(f)) return AOK_E_INVALID;  // not on the 2^-12 grid
        out->O[a] = (int32_t)f;
        out->of[a] = cam->origin[a];
    }
    // view-pyramid side planes (conservative): every pixel direction
    // d = u c0 + v c1 - c2 has |u| < U = t W/H and |v| < V = t
    double c[3][3];
    for (int j = 0; j < 3; j++)
        for (int i = 0; i < 3; i++) c[j][i] = cam->R[3 * i + j];
    const double t = cam->tan_half_fovy, asp = (double)cam->width / (double)cam->height;
    const double U = t * asp * (1.0 + 1e-5), V = t * (1.0 + 1e-5);
    auto cross = [](const double* a, const double* b, double* r) {
        r[0] = a[1] * b[2] - a[2] * b[1];
        r[1] = a[2] * b[0] - a[0] * b[2];
        r[2] = a[0] * b[1] - a[1] * b[0];
    };
    for (int p = 0; p < 4; p++) {
        // p = 0: u = +U, 1: u = -U, 2: v = +V, 3: v = -V
        const int along = p < 2 ? 0 : 1, other = p < 2 ? 1 : 0;
        const double s = (p % 2 == 0) ? 1.0 : -1.0;
        const double lim = p < 2 ? U : V;
        double edge[3], n[3];
        for (int i = 0; i < 3; i++) edge[i] = s * lim * c[along][i] - c[2][i];
        cross(c[other], edge, n);
        double dot = n[0] * c[along][0] + n[1] * c[along][1] + n[2] * c[along][2];
        if (s * dot < 0) for (int i = 0; i < 3; i++) n[i] = -n[i];
        double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int i = 0; i < 3; i++) out->planes[p][i] = len > 0 ? (float)(n[i] / len) : 0.0f;
        out->planes[p][3] = 0.0f;
    }
    // StreamingFactor from the pixel threshold (fixed FP64 operation order)
    const double fpx = (double)cam->height / (2.0 * (double)cam->tan_half_fovy);
    out->sf = fpx / (tau * (double)sc->desc.chunk_res);
    return AOK_OK;
}

SceneDev scene_dev(const Scene* sc) {
    SceneDev s;
    s.nodes = sc->d_nodes;
    s.leaves = sc->d_leaves;
    s.mats = sc->d_mats;
    s.desc = sc->d_desc;
    for (int a = 0; a < 3; a++) s.grid[a] = sc->desc.grid[a];
    s.mlog = sc->mlog;
    s.n_lods = sc->desc.n_lods;
    s.view_dist = sc->desc.view_dist;
    return s;
}

}  // namespace aok

// ---------------------------------------------------------------------------
// blob validation + rebasing (host)
// ---------------------------------------------------------------------------
static int validate_blob(const aok_chunk_blob* b, int res, int M) {
    const uint64_t nw = b->n_node_words;
    if (nw == 0) return (b->n_leaves == 0 && b->n_mats == 0) ? AOK_OK : AOK_E_CORRUPT;
    if (!b->nodes || b->root >= nw || (b->n_leaves && !b->leaves) || (b->n_mats && !b->mats)) return AOK_E_CORRUPT;
    if (nw > 0xFFFFFFFFull || b->n_leaves > 0xFFFFFFFFull) return AOK_E_CORRUPT;
    const int n_int = ilog2i(res) - 2;
    std::vector<int8_t> depth(nw, -1);
    std::vector<std::pair<uint32_t, int>> st;
    st.emplace_back(b->root, 0);
    while (!st.empty()) {
        auto [node, d] = st.back();
        st.pop_back();
        if (depth[node] >= 0) {
            if (depth[node] != d) return AOK_E_CORRUPT;
            continue;
        }
        depth[node] = (int8_t)d;
        if ((uint64_t)node + 2 > nw) return AOK_E_CORRUPT;
        const uint32_t hdr = b->nodes[node];
        if ((hdr >> 8) != 0 || (hdr & 0xFFu) == 0) return AOK_E_CORRUPT;
        const int k = __builtin_popcount(hdr);
        if ((uint64_t)node + 2 + k > nw) return AOK_E_CORRUPT;
        const bool leafkids = d == n_int - 1;
        uint64_t sum = 0;
        for (int i = 0; i < k; i++) {
            const uint32_t ch = b->nodes[node + 2 + i];
            if (leafkids) {
                if (ch >= b->n_leaves || b->leaves[ch] == 0) return AOK_E_CORRUPT;
                sum += (uint64_t)__builtin_popcountll(b->leaves[ch]);
            } else {
                if ((uint64_t)ch + 2 > nw) return AOK_E_CORRUPT;
                sum += b->nodes[ch + 1];
                st.emplace_back(ch, d + 1);
            }
        }
        if (sum != b->nodes[node + 1]) return AOK_E_CORRUPT;
    }
    if ((uint64_t)b->nodes[b->root + 1] != b->n_mats) return AOK_E_CORRUPT;
    for (int a = 0; a < 3; a++)
        if (b->aabb_lo[a] < 0 || b->aabb_hi[a] > M || b->aabb_lo[a] >= b->aabb_hi[a]) return AOK_E_CORRUPT;
    return AOK_OK;
}

// Device layout of a validated blob: every node reachable from the root,
// in ascending blob order, as [header, count, (child, prefix) x k] where
// prefix = summed counts of the earlier children, so that the depth-first
// index of a voxel needs one word per level instead of every earlier
// sibling's count.  Child pointers are rebased (node_base: device word
// offset of this chunk's nodes, leaf_base: of its leaves).  The header keeps
// the child mask in bits 0-7; bits 8-31 hold the box of the node's solid
// voxels within its cell, per axis (x, y, z from bit 8) a 4-bit lower bound
// and a 4-bit upper bound - 1 in 16ths of the cell's side (rounded outward),
// which the beam pass projects instead of the whole cell.  Returns the word
// count; with out == nullptr only sizes are computed.
static uint64_t layout_blob(const aok_chunk_blob* b, int res, uint32_t node_base, uint32_t leaf_base, uint32_t* out,
                            uint32_t* root_out) {
    const uint64_t nw = b->n_node_words;
    if (!nw) return 0;
    const int n_int = ilog2i(res) - 2;
    std::vector<int8_t> depth(nw, -1);
    std::vector<uint32_t> st{b->root};
    depth[b->root] = 0;
    while (!st.empty()) {
        const uint32_t node = st.back();
        st.pop_back();
        if (depth[node] == n_int - 1) continue;
        const int k = __builtin_popcount(b->nodes[node]);
        for (int i = 0; i < k; i++) {
            const uint32_t ch = b->nodes[node + 2 + i];
            if (depth[ch] < 0) {
                depth[ch] = (int8_t)(depth[node] + 1);
                st.push_back(ch);
            }
        }
    }
    std::vector<uint32_t> off(out ? nw : 0, 0);
    uint64_t w = 0;
    for (uint64_t i = 0; i < nw; i++) {
        if (depth[i] < 0) continue;
        if (out) off[i] = (uint32_t)w;
        w += 2 + 2 * (uint64_t)__builtin_popcount(b->nodes[i]);
    }
    if (!out) return w;
    // solid-voxel box of every node in its own cell (LOD voxels), deepest first
    std::vector<uint32_t> order;
    for (uint64_t i = 0; i < nw; i++)
        if (depth[i] >= 0) order.push_back((uint32_t)i);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t c) { return depth[a] > depth[c]; });
    std::vector<uint16_t> box(6 * nw, 0);  // lo x, y, z, hi x, y, z
    for (uint32_t i : order) {
        const int side = res >> depth[i], half = side >> 1;
        const bool leafkids = depth[i] == n_int - 1;
        int lo[3] = {side, side, side}, hi[3] = {0, 0, 0};
        uint32_t m = b->nodes[i] & 0xFFu;
        for (int c = 0; m; c++) {
            const int oc = __builtin_ctz(m);
            m &= m - 1;
            const uint32_t ch = b->nodes[i + 2 + c];
            int clo[3], chi[3];
            if (leafkids) {  // a 4^3 leaf mask, bit x + 4y + 16z: the rows present per axis
                const uint64_t lm = b->leaves[ch];
                uint64_t t = lm | (lm >> 32);
                t |= t >> 16;  // bit x + 4y: any z
                const uint32_t xy = (uint32_t)t & 0xFFFFu;
                const uint32_t bits[3] = {
                    (xy | xy >> 4 | xy >> 8 | xy >> 12) & 0xFu,
                    (uint32_t)((xy & 0xFu) != 0) | (uint32_t)((xy & 0xF0u) != 0) << 1 |
                        (uint32_t)((xy & 0xF00u) != 0) << 2 | (uint32_t)((xy & 0xF000u) != 0) << 3,
                    (uint32_t)((lm & 0xFFFFull) != 0) | (uint32_t)(((lm >> 16) & 0xFFFFull) != 0) << 1 |
                        (uint32_t)(((lm >> 32) & 0xFFFFull) != 0) << 2 | (uint32_t)((lm >> 48) != 0) << 3};
                for (int a = 0; a < 3; a++) {
                    clo[a] = __builtin_ctz(bits[a]);
                    chi[a] = 32 - __builtin_clz(bits[a]);
                }
            } else {
                for (int a = 0; a < 3; a++) {
                    clo[a] = box[6 * (size_t)ch + a];
                    chi[a] = box[6 * (size_t)ch + 3 + a];
                }
            }
            for (int a = 0; a < 3; a++) {
                const int at = ((oc >> a) & 1) * half;
                lo[a] = std::min(lo[a], at + clo[a]);
                hi[a] = std::max(hi[a], at + chi[a]);
            }
        }
        for (int a = 0; a < 3; a++) {
            box[6 * (size_t)i + a] = (uint16_t)lo[a];
            box[6 * (size_t)i + 3 + a] = (uint16_t)hi[a];
        }
    }
    for (uint64_t i = 0; i < nw; i++) {
        if (depth[i] < 0) continue;
        const uint32_t hdr = b->nodes[i], o = off[i];
        const int k = __builtin_popcount(hdr & 0xFFu);
        const bool leafkids = depth[i] == n_int - 1;
        const int side = res >> depth[i];
        uint32_t q = 0;
        for (int a = 0; a < 3; a++) {
            const uint32_t ql = (uint32_t)(box[6 * i + a] * 16 / side);                  // rounded down
            const uint32_t qh = (uint32_t)((box[6 * i + 3 + a] * 16 + side - 1) / side);  // rounded up, >= 1
            q |= (ql | (qh - 1) << 4) << (8 * a);
        }
        out[o] = (hdr & 0xFFu) | q << 8;
        out[o + 1] = b->nodes[i + 1];
        uint32_t pre = 0;
        for (int c = 0; c < k; c++) {
            const uint32_t ch = b->nodes[i + 2 + c];
            out[o + 2 + 2 * c] = leafkids ? ch + leaf_base : off[ch] + node_base;
            out[o + 3 + 2 * c] = pre;
            pre += leafkids ? (uint32_t)__builtin_popcountll(b->leaves[ch]) : b->nodes[ch + 1];
        }
    }
    *root_out = off[b->root] + node_base;
    return w;
}

static void pipe_release(aok_ctx* ctx);

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* aok_status_str(int s) {
    switch (s) {
        case AOK_OK: return "ok";
        case AOK_PENDING: return "pending";
        case AOK_E_INVALID: return "invalid argument";
        case AOK_E_OOM: return "out of device memory budget";
        case AOK_E_NOT_RESIDENT: return "not resident";
        case AOK_E_TIMEOUT: return "timeout";
        case AOK_E_CUDA: return "CUDA error";
        case AOK_E_BUSY: return "busy";
        case AOK_E_CORRUPT: return "corrupt chunk blob";
        default: return "unknown status";
    }
}

int aok_create(aok_ctx** out, int device, size_t budget) {
    if (!out) return AOK_E_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return AOK_E_INVALID;
    }
    if (cudaSetDevice(device) != cudaSuccess) return AOK_E_CUDA;
    aok_ctx* ctx = new (std::nothrow) aok_ctx();
    if (!ctx) return AOK_E_OOM;
    ctx->device = device;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    ctx->budget = budget ? budget : (size_t)((double)fr * 0.9);
    if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&ctx->pinned_word, sizeof(uint32_t)) != cudaSuccess) {
        delete ctx;
        return AOK_E_CUDA;
    }
    if (dev_alloc(ctx, (void**)&ctx->d_counter, sizeof(uint32_t) * 16) != AOK_OK ||
        dev_alloc(ctx, (void**)&ctx->d_single_queue, 2 * sizeof(unsigned long long)) != AOK_OK ||
        cudaMemset(ctx->d_counter, 0, sizeof(uint32_t) * 16) != cudaSuccess ||
        cudaMemset(ctx->d_single_queue, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        delete ctx;
        return AOK_E_CUDA;
    }
    ctx->sm_count = aokk_sm_count(device);
    *out = ctx;
    return AOK_OK;
}

void aok_destroy(aok_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    aok_serve_stop(ctx);
    cudaDeviceSynchronize();
    std::vector<uint32_t> ids;
    for (auto& kv : ctx->scenes) ids.push_back(kv.first);
    for (uint32_t id : ids) aok_scene_destroy(ctx, id);
    batch_release(ctx);
    dev_free(ctx, ctx->host_hit_dev, ctx->host_frame_px * 16);
    dev_free(ctx, ctx->host_t_dev, ctx->host_frame_px * 4);
    dev_free(ctx, ctx->d_counter, sizeof(uint32_t) * 16);
    dev_free(ctx, ctx->d_single_queue, 2 * sizeof(unsigned long long));
    dev_free(ctx, ctx->tiles.block, ctx->tiles.bytes);
    dev_free(ctx, ctx->beam.qblock, ctx->beam.qbytes);
    dev_free(ctx, ctx->beam.bounds, ctx->beam.bounds_cap * 8);
    pipe_release(ctx);
    if (ctx->pipe.prep) cudaStreamDestroy(ctx->pipe.prep);
    if (ctx->pipe.render) cudaStreamDestroy(ctx->pipe.render);
    if (ctx->pipe.copy) cudaStreamDestroy(ctx->pipe.copy);
    if (ctx->staging) cudaFreeHost(ctx->staging);
    if (ctx->pinned_word) cudaFreeHost(ctx->pinned_word);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    delete ctx;
}

int aok_memory(aok_ctx* ctx, size_t* used, size_t* budget) {
    if (!ctx) return AOK_E_INVALID;
    std::lock_guard<std::mutex> g(ctx->mem_mu);
    if (used) *used = ctx->used;
    if (budget) *budget = ctx->budget;
    return AOK_OK;
}

int aok_scene_create(aok_ctx* ctx, const aok_scene_desc* d, uint32_t* scene_id) {
    if (!ctx || !d || !scene_id) return AOK_E_INVALID;
    const int M = d->chunk_res;
    if (M < 8 || M > 512 || (M & (M - 1)) || d->n_lods < 1 || (M >> (d->n_lods - 1)) < 8) return AOK_E_INVALID;
    for (int a = 0; a < 3; a++)
        if (d->grid[a] < 1 || (int64_t)d->grid[a] * M > 131072) return AOK_E_INVALID;
    if (d->node_words > 0x7FFFFFFFull || d->leaf_count > 0xFFFFFFFFull || !(d->view_dist >= 0.0f)) return AOK_E_INVALID;
    cudaSetDevice(ctx->device);
    Scene* sc = new Scene();
    sc->desc = *d;
    sc->mlog = ilog2i(M);
    sc->n_chunks = (int64_t)d->grid[0] * d->grid[1] * d->grid[2];
    sc->nodes.cap = std::max<uint64_t>(2 * d->node_words, 2);  // device layout: (child, prefix) pairs
    sc->leaves.cap = std::max<uint64_t>(d->leaf_count, 1);
    sc->mats.cap = std::max<uint64_t>(d->mat_bytes, 1);
    const size_t ndesc = (size_t)sc->n_chunks * d->n_lods;
    int st = dev_alloc(ctx, (void**)&sc->d_nodes, sc->nodes.cap * 4);
    if (!st) st = dev_alloc(ctx, (void**)&sc->d_leaves, sc->leaves.cap * 8);
    if (!st) st = dev_alloc(ctx, (void**)&sc->d_mats, sc->mats.cap);
    if (!st) st = dev_alloc(ctx, (void**)&sc->d_desc, ndesc * sizeof(ChunkRef));
    if (!st) st = dev_alloc(ctx, (void**)&sc->d_frame, (size_t)sc->n_chunks * sizeof(ChunkRef));
    if (st) {
        dev_free(ctx, sc->d_nodes, sc->nodes.cap * 4);
        dev_free(ctx, sc->d_leaves, sc->leaves.cap * 8);
        dev_free(ctx, sc->d_mats, sc->mats.cap);
        dev_free(ctx, sc->d_desc, ndesc * sizeof(ChunkRef));
        delete sc;
        return st;
    }
    ChunkRef empty;
    std::memset(&empty, 0, sizeof(empty));
    empty.root = kNone;
    sc->h_desc.assign(ndesc, empty);
    sc->alloc.assign(ndesc, ChunkAlloc());
    for (size_t i = 0; i < ndesc; i++) sc->h_desc[i].lod = (uint32_t)(i % d->n_lods);
    cudaError_t e = cudaMemcpy(sc->d_desc, sc->h_desc.data(), ndesc * sizeof(ChunkRef), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        int r = cuda_status(ctx, e);
        delete sc;
        return r;
    }
    std::lock_guard<std::mutex> g(ctx->scene_mu);
    uint32_t id = ++ctx->next_scene;
    ctx->scenes[id] = sc;
    *scene_id = id;
    return AOK_OK;
}

int aok_scene_destroy(aok_ctx* ctx, uint32_t id) {
    if (!ctx) return AOK_E_INVALID;
    Scene* sc;
    {
        std::lock_guard<std::mutex> g(ctx->scene_mu);
        auto it = ctx->scenes.find(id);
        if (it == ctx->scenes.end()) return AOK_E_NOT_RESIDENT;
        sc = it->second;
        ctx->scenes.erase(it);
    }
    cudaSetDevice(ctx->device);
    std::vector<aok_stream*> streams;
    {
        std::lock_guard<std::mutex> g(sc->mu);
        streams.swap(sc->streams);
    }
    for (aok_stream* s : streams) stream_detach(s);  // their workers write into this scene's pools
    cudaDeviceSynchronize();
    const size_t ndesc = (size_t)sc->n_chunks * sc->desc.n_lods;
    dev_free(ctx, sc->d_nodes, sc->nodes.cap * 4);
    dev_free(ctx, sc->d_leaves, sc->leaves.cap * 8);
    dev_free(ctx, sc->d_mats, sc->mats.cap);
    dev_free(ctx, sc->d_desc, ndesc * sizeof(ChunkRef));
    dev_free(ctx, sc->d_frame, (size_t)sc->n_chunks * sizeof(ChunkRef));
    delete sc;
    return AOK_OK;
}

static int chunk_index(const Scene* sc, int32_t cx, int32_t cy, int32_t cz, uint32_t lod, int64_t* out) {
    if (cx < 0 || cy < 0 || cz < 0 || cx >= sc->desc.grid[0] || cy >= sc->desc.grid[1] || cz >= sc->desc.grid[2] ||
        lod >= (uint32_t)sc->desc.n_lods)
        return AOK_E_INVALID;
    *out = ((int64_t)cx + (int64_t)sc->desc.grid[0] * ((int64_t)cy + (int64_t)sc->desc.grid[1] * cz)) * sc->desc.n_lods + lod;
    return AOK_OK;
}

}  // extern "C"

void aok::free_alloc(Scene* sc, ChunkAlloc& a) {
    sc->nodes.release(a.node_off, a.node_n);
    sc->leaves.release(a.leaf_off, a.leaf_n);
    sc->mats.release(a.mat_off, a.mat_n);
    a = ChunkAlloc();
}

// Colour blocks of a DFS colour array (Sec. 3.3): entries are taken left to
// right; one within tol = e_c * 255 of the current block's colour joins it and
// the colour becomes the rounded mean of the block's entries, any other opens
// a new block.
static void color_blocks(const uint8_t* v, uint64_t n, double e_c, std::vector<uint32_t>& first,
                         std::vector<uint8_t>& colour) {
    first.clear();
    colour.clear();
    const double tol = e_c * 255.0;
    uint64_t sum = 0, cnt = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (cnt && std::fabs((double)v[i] - (double)colour.back()) <= tol) {
            sum += v[i];
            cnt++;
            colour.back() = (uint8_t)((sum + cnt / 2) / cnt);
        } else {
            first.push_back((uint32_t)i);
            colour.push_back(v[i]);
            sum = v[i];
            cnt = 1;
        }
    }
}

// Validate a blob, allocate pool space for it and copy its device image
// (node layout, leaves, colour array or blocks) through the staging memory
// `sg` on its stream, waiting for the copies.  Nothing is published: *a and
// *ref describe the staged (chunk, lod) for the caller to install in the
// descriptor table.  When the pools are full and evict_old_first is set, the
// previous upload of descriptor di is evicted first (after the device is
// idle).  The pools are touched under *pool_mu, or under the caller's hold of
// sc->mu when pool_mu is null.
int aok::stage_chunk(aok_ctx* ctx, Scene* sc, int64_t di, uint32_t lod, const aok_chunk_blob* blob,
                     bool evict_old_first, Staging* sg, std::mutex* pool_mu, ChunkAlloc* out_a, ChunkRef* out_ref) {
    const int M = sc->desc.chunk_res, res = M >> lod;
    // 1. validate before touching anything: a rejected blob changes nothing
    int st = validate_blob(blob, res, M);
    if (st) return st;
    uint32_t droot = 0;
    const uint64_t nw = layout_blob(blob, res, 0, 0, nullptr, &droot);  // device words (even)
    // material storage: colour blocks when the scene asks for them and they are
    // smaller than the raw array (3 bytes of slack align the uint32 indices)
    std::vector<uint32_t> bfirst;
    std::vector<uint8_t> bcol, decoded;
    uint64_t mat_n = blob->n_mats;
    const uint8_t* raw_mats = blob->mats;
    if (sc->color_tol >= 0.0 && blob->n_mats) {
        color_blocks(blob->mats, blob->n_mats, sc->color_tol, bfirst, bcol);
        const uint64_t cb = 4ull * (1 + (blob->n_mats + 127) / 128) + 5ull * bfirst.size() + 3;
        if (cb < blob->n_mats) {
            mat_n = cb;
        } else {
            // not smaller: one byte per entry, holding the colour its block gives
            decoded.resize(blob->n_mats);
            for (size_t b = 0; b < bfirst.size(); b++) {
                const uint64_t end = b + 1 < bfirst.size() ? bfirst[b + 1] : blob->n_mats;
                std::memset(decoded.data() + bfirst[b], bcol[b], end - bfirst[b]);
            }
            raw_mats = decoded.data();
            bfirst.clear();
        }
    }
    // staging: laid-out node words + leaves + mats, 16-byte aligned segments
    const size_t nb = (nw * 4 + 15) & ~(size_t)15, lb = (blob->n_leaves * 8 + 15) & ~(size_t)15;
    const size_t need = nb + lb + mat_n + 16;
    if (need > sg->cap) {
        if (sg->buf) cudaFreeHost(sg->buf);
        sg->buf = nullptr;
        sg->cap = 0;
        size_t cap = std::max<size_t>(need, sg->min_cap);
        if (cudaMallocHost(&sg->buf, cap) != cudaSuccess) {
            cudaGetLastError();
            return AOK_E_OOM;
        }
        sg->cap = cap;
    }
    uint8_t* stg = (uint8_t*)sg->buf;
    // 2. allocate; if the pools are too full, evict the previous upload of this
    //    (chunk, lod) first (after the GPU is idle) and retry
    auto evict_old = [&]() {
        ChunkAlloc& old = sc->alloc[di];
        if (!(old.node_n || old.leaf_n || old.mat_n)) return;
        cudaDeviceSynchronize();
        free_alloc(sc, old);
        ChunkRef none;
        std::memset(&none, 0, sizeof(none));
        none.root = kNone;
        none.lod = lod;
        sc->h_desc[di] = none;
        cudaMemcpy(sc->d_desc + di, &none, sizeof(none), cudaMemcpyHostToDevice);
    };
    auto try_alloc = [&](ChunkAlloc& a) -> bool {
        a = ChunkAlloc();
        if (!nw) return true;
        a.node_off = sc->nodes.alloc(nw);
        a.leaf_off = sc->leaves.alloc(blob->n_leaves);
        a.mat_off = sc->mats.alloc(mat_n);
        a.node_n = nw;
        a.leaf_n = blob->n_leaves;
        a.mat_n = mat_n;
        if (a.node_off == kNoRange || a.leaf_off == kNoRange || a.mat_off == kNoRange ||
            a.node_off + nw > 0xFFFFFFFFull || a.leaf_off + blob->n_leaves > 0xFFFFFFFFull) {
            if (a.node_off != kNoRange) sc->nodes.release(a.node_off, nw);
            if (a.leaf_off != kNoRange) sc->leaves.release(a.leaf_off, blob->n_leaves);
            if (a.mat_off != kNoRange) sc->mats.release(a.mat_off, mat_n);
            a = ChunkAlloc();
            return false;
        }
        return true;
    };
    ChunkAlloc a;
    {
        std::unique_lock<std::mutex> pl;
        if (pool_mu) pl = std::unique_lock<std::mutex>(*pool_mu);
        if (!try_alloc(a)) {
            if (!evict_old_first) return AOK_E_OOM;
            evict_old();
            if (!try_alloc(a)) return AOK_E_OOM;
        }
    }
    // 3. lay the (valid) blob out at its pool offsets and copy it
    layout_blob(blob, res, (uint32_t)a.node_off, (uint32_t)a.leaf_off, (uint32_t*)stg, &droot);
    ChunkRef ref;
    std::memset(&ref, 0, sizeof(ref));
    ref.root = kNone;
    ref.lod = lod | kResidentBit;  // an uploaded, empty DAG until the root is set below
    uint64_t mat_base = a.mat_off;
    if (nw) {
        std::memcpy(stg + nb, blob->leaves, blob->n_leaves * 8);
        if (bfirst.empty()) {
            std::memcpy(stg + nb + lb, raw_mats, blob->n_mats);
        } else {
            // [pad to 4][nt][nt x uint32: block holding entry 128 j]
            // [nblocks x uint32 first index][nblocks x uint8 colour]
            mat_base = (a.mat_off + 3) & ~(uint64_t)3;
            const size_t nt = (blob->n_mats + 127) / 128;
            std::vector<uint32_t> head(1 + nt);
            head[0] = (uint32_t)nt;
            for (size_t j = 0, b = 0; j < nt; j++) {
                while (b + 1 < bfirst.size() && bfirst[b + 1] <= 128 * j) b++;
                head[1 + j] = (uint32_t)b;
            }
            uint8_t* seg = stg + nb + lb;
            std::memset(seg, 0, mat_n);
            uint8_t* q = seg + (mat_base - a.mat_off);
            std::memcpy(q, head.data(), head.size() * 4);
            std::memcpy(q + head.size() * 4, bfirst.data(), bfirst.size() * 4);
            std::memcpy(q + head.size() * 4 + bfirst.size() * 4, bcol.data(), bcol.size());
        }
        cudaError_t e = cudaMemcpyAsync(sc->d_nodes + a.node_off, stg, nw * 4, cudaMemcpyHostToDevice, sg->stream);
        if (e == cudaSuccess && blob->n_leaves)
            e = cudaMemcpyAsync(sc->d_leaves + a.leaf_off, stg + nb, blob->n_leaves * 8, cudaMemcpyHostToDevice,
                                sg->stream);
        if (e == cudaSuccess && mat_n)
            e = cudaMemcpyAsync(sc->d_mats + a.mat_off, stg + nb + lb, mat_n, cudaMemcpyHostToDevice, sg->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sg->stream);
        if (e != cudaSuccess) {
            std::unique_lock<std::mutex> pl;
            if (pool_mu) pl = std::unique_lock<std::mutex>(*pool_mu);
            free_alloc(sc, a);
            return cuda_status(ctx, e);
        }
        ref.root = droot;
        ref.lod = lod;
        ref.mat_base = mat_base;
        ref.nblocks = (uint32_t)bfirst.size();
        for (int i = 0; i < 3; i++) {
            ref.aabb[i] = (uint16_t)blob->aabb_lo[i];
            ref.aabb[3 + i] = (uint16_t)blob->aabb_hi[i];
        }
    }
    *out_a = a;
    *out_ref = ref;
    return AOK_OK;
}

extern "C" {

int aok_scene_upload_chunk(aok_ctx* ctx, uint32_t scene, int32_t cx, int32_t cy, int32_t cz, uint32_t lod,
                           const aok_chunk_blob* blob) {
    if (!ctx || !blob) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    int64_t di;
    int st = chunk_index(sc, cx, cy, cz, lod, &di);
    if (st) return st;
    cudaSetDevice(ctx->device);
    std::lock_guard<std::mutex> g(sc->mu);
    ChunkAlloc a;
    ChunkRef ref;
    {
        std::lock_guard<std::mutex> up(ctx->upload_mu);
        Staging sg{ctx->staging, ctx->staging_cap, ctx->copy_stream};
        st = stage_chunk(ctx, sc, di, lod, blob, true, &sg, nullptr, &a, &ref);
        ctx->staging = sg.buf;
        ctx->staging_cap = sg.cap;
    }
    if (st) return st;
    ChunkAlloc& old = sc->alloc[di];
    if (old.node_n || old.leaf_n || old.mat_n) {
        cudaDeviceSynchronize();
        free_alloc(sc, old);
    }
    sc->alloc[di] = a;
    sc->h_desc[di] = ref;
    cudaError_t e = cudaMemcpy(sc->d_desc + di, &ref, sizeof(ref), cudaMemcpyHostToDevice);
    return cuda_status(ctx, e);
}

int aok_scene_set_color_blocks(aok_ctx* ctx, uint32_t scene, double e_c) {
    if (!ctx || !(e_c == e_c) || e_c > 1.0) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    std::lock_guard<std::mutex> g(sc->mu);
    sc->color_tol = e_c < 0.0 ? -1.0 : e_c;
    return AOK_OK;
}

int aok_scene_usage(aok_ctx* ctx, uint32_t scene, uint64_t* usage) {
    if (!ctx || !usage) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    std::lock_guard<std::mutex> g(sc->mu);
    uint64_t u[4] = {0, 0, 0, 0};
    for (const ChunkAlloc& a : sc->alloc) {
        u[0] += a.node_n;
        u[1] += a.leaf_n;
        u[2] += a.mat_n;
        u[3] += (a.node_n || a.leaf_n || a.mat_n) ? 1 : 0;
    }
    u[0] *= 4;
    u[1] *= 8;
    std::memcpy(usage, u, sizeof(u));
    return AOK_OK;
}

int aok_validate_chunk(const aok_chunk_blob* blob, int32_t M, uint32_t lod) {
    if (!blob || M < 8 || M > 512 || (M & (M - 1)) || lod > 6 || (M >> lod) < 8) return AOK_E_INVALID;
    if (blob->n_node_words > (1ull << 32)) return AOK_E_CORRUPT;
    return validate_blob(blob, M >> lod, M);
}

int aok_scene_evict_chunk(aok_ctx* ctx, uint32_t scene, int32_t cx, int32_t cy, int32_t cz, uint32_t lod) {
    if (!ctx) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    int64_t di;
    int st = chunk_index(sc, cx, cy, cz, lod, &di);
    if (st) return st;
    cudaSetDevice(ctx->device);
    std::lock_guard<std::mutex> g(sc->mu);
    ChunkRef ref;
    std::memset(&ref, 0, sizeof(ref));
    ref.root = kNone;
    ref.lod = lod;
    cudaDeviceSynchronize();
    free_alloc(sc, sc->alloc[di]);
    sc->h_desc[di] = ref;
    return cuda_status(ctx, cudaMemcpy(sc->d_desc + di, &ref, sizeof(ref), cudaMemcpyHostToDevice));
}

int aok_select_chunks(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double tau, int8_t* lod_out,
                      uint8_t* vis_out, uint32_t* n_visible_out, void* stream) {
    if (!ctx) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    CamDev cd;
    int st = make_cam(ctx, sc, cam, tau, &cd);
    if (st) return st;
    cudaSetDevice(ctx->device);
    SceneDev sd = scene_dev(sc);
    cudaStream_t s = (cudaStream_t)stream;
    if (n_visible_out) {
        st = cuda_status(ctx, cudaMemsetAsync(ctx->d_counter, 0, sizeof(uint32_t), s));
        if (st) return st;
    }
    sc->select_gen++;
    st = aokk_select(&sd, &cd, sc->d_frame, lod_out, vis_out, n_visible_out ? ctx->d_counter : nullptr, stream);
    if (st) return launch_failure(ctx);
    if (n_visible_out) {
        cudaError_t e = cudaMemcpyAsync(ctx->pinned_word, ctx->d_counter, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(ctx, e);
        *n_visible_out = *ctx->pinned_word;
    }
    return AOK_OK;
}

// Eq. 1 on the host with the kernel's operation order (compiled without
// floating-point contraction, so the results are bit-identical).
static bool host_lod_loads(int n, const int b[3], int mlog, const float o[3], double sf) {
    const double S = (double)(1ll << (mlog + n));
    double e2 = 0.0;
    for (int a = 0; a < 3; a++) {
        const double c = (double)b[a] * S + 0.5 * S;
        const double dd = c - (double)o[a];
        e2 = e2 + dd * dd;
    }
    const double thr = S * sf;
    return e2 >= thr * thr;
}

int aok_plan_residency(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double tau, uint8_t* lod_out,
                       uint32_t* n_kept) {
    if (!ctx || !lod_out) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    CamDev cd;
    int st = make_cam(ctx, sc, cam, tau, &cd);
    if (st) return st;
    const int G0 = sc->desc.grid[0], G1 = sc->desc.grid[1], G2 = sc->desc.grid[2], M = sc->desc.chunk_res;
    const double vd = sc->desc.view_dist;
    uint32_t kept = 0;
    for (int cz = 0; cz < G2; cz++)
        for (int cy = 0; cy < G1; cy++)
            for (int cx = 0; cx < G0; cx++) {
                const size_t i = (size_t)cx + (size_t)G0 * ((size_t)cy + (size_t)G1 * cz);
                if (vd > 0) {  // distance from the camera to the region's cell
                    const int c[3] = {cx, cy, cz};
                    double d2 = 0;
                    for (int a = 0; a < 3; a++) {
                        const double lo = (double)c[a] * M, hi = lo + M, o = cd.of[a];
                        const double q = o < lo ? lo - o : (o > hi ? o - hi : 0.0);
                        d2 += q * q;
                    }
                    if (d2 > (vd + 2.0) * (vd + 2.0)) { lod_out[i] = 0xFF; continue; }
                }
                int sel = 0;
                for (int n = sc->desc.n_lods - 1; n >= 1; n--) {
                    const int b[3] = {cx >> n, cy >> n, cz >> n};
                    if (host_lod_loads(n, b, sc->mlog, cd.of, cd.sf)) { sel = n; break; }
                }
                lod_out[i] = (uint8_t)sel;
                kept++;
            }
    if (n_kept) *n_kept = kept;
    return AOK_OK;
}

// Pool sizes and the error word of a checked cast (null when checking is off).
static const CheckDev* check_dev(aok_ctx* ctx, const Scene* sc, CheckDev* ck) {
    if (!ctx->checked) return nullptr;
    ck->n_nodes = sc->nodes.cap;
    ck->n_leaves = sc->leaves.cap;
    ck->n_mats = sc->mats.cap;
    ck->err = ctx->d_counter + 8;
    return ck;
}

// ---------------------------------------------------------------------------
// beam pass
// ---------------------------------------------------------------------------
static constexpr uint32_t kBeamCap = 1u << 20;  // queued nodes per level

// The walk's queues, counters and launch grid (shared by single-view and
// batch passes, which run in stream order).
static int ensure_beam_queues(aok_ctx* ctx) {
    BeamState& b = ctx->beam;
    std::lock_guard<std::mutex> lk(b.mu);
    if (b.qblock) return AOK_OK;
    const size_t sq = (size_t)kBeamCap * 16, sc = 2 * kBeamLevels * 4;
    void* block = nullptr;
    int st = dev_alloc(ctx, &block, 2 * sq + sc);
    if (st) return st;
    b.q[0] = (uint4*)block;
    b.q[1] = (uint4*)((char*)block + sq);
    b.cnt = (uint32_t*)((char*)block + 2 * sq);
    b.hist = b.cnt + kBeamLevels;
    b.qblock = block;
    b.qbytes = 2 * sq + sc;
    b.grid = aokk_beam_grid(ctx->sm_count);
    if (!b.grid) return AOK_E_CUDA;
    if (!b.P) b.P.reset(new BeamBatch);
    return AOK_OK;
}

// A grow-only array of bound entries, all without a pass tag when allocated
// (entries carry their pass's tag, so a change of layout needs no clearing).
static int ensure_bounds(aok_ctx* ctx, unsigned long long** buf, size_t* cap, size_t need) {
    if (need <= *cap) return AOK_OK;
    if (*buf) {
        cudaDeviceSynchronize();
        dev_free(ctx, *buf, *cap * 8);
        *buf = nullptr;
        *cap = 0;
    }
    int st = dev_alloc(ctx, (void**)buf, need * 8);
    if (st) return st;
    if (cudaMemset(*buf, 0xFF, need * 8) != cudaSuccess) return cuda_status(ctx, cudaGetLastError());
    *cap = need;
    return AOK_OK;
}

// The next pass's tag (tags count down); before they wrap every bound array
// is cleared.
static int next_beam_tag(aok_ctx* ctx, void* stream, uint32_t* tag) {
    BeamState& b = ctx->beam;
    std::lock_guard<std::mutex> lk(b.mu);
    if (++b.passes >= 0xFFFFFFF0u) {
        const cudaStream_t s = (cudaStream_t)stream;
        if ((b.bounds && cudaMemsetAsync(b.bounds, 0xFF, b.bounds_cap * 8, s) != cudaSuccess) ||
            (ctx->batch.beam_bounds &&
             cudaMemsetAsync(ctx->batch.beam_bounds, 0xFF, ctx->batch.beam_cap * 8, s) != cudaSuccess))
            return AOK_E_CUDA;
        b.passes = 1;
        b.valid = false;
    }
    *tag = 0xFFFFFFFFu - b.passes;
    return AOK_OK;
}

// Fill the pass header of P (views and regions are filled by the caller).
static void beam_header(aok_ctx* ctx, BeamBatch* P, uint32_t tag) {
    P->expand = ctx->beam_refine;
    P->smin = ctx->beam_min_log2;
    P->tag = tag;
    P->cap = ctx->beam_queue && ctx->beam_queue < kBeamCap ? ctx->beam_queue : kBeamCap;
    P->q[0] = ctx->beam.q[0];
    P->q[1] = ctx->beam.q[1];
    P->cnt = ctx->beam.cnt;
    P->hist = ctx->beam.hist;
    P->select = 0;
    std::memset(&P->ck, 0, sizeof(P->ck));  // unchecked
}

// The beam pass over the scene's current frame table, remembered with what
// it was computed for.  select: the frame table is not selected yet; the
// pass selects it as its first step (one launch fewer), or, for a view
// without a usable projection, the selection kernel does.  ck: checked
// casting's pool sizes and error word (the pass tests its node and leaf
// indices too), or null.
static int run_beam(aok_ctx* ctx, uint32_t scene, Scene* sc, const SceneDev& sd, const CamDev& cd, void* stream,
                    bool select = false, const CheckDev* ck = nullptr) {
    int st = ensure_beam_queues(ctx);
    if (st) return st;
    BeamState& b = ctx->beam;
    st = ensure_bounds(ctx, &b.bounds, &b.bounds_cap, beam_entries((uint32_t)cd.W, (uint32_t)cd.H));
    if (st) return st;
    b.valid = false;
    uint32_t tag;
    st = next_beam_tag(ctx, stream, &tag);
    if (st) return st;
    BeamBatch* P = b.P.get();
    beam_header(ctx, P, tag);
    if (ck) P->ck = *ck;
    P->n_views = 0;
    P->n_regions = 0;
    b.read.bounds = nullptr;  // no usable projection: no bounds, nothing is skipped
    b.read.tag = tag;
    if (aokk_beam_view(&sd, &cd, sc->d_frame, b.bounds, &P->v[0])) {
        P->v[0].region_begin = 0;
        P->n_views = 1;
        P->n_regions = (uint32_t)sc->n_chunks;
        b.read.bounds = b.bounds;
        if (select) {
            P->select = 1;
            P->cam = cd;
        }
    } else if (select) {
        st = aokk_select(&sd, &cd, sc->d_frame, nullptr, nullptr, nullptr, stream);
        if (st) return st;
    }
    st = aokk_beam_run(P, b.grid, stream);
    if (st) return st;
    b.valid = true;
    b.scene = scene;
    b.gen = sc->select_gen;
    b.cam = cd;
    b.cam.sf = 0.0;  // the LOD threshold does not enter the bounds
    b.W = cd.W;
    b.H = cd.H;
    return AOK_OK;
}

extern "C++" bool aok::beam_wanted(const aok_ctx* ctx, int32_t W, int32_t H) {
    return ctx->beam_on && (uint64_t)W * (uint64_t)H >= ctx->beam_min_pixels;
}

extern "C++" int aok::beam_for_batch(aok_ctx* ctx, BatchParams* groups, uint32_t ngroups,
                                     std::vector<BeamBatch>& out, void* stream,
                                     unsigned long long* const* view_bounds) {
    out.clear();
    if (!ctx->beam_on) return AOK_OK;
    size_t need = 0, n_big = 0;
    for (uint32_t g = 0; g < ngroups; g++)
        for (uint32_t i = 0; i < groups[g].n_views; i++) {
            const CamDev& c = groups[g].v[i].cam;
            if (beam_wanted(ctx, c.W, c.H)) {
                need += beam_entries((uint32_t)c.W, (uint32_t)c.H);
                n_big++;
            }
        }
    if (!n_big) return AOK_OK;
    int st = ensure_beam_queues(ctx);
    if (!st && !view_bounds) st = ensure_bounds(ctx, &ctx->batch.beam_bounds, &ctx->batch.beam_cap, need);
    uint32_t tag = 0;
    if (!st) st = next_beam_tag(ctx, stream, &tag);
    if (st) return st;
    out.resize(ngroups);
    size_t off = 0, flat = 0;
    for (uint32_t g = 0; g < ngroups; g++) {
        BeamBatch& B = out[g];
        beam_header(ctx, &B, tag);
        B.n_views = 0;
        B.n_regions = 0;
        groups[g].beam_tag = tag;
        for (uint32_t i = 0; i < groups[g].n_views; i++, flat++) {
            ViewDev& d = groups[g].v[i];
            d.beam = nullptr;
            if (!beam_wanted(ctx, d.cam.W, d.cam.H)) continue;
            unsigned long long* bnd = view_bounds ? view_bounds[flat] : ctx->batch.beam_bounds + off;
            off += beam_entries((uint32_t)d.cam.W, (uint32_t)d.cam.H);
            if (!bnd) continue;
            if (!aokk_beam_view(&d.scene, &d.cam, d.frame, bnd, &B.v[B.n_views])) continue;  // casts without
            B.v[B.n_views].region_begin = B.n_regions;
            B.n_regions += (uint32_t)(d.scene.grid[0] * d.scene.grid[1] * d.scene.grid[2]);
            B.n_views++;
            d.beam = bnd;
        }
    }
    return AOK_OK;
}

static bool beam_fresh(const aok_ctx* ctx, uint32_t scene, const Scene* sc, const CamDev& cd) {
    const BeamState& b = ctx->beam;
    if (!b.valid || b.scene != scene || b.gen != sc->select_gen) return false;
    CamDev k = cd;
    k.sf = 0.0;
    return std::memcmp(&k, &b.cam, sizeof(CamDev)) == 0;
}

// The casting launch of a single view: with the beam pass on the casting
// kernel takes the pass's per-tile bounds, computed first unless
// aok_beam_selected already did for this selection and camera (with checked
// casting the pass tests its node and leaf indices as well).
// selected: the frame table is already selected; else the beam pass selects
// it (or, without the pass, the selection kernel).
static int cast_single(aok_ctx* ctx, uint32_t scene, Scene* sc, const SceneDev& sd, const CamDev& cd,
                       const aok_frame* frame, uint32_t* counts, void* stream, bool selected = true) {
    CheckDev ck;
    const CheckDev* ckp = check_dev(ctx, sc, &ck);
    const BeamRead* beam = nullptr;
    int st = AOK_OK;
    if (ctx->beam_on && (uint64_t)cd.W * (uint64_t)cd.H >= ctx->beam_min_pixels) {
        if (!selected || !beam_fresh(ctx, scene, sc, cd)) {
            st = run_beam(ctx, scene, sc, sd, cd, stream, !selected, ckp);
            if (st) return st;
            selected = true;
        }
        beam = &ctx->beam.read;
    }
    if (!selected) st = aokk_select(&sd, &cd, sc->d_frame, nullptr, nullptr, nullptr, stream);
    if (st) return st;
    return aokk_cast(&sd, &cd, sc->d_frame, (uint4*)frame->hit, frame->t, counts, stream, ckp, beam);
}

static int render_impl(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double tau, const aok_frame* frame,
                       uint32_t* counts, void* stream) {
    if (!ctx || !frame || !frame->hit || !frame->t) return AOK_E_INVALID;
    if (((uintptr_t)frame->hit & 15) || ((uintptr_t)frame->t & 3) || ((uintptr_t)counts & 3)) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    CamDev cd;
    int st = make_cam(ctx, sc, cam, tau, &cd);
    if (st) return st;
    cudaSetDevice(ctx->device);
    SceneDev sd = scene_dev(sc);
    sc->select_gen++;
    if (ctx->single_persistent && !counts) {
        st = render_persistent(ctx, sc, cd, frame, stream, true);
    } else {
        st = cast_single(ctx, scene, sc, sd, cd, frame, counts, stream, false);
    }
    if (st == AOK_E_CUDA) return launch_failure(ctx);
    return st;
}

int aok_render(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double tau, const aok_frame* frame, void* stream) {
    return render_impl(ctx, scene, cam, tau, frame, nullptr, stream);
}

int aok_render_noalloc(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double tau, const aok_frame* frame,
                       void* stream) {
    if (!ctx || !frame || !frame->hit || !frame->t) return AOK_E_INVALID;
    if (((uintptr_t)frame->hit & 15) || ((uintptr_t)frame->t & 3)) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    if (sc->n_chunks > AOK_NOALLOC_MAX_CHUNKS) return AOK_E_INVALID;
    CamDev cd;
    int st = make_cam(ctx, sc, cam, tau, &cd);
    if (st) return st;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_status(ctx, cudaGetLastError());
    SceneDev sd = scene_dev(sc);
    CheckDev ck;
    st = aokk_render_noalloc(&sd, &cd, (uint4*)frame->hit, frame->t, stream, check_dev(ctx, sc, &ck));
    if (st == AOK_E_CUDA) return launch_failure(ctx);
    return st;
}

int aok_render_counted(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double tau, const aok_frame* frame,
                       uint32_t* counts, void* stream) {
    if (!counts) return AOK_E_INVALID;
    return render_impl(ctx, scene, cam, tau, frame, counts, stream);
}

int aok_cast_selected(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, const aok_frame* frame, void* stream) {
    if (!ctx || !frame || !frame->hit || !frame->t) return AOK_E_INVALID;
    if (((uintptr_t)frame->hit & 15) || ((uintptr_t)frame->t & 3)) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    CamDev cd;
    int st = make_cam(ctx, sc, cam, 1.0, &cd);
    if (st) return st;
    cudaSetDevice(ctx->device);
    SceneDev sd = scene_dev(sc);
    if (ctx->single_persistent) st = render_persistent(ctx, sc, cd, frame, stream, false);
    else st = cast_single(ctx, scene, sc, sd, cd, frame, nullptr, stream);
    return st == AOK_E_CUDA ? launch_failure(ctx) : st;
}

// ---------------------------------------------------------------------------
// tile-chunk pipeline (Sec. 3.5)
// ---------------------------------------------------------------------------
static constexpr uint32_t kFarBits = 0x7F7F7F7Fu;  // 3.4e38 as float: "no Hi-Z history"

// (Re)allocate the pipeline's buffers for W x H and n_chunks regions; a new
// scene or size starts without Hi-Z history.
static int ensure_tiles(aok_ctx* ctx, uint32_t scene, int32_t W, int32_t H, int64_t nch, cudaStream_t s) {
    TileState& ts = ctx->tiles;
    if (ts.block && ts.W == W && ts.H == H && ts.n_chunks == nch) {
        if (ts.scene != scene) {
            const size_t tiles = (size_t)ts.dev.tiles_x * ts.dev.tiles_y;
            if (cudaMemsetAsync(ts.dev.hiz_prev, 0x7F, tiles * sizeof(float), s) != cudaSuccess)
                return cuda_status(ctx, cudaGetLastError());
            ts.scene = scene;
        }
        return AOK_OK;
    }
    if (ts.block) {
        cudaDeviceSynchronize();
        dev_free(ctx, ts.block, ts.bytes);
        ts = TileState{};
    }
    const int32_t tx = (W + 7) / 8, ty = (H + 7) / 8;
    const size_t tiles = (size_t)tx * ty, px = (size_t)W * H, n = (size_t)nch;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t sz[] = {px * 16, tiles * 4, tiles * 4, tiles * 4, n * 16, n * 4, n * 4, n * 4, (n + 1) * 8,
                         kTileStats * 8, n * 4};
    constexpr int kParts = (int)(sizeof(sz) / sizeof(sz[0]));
    size_t total = 0;
    for (size_t b : sz) total += al(b);
    void* block = nullptr;
    int st = dev_alloc(ctx, &block, total);
    if (st) return st;
    char* p = (char*)block;
    char* q[kParts];
    for (int i = 0; i < kParts; i++) { q[i] = p; p += al(sz[i]); }
    TileDev& d = ts.dev;
    d.vis = (unsigned long long*)q[0];
    d.hiz_prev = (float*)q[1];
    d.hiz = (float*)q[2];
    d.hiz_next = (float*)q[3];
    d.rect = (int4*)q[4];
    d.dmin = (float*)q[5];
    d.area = (uint32_t*)q[6];
    d.list = (uint32_t*)q[7];
    d.offs = (unsigned long long*)q[8];
    d.stats = (unsigned long long*)q[9];
    d.dfar = (int32_t*)q[10];
    d.tiles_x = tx;
    d.tiles_y = ty;
    cudaError_t e = cudaMemsetAsync(d.vis, 0xFF, px * 16, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.hiz_prev, 0x7F, tiles * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.stats, 0, kTileStats * 8, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        dev_free(ctx, block, total);
        ts = TileState{};
        return cuda_status(ctx, e);
    }
    ts.block = block;
    ts.bytes = total;
    ts.W = W;
    ts.H = H;
    ts.n_chunks = nch;
    ts.scene = scene;
    return AOK_OK;
}

int aok_render_tiles(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double tau, const aok_frame* frame,
                     void* stream) {
    if (!ctx || !frame || !frame->hit || !frame->t) return AOK_E_INVALID;
    if (((uintptr_t)frame->hit & 15) || ((uintptr_t)frame->t & 3)) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    if (sc->n_chunks > AOK_TILES_MAX_CHUNKS) return AOK_E_INVALID;
    CamDev cd;
    int st = make_cam(ctx, sc, cam, tau, &cd);
    if (st) return st;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_status(ctx, cudaGetLastError());
    st = ensure_tiles(ctx, scene, cd.W, cd.H, sc->n_chunks, (cudaStream_t)stream);
    if (st) return st;
    SceneDev sd = scene_dev(sc);
    sc->select_gen++;
    st = aokk_select(&sd, &cd, sc->d_frame, nullptr, nullptr, nullptr, stream);
    // the beam pass's bounds cull the pairs in front of every voxel a tile's
    // rays can meet and restart the rays of the others (as in the march)
    const BeamRead* beam = nullptr;
    if (!st && beam_wanted(ctx, cd.W, cd.H)) {
        st = run_beam(ctx, scene, sc, sd, cd, stream);
        beam = &ctx->beam.read;
    }
    if (!st) st = aokk_tiles_frame(&sd, &cd, sc->d_frame, &ctx->tiles.dev, (uint4*)frame->hit, frame->t,
                                   ctx->sm_count, stream, beam);
    if (st) return st == AOK_E_CUDA ? launch_failure(ctx) : st;
    std::swap(ctx->tiles.dev.hiz_prev, ctx->tiles.dev.hiz_next);  // this frame's depth culls the next one
    return AOK_OK;
}

int aok_tiles_stats(aok_ctx* ctx, uint64_t* stats) {
    if (!ctx || !stats) return AOK_E_INVALID;
    if (!ctx->tiles.block) return AOK_E_INVALID;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(stats, ctx->tiles.dev.stats, kTileStats * 8, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? AOK_OK : cuda_status(ctx, e);
}

int aok_tiles_forget(aok_ctx* ctx) {
    if (!ctx) return AOK_E_INVALID;
    ctx->tiles.scene = 0xFFFFFFFFu;
    return AOK_OK;
}

int aok_set_beam(aok_ctx* ctx, int on) {
    if (!ctx) return AOK_E_INVALID;
    ctx->beam_on = on ? 1 : 0;
    return AOK_OK;
}

int aok_beam_tune(aok_ctx* ctx, uint32_t refine_tiles, int32_t min_node_log2, uint64_t min_pixels,
                  uint32_t queue_nodes) {
    if (!ctx || min_node_log2 < 2 || min_node_log2 > 16) return AOK_E_INVALID;
    ctx->beam_refine = refine_tiles;
    ctx->beam_min_log2 = min_node_log2;
    ctx->beam_min_pixels = min_pixels;
    ctx->beam_queue = queue_nodes;
    return AOK_OK;
}

int aok_beam_selected(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, void* stream) {
    if (!ctx) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    CamDev cd;
    int st = make_cam(ctx, sc, cam, 1.0, &cd);
    if (st) return st;
    cudaSetDevice(ctx->device);
    SceneDev sd = scene_dev(sc);
    st = run_beam(ctx, scene, sc, sd, cd, stream);
    if (st == AOK_E_CUDA) return launch_failure(ctx);
    return st;
}

int aok_select_beam(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double tau, void* stream) {
    if (!ctx) return AOK_E_INVALID;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    CamDev cd;
    int st = make_cam(ctx, sc, cam, tau, &cd);
    if (st) return st;
    cudaSetDevice(ctx->device);
    SceneDev sd = scene_dev(sc);
    sc->select_gen++;
    CheckDev ck;
    if (ctx->beam_on && (uint64_t)cd.W * (uint64_t)cd.H >= ctx->beam_min_pixels)
        st = run_beam(ctx, scene, sc, sd, cd, stream, true, check_dev(ctx, sc, &ck));
    else
        st = aokk_select(&sd, &cd, sc->d_frame, nullptr, nullptr, nullptr, stream);
    if (st == AOK_E_CUDA) return launch_failure(ctx);
    return st;
}

int aok_beam_info(aok_ctx* ctx, int32_t* bounds, uint64_t n_bounds, uint32_t* level_counts, int32_t* tiles_xy) {
    if (!ctx) return AOK_E_INVALID;
    const BeamState& b = ctx->beam;
    if (!b.valid) return AOK_E_INVALID;
    const uint32_t tx = (uint32_t)(b.W + kBeamTileW - 1) / kBeamTileW, ty = (uint32_t)(b.H + kBeamTileH - 1) / kBeamTileH;
    const uint64_t n = (uint64_t)tx * ty;
    if (bounds && n_bounds < n) return AOK_E_INVALID;
    cudaSetDevice(ctx->device);
    if (cudaDeviceSynchronize() != cudaSuccess) return cuda_status(ctx, cudaGetLastError());
    if (bounds) {
        // the bounds the casting kernel uses: each tile's minimum over its
        // cells of the pyramid among entries of the last pass's tag, or 0
        // everywhere if that pass could not project
        std::vector<unsigned long long> e(beam_entries((uint32_t)b.W, (uint32_t)b.H));
        if (b.read.bounds &&
            cudaMemcpy(e.data(), b.read.bounds, e.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return cuda_status(ctx, cudaGetLastError());
        const unsigned long long tag = (unsigned long long)b.read.tag << 32;
        for (uint32_t y = 0; y < ty; y++)
            for (uint32_t x = 0; x < tx; x++) {
                unsigned long long v = ~0ull;
                for (int L = 0; L < kBeamPyr; L++) {
                    const uint32_t wl = (tx + (1u << L) - 1) >> L;
                    v = std::min(v, e[beam_level_offset(tx, ty, L) + (size_t)(y >> L) * wl + (x >> L)]);
                }
                bounds[(size_t)y * tx + x] =
                    !b.read.bounds ? 0 : ((v & 0xFFFFFFFF00000000ull) == tag ? (int32_t)(uint32_t)v : INT32_MAX);
            }
    }
    if (level_counts && cudaMemcpy(level_counts, b.hist, kBeamLevels * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_status(ctx, cudaGetLastError());
    if (tiles_xy) {
        tiles_xy[0] = (int32_t)tx;
        tiles_xy[1] = (int32_t)ty;
    }
    return AOK_OK;
}

int aok_set_checked(aok_ctx* ctx, int on) {
    if (!ctx || on < 0 || on > 1) return AOK_E_INVALID;
    ctx->checked = on;
    return AOK_OK;
}

int aok_checked_errors(aok_ctx* ctx, uint32_t* errors) {
    if (!ctx || !errors) return AOK_E_INVALID;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(errors, ctx->d_counter + 8, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_counter + 8, 0, sizeof(uint32_t));
    return e == cudaSuccess ? AOK_OK : cuda_status(ctx, e);
}

int aok_set_single_view_kernel(aok_ctx* ctx, int persistent) {
    if (!ctx || persistent < 0 || persistent > 1) return AOK_E_INVALID;
    ctx->single_persistent = persistent;
    return AOK_OK;
}

int aok_render_host(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double tau, void* hit_host, float* t_host,
                    void* stream) {
    if (!ctx || !cam || !hit_host || !t_host || cam->width <= 0 || cam->height <= 0) return AOK_E_INVALID;
    const size_t px = (size_t)cam->width * cam->height;
    cudaSetDevice(ctx->device);
    if (px > ctx->host_frame_px) {
        cudaDeviceSynchronize();
        dev_free(ctx, ctx->host_hit_dev, ctx->host_frame_px * 16);
        dev_free(ctx, ctx->host_t_dev, ctx->host_frame_px * 4);
        ctx->host_hit_dev = nullptr;
        ctx->host_t_dev = nullptr;
        ctx->host_frame_px = 0;
        int st = dev_alloc(ctx, &ctx->host_hit_dev, px * 16);
        if (!st) st = dev_alloc(ctx, (void**)&ctx->host_t_dev, px * 4);
        if (st) {
            dev_free(ctx, ctx->host_hit_dev, px * 16);
            ctx->host_hit_dev = nullptr;
            return st;
        }
        ctx->host_frame_px = px;
    }
    aok_frame f{ctx->host_hit_dev, ctx->host_t_dev};
    int st = aok_render(ctx, scene, cam, tau, &f, stream);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(hit_host, ctx->host_hit_dev, px * 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t_host, ctx->host_t_dev, px * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_status(ctx, e);
}

// ---------------------------------------------------------------------------
// pipelined rendering into host memory
// ---------------------------------------------------------------------------
extern "C++" {
static void pipe_release(aok_ctx* ctx) {
    HostPipe& p = ctx->pipe;
    for (HostSlot& sl : p.slot) {
        if (sl.copied) cudaEventSynchronize(sl.copied);
        dev_free(ctx, sl.hit, p.px * 16);
        dev_free(ctx, sl.t, p.px * 4);
        dev_free(ctx, sl.frame, sl.frame_cap * sizeof(ChunkRef));
        dev_free(ctx, sl.bounds, sl.bounds_cap * 8);
        if (sl.prepped) cudaEventDestroy(sl.prepped);
        if (sl.rendered) cudaEventDestroy(sl.rendered);
        if (sl.copied) cudaEventDestroy(sl.copied);
        sl = HostSlot();
    }
    p.px = 0;
}

static int pipe_ensure(aok_ctx* ctx, size_t px) {
    HostPipe& p = ctx->pipe;
    if (!p.render) {
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (cudaStreamCreateWithPriority(&p.prep, cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaStreamCreateWithFlags(&p.render, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&p.copy, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_status(ctx, cudaGetLastError());
        p.P.reset(new BeamBatch);
    }
    if (px <= p.px) return AOK_OK;
    pipe_release(ctx);
    for (HostSlot& sl : p.slot) {
        int st = dev_alloc(ctx, &sl.hit, px * 16);
        if (!st) st = dev_alloc(ctx, (void**)&sl.t, px * 4);
        if (!st && (cudaEventCreateWithFlags(&sl.prepped, cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventCreateWithFlags(&sl.rendered, cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming) != cudaSuccess))
            st = cuda_status(ctx, cudaGetLastError());
        if (st) {
            p.px = px;
            pipe_release(ctx);
            return st;
        }
    }
    p.px = px;
    return AOK_OK;
}

// A slot's frame: selection into the slot's chunk table and the beam pass
// into its pyramid on the prep stream, then the cast on the render stream.
static int pipe_render(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double tau, HostSlot& sl) {
    HostPipe& p = ctx->pipe;
    Scene* sc = find_scene(ctx, scene);
    if (!sc) return AOK_E_NOT_RESIDENT;
    CamDev cd;
    int st = make_cam(ctx, sc, cam, tau, &cd);
    if (st) return st;
    if ((size_t)sc->n_chunks > sl.frame_cap) {
        dev_free(ctx, sl.frame, sl.frame_cap * sizeof(ChunkRef));
        sl.frame = nullptr;
        sl.frame_cap = 0;
        st = dev_alloc(ctx, (void**)&sl.frame, (size_t)sc->n_chunks * sizeof(ChunkRef));
        if (st) return st;
        sl.frame_cap = (size_t)sc->n_chunks;
    }
    const bool beam = beam_wanted(ctx, cd.W, cd.H);
    if (beam) {
        st = ensure_beam_queues(ctx);
        if (!st) st = ensure_bounds(ctx, &sl.bounds, &sl.bounds_cap, beam_entries((uint32_t)cd.W, (uint32_t)cd.H));
        if (st) return st;
    }
    const SceneDev sd = scene_dev(sc);
    // the selection kernel, then the pass (measured faster here than the pass
    // that selects first: the pass runs beside the previous frame's cast)
    st = aokk_select(&sd, &cd, sl.frame, nullptr, nullptr, nullptr, p.prep);
    if (st) return launch_failure(ctx);
    BeamRead rd{nullptr, 0};
    if (beam) {
        uint32_t tag;
        st = next_beam_tag(ctx, p.prep, &tag);
        if (st) return st;
        BeamBatch* P = p.P.get();
        beam_header(ctx, P, tag);
        P->n_views = 0;
        P->n_regions = 0;
        if (aokk_beam_view(&sd, &cd, sl.frame, sl.bounds, &P->v[0])) {
            P->v[0].region_begin = 0;
            P->n_views = 1;
            P->n_regions = (uint32_t)sc->n_chunks;
            rd.bounds = sl.bounds;
            rd.tag = tag;
        }
        st = aokk_beam_run(P, ctx->beam.grid, p.prep, 1);  // beside the previous frame's cast
        if (st) return launch_failure(ctx);
    }
    cudaError_t e = cudaEventRecord(sl.prepped, p.prep);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p.render, sl.prepped, 0);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    st = aokk_cast(&sd, &cd, sl.frame, (uint4*)sl.hit, sl.t, nullptr, p.render, nullptr, rd.bounds ? &rd : nullptr);
    return st ? launch_failure(ctx) : AOK_OK;
}
}  // extern "C++"

int aok_render_host_async(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double tau, void* hit_host,
                          float* t_host, uint64_t* ticket) {
    if (!ctx || !cam || !hit_host || !t_host || !ticket || cam->width <= 0 || cam->height <= 0) return AOK_E_INVALID;
    const size_t px = (size_t)cam->width * cam->height;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_status(ctx, cudaGetLastError());
    int st = pipe_ensure(ctx, px);
    if (st) return st;
    HostPipe& p = ctx->pipe;
    HostSlot& sl = p.slot[p.next % kHostSlots];
    // the slot's previous frame must have left the device buffers
    if (sl.ticket && cudaEventSynchronize(sl.copied) != cudaSuccess) return cuda_status(ctx, cudaGetLastError());
    if (ctx->checked || ctx->single_persistent) {
        // these modes render through the context's own path on the render stream
        aok_frame f{sl.hit, sl.t};
        st = aok_render(ctx, scene, cam, tau, &f, p.render);
    } else {
        st = pipe_render(ctx, scene, cam, tau, sl);
    }
    if (st) return st;
    cudaError_t e = cudaEventRecord(sl.rendered, p.render);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p.copy, sl.rendered, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hit_host, sl.hit, px * 16, cudaMemcpyDeviceToHost, p.copy);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t_host, sl.t, px * 4, cudaMemcpyDeviceToHost, p.copy);
    if (e == cudaSuccess) e = cudaEventRecord(sl.copied, p.copy);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    sl.ticket = ++p.next;
    *ticket = sl.ticket;
    return AOK_OK;
}

int aok_host_frame_wait(aok_ctx* ctx, uint64_t ticket) {
    if (!ctx || ticket == 0 || ticket > ctx->pipe.next) return AOK_E_INVALID;
    for (HostSlot& sl : ctx->pipe.slot)
        if (sl.ticket == ticket) return cuda_status(ctx, cudaEventSynchronize(sl.copied));
    return AOK_OK;  // its slot was reused, which waited for it
}

int aok_ray_dirs(aok_ctx* ctx, const aok_camera* cam, float* dirs, void* stream) {
    if (!ctx || !cam || !dirs || ((uintptr_t)dirs & 3)) return AOK_E_INVALID;
    CamDev cd;
    Scene dummy;
    dummy.desc.chunk_res = 512;
    int st = make_cam(ctx, &dummy, cam, 1.0, &cd);
    if (st) return st;
    cudaSetDevice(ctx->device);
    st = aokk_ray_dirs(&cd, dirs, stream);
    return st ? launch_failure(ctx) : AOK_OK;
}

int aok_read_bandwidth(aok_ctx* ctx, uint64_t bytes, int reps, double* gbs) {
    if (!ctx || !gbs || bytes < 16 || reps < 1) return AOK_E_INVALID;
    cudaSetDevice(ctx->device);
    bytes &= ~(uint64_t)15;
    void* buf = nullptr;
    int st = dev_alloc(ctx, &buf, bytes + 16);
    if (st) return st;
    uint32_t* sink = (uint32_t*)((char*)buf + bytes);
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0x5A, bytes + 16, s);
    const int sms = aokk_sm_count(ctx->device);
    // warm-up passes (below the L2 size they also make the buffer resident), then one timed launch
    if (e == cudaSuccess && aokk_read_bw(buf, bytes / 16, 2, sink, sms, s)) e = aokk_take_launch_error();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess && aokk_read_bw(buf, bytes / 16, reps, sink, sms, s)) e = aokk_take_launch_error();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    dev_free(ctx, buf, bytes + 16);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    *gbs = ms > 0.0f ? (double)bytes * reps / (ms * 1e-3) / 1e9 : 0.0;
    return AOK_OK;
}

}  // extern "C"
