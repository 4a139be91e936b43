// Offline chunk preparation (Sec. 3.1-3.4): per chunk region, LOD aggregation
// (density 2, average material) and one sparse voxel DAG per LOD with
// subtree leaf counts and a depth-first material array, in the blob format
// of aok.h.  Input voxels come from scenegen; chunks are built in parallel.
//
// Layout choices (not fixed by the paper): occupancy is bit-packed (x
// fastest); identical subtrees are merged by hash-consing per level; the
// final node pool is laid out breadth-first from the root, so a chunk's
// upper levels are contiguous, and leaves follow in first-reference order.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/aok.h"
#include "../../scenegen/scenegen.h"

namespace {

// ---- bit grid: side r, rows of w64 = ceil(r/64) words, row index y + r*z ----
struct BitGrid {
    int r = 0, w64 = 0;
    std::vector<uint64_t> w;
    void init(int side) {
        r = side;
        w64 = (side + 63) / 64;
        w.assign((size_t)w64 * side * side, 0);
    }
    inline bool get(int x, int y, int z) const {
        return (w[(size_t)(x >> 6) + (size_t)w64 * ((size_t)y + (size_t)r * z)] >> (x & 63)) & 1;
    }
    inline uint64_t row_bits(int x, int y, int z, int n) const {  // n <= 4 bits from x (x aligned to n)
        return (w[(size_t)(x >> 6) + (size_t)w64 * ((size_t)y + (size_t)r * z)] >> (x & 63)) & ((1ull << n) - 1);
    }
};

inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 33)) * 0xff51afd7ed558ccdull;
    z = (z ^ (z >> 33)) * 0xc4ceb9fe1a85ec53ull;
    return z ^ (z >> 33);
}

// open-addressing hash-consing table over variable-length word sequences
struct NodeTable {
    std::vector<uint32_t> slots;  // node offset + 1 into `words`, 0 = empty
    std::vector<uint32_t> words;  // [mask, count, children...] per node
    size_t n = 0;
    void reset(size_t expect) {
        size_t cap = 64;
        while (cap < expect * 2) cap <<= 1;
        slots.assign(cap, 0);
        words.clear();
        n = 0;
    }
    uint32_t intern(const uint32_t* key, int len) {  // key = [mask, count, children...]
        uint64_t h = 0x9E3779B97F4A7C15ull;
        for (int i = 0; i < len; i++) h = mix64(h ^ key[i]);
        size_t m = slots.size() - 1, i = (size_t)h & m;
        for (;;) {
            uint32_t s = slots[i];
            if (!s) break;
            const uint32_t* cand = &words[s - 1];
            int clen = 2 + __builtin_popcount(cand[0]);
            if (clen == len && std::memcmp(cand, key, sizeof(uint32_t) * len) == 0) return s - 1;
            i = (i + 1) & m;
        }
        uint32_t off = (uint32_t)words.size();
        words.insert(words.end(), key, key + len);
        slots[i] = off + 1;
        if (++n * 2 > slots.size()) grow();
        return off;
    }
    void grow() {
        std::vector<uint32_t> old;
        old.swap(slots);
        slots.assign(old.size() * 2, 0);
        size_t m = slots.size() - 1;
        for (uint32_t s : old) {
            if (!s) continue;
            const uint32_t* key = &words[s - 1];
            int len = 2 + __builtin_popcount(key[0]);
            uint64_t h = 0x9E3779B97F4A7C15ull;
            for (int i = 0; i < len; i++) h = mix64(h ^ key[i]);
            size_t i = (size_t)h & m;
            while (slots[i]) i = (i + 1) & m;
            slots[i] = s;
        }
    }
};

struct LeafTable {
    std::vector<uint64_t> keys;
    std::vector<uint32_t> ids;  // id + 1
    std::vector<uint64_t> masks;
    void reset(size_t expect) {
        size_t cap = 64;
        while (cap < expect * 2) cap <<= 1;
        keys.assign(cap, 0);
        ids.assign(cap, 0);
        masks.clear();
    }
    uint32_t intern(uint64_t m) {
        size_t cap = keys.size() - 1, i = (size_t)mix64(m) & cap;
        while (ids[i]) {
            if (keys[i] == m) return ids[i] - 1;
            i = (i + 1) & cap;
        }
        keys[i] = m;
        ids[i] = (uint32_t)masks.size() + 1;
        masks.push_back(m);
        if (masks.size() * 2 > keys.size()) {
            std::vector<uint64_t> ok;
            std::vector<uint32_t> oi;
            ok.swap(keys);
            oi.swap(ids);
            keys.assign(ok.size() * 2, 0);
            ids.assign(ok.size() * 2, 0);
            size_t c2 = keys.size() - 1;
            for (size_t j = 0; j < ok.size(); j++) {
                if (!oi[j]) continue;
                size_t k = (size_t)mix64(ok[j]) & c2;
                while (ids[k]) k = (k + 1) & c2;
                keys[k] = ok[j];
                ids[k] = oi[j];
            }
        }
        return (uint32_t)masks.size() - 1;
    }
};

struct Blob {
    std::vector<uint32_t> nodes;
    std::vector<uint64_t> leaves;
    std::vector<uint8_t> mats;
    uint32_t root = 0;
    int32_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
};

constexpr uint32_t NONE = 0xFFFFFFFFu;

// Build the DAG of one dense LOD grid (bits, side r); mat(x, y, z) gives the
// material of a solid voxel (LOD-local coordinates).
template <class MatFn>
void build_dag(const BitGrid& g, MatFn mat, Blob& out) {
    const int r = g.r, nb = r / 4;
    const size_t nblk = (size_t)nb * nb * nb;
    // 4x4x4 leaf masks, bit x + 4y + 16z, block index bx + nb*(by + nb*bz)
    std::vector<uint64_t> lm(nblk, 0);
    size_t nonempty = 0;
    // per row of blocks (by, bz) and 64-bit word of x: the 16 words of its 4 x 4
    // voxel rows; all zero = 16 (or r / 4) empty blocks at once
    const int bpw = std::min(16, nb);  // blocks per word
    for (int bz = 0; bz < nb; bz++)
        for (int by = 0; by < nb; by++)
            for (int wx = 0; wx < g.w64; wx++) {
                uint64_t rw[16], any = 0;
                for (int z = 0; z < 4; z++)
                    for (int y = 0; y < 4; y++) {
                        rw[4 * z + y] = g.w[(size_t)wx + (size_t)g.w64 * ((size_t)(4 * by + y) + (size_t)r * (4 * bz + z))];
                        any |= rw[4 * z + y];
                    }
                if (!any) continue;
                for (int j = 0; j < bpw; j++) {
                    uint64_t m = 0;
                    for (int q = 0; q < 16; q++) m |= ((rw[q] >> (4 * j)) & 0xFull) << (4 * q);
                    if (!m) continue;
                    const int bx = wx * 16 + j;
                    lm[(size_t)bx + (size_t)nb * ((size_t)by + (size_t)nb * bz)] = m;
                    nonempty++;
                }
            }
    if (!nonempty) {  // empty chunk
        out = Blob();
        return;
    }
    // leaves: hash-consed ids per block
    LeafTable lt;
    lt.reset(nonempty);
    std::vector<uint32_t> ids(nblk, NONE);
    for (size_t i = 0; i < nblk; i++)
        if (lm[i]) ids[i] = lt.intern(lm[i]);
    // interior levels bottom-up; per level keep the id grid (for DFS emission)
    int levels = 0;
    for (int s = r; s > 4; s >>= 1) levels++;  // interior levels: node sides r .. 8
    std::vector<NodeTable> tabs(levels);
    std::vector<std::vector<uint32_t>> grids(levels + 1);  // grids[levels] = leaf ids
    grids[levels] = std::move(ids);
    std::vector<uint64_t> cnt_leaf(lt.masks.size());
    for (size_t i = 0; i < lt.masks.size(); i++) cnt_leaf[i] = (uint64_t)__builtin_popcountll(lt.masks[i]);
    int n = nb;
    for (int lev = levels - 1; lev >= 0; lev--) {
        const int p = n / 2;
        const std::vector<uint32_t>& cg = grids[lev + 1];
        std::vector<uint32_t> pg((size_t)p * p * p, NONE);
        NodeTable& t = tabs[lev];
        t.reset(std::max<size_t>(16, (size_t)p * p * p / 8));
        const bool leaf_children = lev == levels - 1;
        uint32_t key[10];
        for (int z = 0; z < p; z++)
            for (int y = 0; y < p; y++)
                for (int x = 0; x < p; x++) {
                    uint32_t mask = 0;
                    int k = 2;
                    uint64_t c = 0;
                    for (int o = 0; o < 8; o++) {
                        size_t ci = (size_t)(2 * x + (o & 1)) +
                                    (size_t)n * ((size_t)(2 * y + ((o >> 1) & 1)) + (size_t)n * (size_t)(2 * z + (o >> 2)));
                        uint32_t ch = cg[ci];
                        if (ch == NONE) continue;
                        mask |= 1u << o;
                        key[k++] = ch;
                        c += leaf_children ? cnt_leaf[ch] : tabs[lev + 1].words[ch + 1];
                    }
                    if (!mask) continue;
                    key[0] = mask;
                    key[1] = (uint32_t)c;
                    pg[(size_t)x + (size_t)p * ((size_t)y + (size_t)p * z)] = t.intern(key, k);
                }
        grids[lev] = std::move(pg);
        n = p;
    }
    // breadth-first relayout: level by level from the root
    std::vector<std::vector<uint32_t>> newoff(levels);
    std::vector<uint32_t> leafnew(lt.masks.size(), NONE);
    out.nodes.clear();
    out.leaves.clear();
    std::vector<uint32_t> frontier{grids[0][0]}, next;
    newoff[0].assign(tabs[0].words.size(), NONE);
    newoff[0][grids[0][0]] = 0;
    // first pass assigns offsets level by level, second pass writes words
    std::vector<std::vector<uint32_t>> order(levels);
    order[0] = frontier;
    uint32_t woff = 2 + __builtin_popcount(tabs[0].words[grids[0][0]]);
    for (int lev = 0; lev < levels; lev++) {
        next.clear();
        if (lev + 1 < levels) newoff[lev + 1].assign(tabs[lev + 1].words.size(), NONE);
        for (uint32_t id : order[lev]) {
            const uint32_t* w = &tabs[lev].words[id];
            int k = __builtin_popcount(w[0]);
            for (int c = 0; c < k; c++) {
                uint32_t ch = w[2 + c];
                if (lev + 1 < levels) {
                    if (newoff[lev + 1][ch] == NONE) {
                        newoff[lev + 1][ch] = woff;
                        woff += 2 + __builtin_popcount(tabs[lev + 1].words[ch]);
                        next.push_back(ch);
                    }
                } else if (leafnew[ch] == NONE) {
                    leafnew[ch] = (uint32_t)out.leaves.size();
                    out.leaves.push_back(lt.masks[ch]);
                }
            }
        }
        if (lev + 1 < levels) order[lev + 1] = next;
    }
    out.nodes.resize(woff);
    for (int lev = 0; lev < levels; lev++) {
        for (uint32_t id : order[lev]) {
            const uint32_t* w = &tabs[lev].words[id];
            int k = __builtin_popcount(w[0]);
            uint32_t o = newoff[lev][id];
            out.nodes[o] = w[0];
            out.nodes[o + 1] = w[1];
            for (int c = 0; c < k; c++) out.nodes[o + 2 + c] = lev + 1 < levels ? newoff[lev + 1][w[2 + c]] : leafnew[w[2 + c]];
        }
    }
    out.root = 0;
    // depth-first materials and AABB, walking tree positions (ascending octant, then leaf bit)
    out.mats.clear();
    out.mats.reserve(tabs[0].words[grids[0][0] + 1]);
    int lo[3] = {r, r, r}, hi[3] = {-1, -1, -1};
    struct Frame { int lev, x, y, z, oct; };
    std::vector<Frame> st;
    st.push_back({0, 0, 0, 0, 0});
    while (!st.empty()) {
        Frame& f = st.back();
        if (f.oct == 8) { st.pop_back(); continue; }
        int o = f.oct++;
        int cx = 2 * f.x + (o & 1), cy = 2 * f.y + ((o >> 1) & 1), cz = 2 * f.z + (o >> 2);
        int side = 1 << (f.lev + 1);  // cells per axis at level lev + 1
        uint32_t ch = grids[f.lev + 1][(size_t)cx + (size_t)side * ((size_t)cy + (size_t)side * cz)];
        if (ch == NONE) continue;
        if (f.lev + 1 < levels) {
            st.push_back({f.lev + 1, cx, cy, cz, 0});
        } else {
            uint64_t m = lt.masks[ch];
            while (m) {
                int bit = __builtin_ctzll(m);
                m &= m - 1;
                int vx = 4 * cx + (bit & 3), vy = 4 * cy + ((bit >> 2) & 3), vz = 4 * cz + (bit >> 4);
                out.mats.push_back(mat(vx, vy, vz));
                lo[0] = std::min(lo[0], vx); lo[1] = std::min(lo[1], vy); lo[2] = std::min(lo[2], vz);
                hi[0] = std::max(hi[0], vx); hi[1] = std::max(hi[1], vy); hi[2] = std::max(hi[2], vz);
            }
        }
    }
    for (int a = 0; a < 3; a++) { out.lo[a] = lo[a]; out.hi[a] = hi[a] + 1; }
}

// One LOD step (Sec. 3.4): a voxel exists iff >= 2 of its 8 children exist; its
// material is the rounded mean of the existing children's (mat(x, y, z) of
// the finer grid).
template <class MatFn>
void aggregate(const BitGrid& g, MatFn mat, BitGrid& g2, std::vector<uint8_t>& mat2) {
    const int r = g.r, h = r / 2;
    g2.init(h);
    mat2.resize((size_t)h * h * h);
    for (int z = 0; z < h; z++)
        for (int y = 0; y < h; y++)
            for (int x0 = 0; x0 < h; x0 += 32) {
                const int xn = std::min(32, h - x0);
                uint64_t rows[4];
                for (int k = 0; k < 4; k++) {
                    int yy = 2 * y + (k & 1), zz = 2 * z + (k >> 1);
                    int xb = 2 * x0;  // 64 source bits
                    rows[k] = g.w[(size_t)(xb >> 6) + (size_t)g.w64 * ((size_t)yy + (size_t)r * zz)] >> (xb & 63);
                }
                if ((rows[0] | rows[1] | rows[2] | rows[3]) == 0) continue;  // nothing below these 32 voxels
                for (int i = 0; i < xn; i++) {
                    int c = 0;
                    for (int k = 0; k < 4; k++) c += __builtin_popcountll((rows[k] >> (2 * i)) & 3);
                    if (c < 2) continue;
                    int x = x0 + i;
                    int sum = 0;
                    for (int k = 0; k < 4; k++) {
                        int yy = 2 * y + (k & 1), zz = 2 * z + (k >> 1);
                        for (int dx = 0; dx < 2; dx++)
                            if ((rows[k] >> (2 * i + dx)) & 1) sum += mat(2 * x + dx, yy, zz);
                    }
                    g2.w[(size_t)(x >> 6) + (size_t)g2.w64 * ((size_t)y + (size_t)h * z)] |= 1ull << (x & 63);
                    mat2[(size_t)x + (size_t)h * ((size_t)y + (size_t)h * z)] = (uint8_t)((sum + c / 2) / c);
                }
            }
}

void build_chunk(const sg_scene* w, int M, int L, int cx, int cy, int cz, Blob* out /* [L] */,
                 uint32_t lod_mask = 0xFFFFFFFFu) {
    BitGrid g;
    g.init(M);
    uint64_t solid;
    if (M % 64 == 0) {
        solid = sg_fill_bits(w, cx * M, cy * M, cz * M, M, M, M, g.w.data());
    } else {
        std::vector<uint8_t> b((size_t)M * M * M);
        solid = sg_fill_bytes(w, cx * M, cy * M, cz * M, M, M, M, b.data());
        for (int z = 0; z < M; z++)
            for (int y = 0; y < M; y++)
                for (int x = 0; x < M; x++)
                    if (b[(size_t)x + (size_t)M * ((size_t)y + (size_t)M * z)])
                        g.w[(size_t)(x >> 6) + (size_t)g.w64 * ((size_t)y + (size_t)M * z)] |= 1ull << (x & 63);
    }
    if (!solid) {
        for (int l = 0; l < L; l++) out[l] = Blob();
        return;
    }
    // LOD 0 materials straight from the generator; coarser LODs in dense grids
    const int ox = cx * M, oy = cy * M, oz = cz * M;
    auto mat0 = [&](int x, int y, int z) -> uint8_t { return sg_material(w, ox + x, oy + y, oz + z); };
    std::vector<uint8_t> mat;
    int last = -1;
    for (int l = 0; l < L; l++)
        if ((lod_mask >> l) & 1u) last = l;
    for (int l = 0; l <= last; l++) {
        const int rl = g.r;
        auto matl = [&](int x, int y, int z) -> uint8_t {
            return mat[(size_t)x + (size_t)rl * ((size_t)y + (size_t)rl * z)];
        };
        if ((lod_mask >> l) & 1u) {
            if (l == 0) build_dag(g, mat0, out[l]);
            else build_dag(g, matl, out[l]);
            for (int a = 0; a < 3; a++) {  // AABB to chunk-local LOD-0 units
                out[l].lo[a] <<= l;
                out[l].hi[a] <<= l;
            }
        } else {
            out[l] = Blob();
        }
        if (l + 1 <= last) {
            BitGrid g2;
            std::vector<uint8_t> m2;
            if (l == 0) aggregate(g, mat0, g2, m2);
            else aggregate(g, matl, g2, m2);
            g = std::move(g2);
            mat = std::move(m2);
        }
    }
    for (int l = last + 1; l < L; l++) out[l] = Blob();
}

}  // namespace

extern "C" {

typedef struct aokb_world {
    int M, L;
    int64_t n_chunks;
    std::vector<int64_t> chunks;  // chunk index (x fastest) per built entry
    std::vector<Blob> blobs;      // [entry * L + lod]
} aokb_world;

// Build the LODs of the listed chunk regions (chunk index = cx + gx*(cy + gy*cz)),
// or of every chunk region when chunks == NULL.  lod_masks (optional, one per
// listed chunk): bit l set = emit LOD l (other LODs come back empty).
aokb_world* aokb_build_masked(const sg_scene* w, int32_t M, int32_t L, const int64_t* chunks, const uint32_t* lod_masks,
                              int64_t n, int32_t n_threads) {
    const sg_params* p = sg_get_params(w);
    if (M < 8 || (M & (M - 1)) || L < 1 || (M >> (L - 1)) < 8 || p->wx % M || p->wy % M || p->wz % M) return nullptr;
    auto* out = new aokb_world();
    out->M = M;
    out->L = L;
    const int64_t gx = p->wx / M, gy = p->wy / M, gz = p->wz / M;
    out->n_chunks = gx * gy * gz;
    if (chunks) out->chunks.assign(chunks, chunks + n);
    else for (int64_t c = 0; c < out->n_chunks; c++) out->chunks.push_back(c);
    out->blobs.resize(out->chunks.size() * L);
    std::atomic<int64_t> next{0};
    int nt = std::max(1, (int)n_threads);
    std::vector<std::thread> th;
    for (int t = 0; t < nt; t++)
        th.emplace_back([&]() {
            for (;;) {
                int64_t i = next.fetch_add(1);
                if (i >= (int64_t)out->chunks.size()) break;
                int64_t c = out->chunks[i];
                build_chunk(w, M, L, (int)(c % gx), (int)((c / gx) % gy), (int)(c / (gx * gy)), &out->blobs[i * L],
                            (chunks && lod_masks) ? lod_masks[i] : 0xFFFFFFFFu);
            }
        });
    for (auto& t : th) t.join();
    return out;
}

aokb_world* aokb_build(const sg_scene* w, int32_t M, int32_t L, const int64_t* chunks, int64_t n, int32_t n_threads) {
    return aokb_build_masked(w, M, L, chunks, nullptr, n, n_threads);
}

void aokb_free(aokb_world* b) { delete b; }

int64_t aokb_count(const aokb_world* b) { return b ? (int64_t)b->chunks.size() : 0; }

// Entry i: its chunk index and the blob of one LOD (pointers into builder memory).
int aokb_get(const aokb_world* b, int64_t i, int32_t lod, int64_t* chunk, aok_chunk_blob* out) {
    if (!b || i < 0 || i >= (int64_t)b->chunks.size() || lod < 0 || lod >= b->L) return -1;
    const Blob& s = b->blobs[i * b->L + lod];
    *chunk = b->chunks[i];
    out->nodes = s.nodes.data();
    out->n_node_words = s.nodes.size();
    out->leaves = s.leaves.data();
    out->n_leaves = s.leaves.size();
    out->mats = s.mats.data();
    out->n_mats = s.mats.size();
    out->root = s.root;
    for (int a = 0; a < 3; a++) { out->aabb_lo[a] = s.lo[a]; out->aabb_hi[a] = s.hi[a]; }
    return 0;
}

// Chunk source for aok_stream (the callback types of include/aok.h): builds
// one (chunk, LOD) of a world on the calling thread.  The blob points into a
// builder-owned allocation returned through *handle and freed by
// aokb_source_release.
typedef struct aokb_source {
    const sg_scene* w;
    int M, L;
    int64_t gx, gy, gz;
} aokb_source;

aokb_source* aokb_source_create(const sg_scene* w, int32_t M, int32_t L) {
    const sg_params* p = sg_get_params(w);
    if (M < 8 || (M & (M - 1)) || L < 1 || (M >> (L - 1)) < 8 || p->wx % M || p->wy % M || p->wz % M) return nullptr;
    return new aokb_source{w, M, L, p->wx / M, p->wy / M, p->wz / M};
}

void aokb_source_destroy(aokb_source* s) { delete s; }

int aokb_source_build(void* user, int32_t cx, int32_t cy, int32_t cz, uint32_t lod, aok_chunk_blob* out,
                      void** handle) {
    const aokb_source* s = (const aokb_source*)user;
    if (!s || !out || !handle || cx < 0 || cy < 0 || cz < 0 || cx >= s->gx || cy >= s->gy || cz >= s->gz ||
        (int)lod >= s->L)
        return -1;
    std::vector<Blob>* blobs = new std::vector<Blob>(s->L);
    build_chunk(s->w, s->M, s->L, cx, cy, cz, blobs->data(), 1u << lod);
    const Blob& b = (*blobs)[lod];
    out->nodes = b.nodes.data();
    out->n_node_words = b.nodes.size();
    out->leaves = b.leaves.data();
    out->n_leaves = b.leaves.size();
    out->mats = b.mats.data();
    out->n_mats = b.mats.size();
    out->root = b.root;
    for (int a = 0; a < 3; a++) { out->aabb_lo[a] = b.lo[a]; out->aabb_hi[a] = b.hi[a]; }
    *handle = blobs;
    return 0;
}

void aokb_source_release(void* user, void* handle) {
    (void)user;
    delete (std::vector<Blob>*)handle;
}

// Totals over all entries: [0] node words, [1] leaves, [2] material bytes, [3] non-empty blobs.
void aokb_totals(const aokb_world* b, uint64_t out[4]) {
    out[0] = out[1] = out[2] = out[3] = 0;
    if (!b) return;
    for (const Blob& s : b->blobs) {
        out[0] += s.nodes.size();
        out[1] += s.leaves.size();
        out[2] += s.mats.size();
        out[3] += !s.nodes.empty();
    }
}

}  // extern "C"
