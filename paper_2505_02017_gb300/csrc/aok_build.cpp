// Offline chunk preparation (Sec. 3.1-3.4): per chunk region, LOD aggregation
// (density 2, average material) and one sparse voxel DAG per LOD with
// subtree leaf counts and a depth-first material array, in the blob format
// of aok.h.  Input voxels come from scenegen; chunks are built in parallel.
//
// Layout choices (not fixed by the paper): each LOD is held as 64-bit masks
// of 4x4x4 blocks over the z slab that holds solid voxels (the generator's
// bit rows are regrouped once); identical subtrees are merged by hash-consing
// per level; the final node pool is laid out breadth-first from the root, so
// a chunk's upper levels are contiguous, and leaves follow in first-reference
// order.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <list>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/aok.h"
#include "../../scenegen/scenegen.h"

namespace {

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

// ---- one LOD of a chunk region as 4x4x4 blocks ----
// Occupancy per block (bit x + 4y + 16z); only the slab of block layers
// [bz0, bz1) that holds solid voxels is stored, block (bx, by, bz) at
// index bx + nb*(by + nb*(bz - bz0)).  Aggregated LODs keep the materials of
// each non-empty block in a 64-byte slot (entry = bit); LOD 0 materials come
// from the generator.
struct Blocks {
    int r = 0, nb = 0, bz0 = 0, bz1 = 0;
    std::vector<uint64_t> m;
    std::vector<uint32_t> slot;  // material slot per block (NONE: empty), LOD >= 1 only
    std::vector<uint8_t> mat;    // 64 bytes per slot
    size_t index(int bx, int by, int bz) const {
        return (size_t)bx + (size_t)nb * ((size_t)by + (size_t)nb * (size_t)(bz - bz0));
    }
    uint64_t mask(int bx, int by, int bz) const { return bz < bz0 || bz >= bz1 ? 0 : m[index(bx, by, bz)]; }
    void init(int side, int z0, int z1, bool slots) {
        r = side;
        nb = side / 4;
        bz0 = z0;
        bz1 = std::max(z0, z1);
        const size_t n = (size_t)nb * nb * (size_t)(bz1 - bz0);
        m.assign(n, 0);
        if (slots) slot.assign(n, NONE);
        else slot.clear();
        mat.clear();
    }
};

// x, y, z extents of the solid voxels of one block mask (bit sets 0..15 per axis)
inline void block_extent(uint64_t m, uint32_t e[3]) {
    uint64_t t = m | (m >> 32);
    t |= t >> 16;
    const uint32_t xy = (uint32_t)t & 0xFFFFu;
    e[0] = (xy | xy >> 4 | xy >> 8 | xy >> 12) & 0xFu;
    e[1] = (uint32_t)((xy & 0xFu) != 0) | (uint32_t)((xy & 0xF0u) != 0) << 1 | (uint32_t)((xy & 0xF00u) != 0) << 2 |
           (uint32_t)((xy & 0xF000u) != 0) << 3;
    e[2] = (uint32_t)((m & 0xFFFFull) != 0) | (uint32_t)(((m >> 16) & 0xFFFFull) != 0) << 1 |
           (uint32_t)(((m >> 32) & 0xFFFFull) != 0) << 2 | (uint32_t)((m >> 48) != 0) << 3;
}

// Per-thread LOD-0 bit grid (side M, rows of w64 = ceil(M/64) words, row y + M*z),
// reused across chunks: only the rows the last fill wrote are cleared.
struct FillScratch {
    int r = 0, w64 = 0, dz0 = 0, dz1 = 0;  // rows of z in [dz0, dz1) may hold bits
    std::vector<uint64_t> w;
    uint64_t* prepare(int side) {
        if (side != r) {
            r = side;
            w64 = (side + 63) / 64;
            w.assign((size_t)w64 * side * side, 0);
            dz0 = dz1 = 0;
        } else if (dz1 > dz0) {
            std::memset(w.data() + (size_t)w64 * r * dz0, 0, sizeof(uint64_t) * (size_t)w64 * r * (dz1 - dz0));
        }
        dz0 = dz1 = 0;
        return w.data();
    }
};

// Block masks of the rows [z0, z1) of a bit grid; per row of blocks (by, bz)
// and 64-bit word of x, the 16 words of its 4 x 4 voxel rows: all zero = up to
// 16 empty blocks at once.
void blocks_from_bits(const FillScratch& g, int z0, int z1, Blocks& B) {
    B.init(g.r, z0 / 4, (z1 + 3) / 4, false);
    const int nb = B.nb, bpw = std::min(16, nb);
    for (int bz = B.bz0; bz < B.bz1; bz++)
        for (int by = 0; by < nb; by++)
            for (int wx = 0; wx < g.w64; wx++) {
                uint64_t rw[16], any = 0;
                for (int z = 0; z < 4; z++)
                    for (int y = 0; y < 4; y++) {
                        rw[4 * z + y] =
                            g.w[(size_t)wx + (size_t)g.w64 * ((size_t)(4 * by + y) + (size_t)g.r * (size_t)(4 * bz + z))];
                        any |= rw[4 * z + y];
                    }
                if (!any) continue;
                for (int j = 0; j < bpw; j++) {
                    uint64_t m = 0;
                    for (int q = 0; q < 16; q++) m |= ((rw[q] >> (4 * j)) & 0xFull) << (4 * q);
                    B.m[B.index(wx * 16 + j, by, bz)] = m;
                }
            }
}

// Node ids of one DAG level (side n, cells x + n*(y + n*(z - z0)) for z in [z0, z1))
struct Level {
    int n = 0, z0 = 0, z1 = 0;
    std::vector<uint32_t> id;
    void init(int side, int lo, int hi) {
        n = side;
        z0 = lo;
        z1 = std::max(lo, hi);
        id.assign((size_t)n * n * (size_t)(z1 - z0), NONE);
    }
    uint32_t& at(int x, int y, int z) { return id[(size_t)x + (size_t)n * ((size_t)y + (size_t)n * (size_t)(z - z0))]; }
    uint32_t get(int x, int y, int z) const {
        return z < z0 || z >= z1 ? NONE : id[(size_t)x + (size_t)n * ((size_t)y + (size_t)n * (size_t)(z - z0))];
    }
};

// Build the DAG of one LOD (blocks B, side r); matb(B, bx, by, bz, mask, tmp)
// returns the materials of a block's solid voxels (entry = bit).
template <class MatBlock>
void build_dag(const Blocks& B, MatBlock matb, Blob& out) {
    const int r = B.r, nb = B.nb;
    // leaves: hash-consed ids per block
    size_t nonempty = 0;
    for (uint64_t m : B.m) nonempty += m != 0;
    if (!nonempty) {  // empty chunk
        out = Blob();
        return;
    }
    LeafTable lt;
    lt.reset(nonempty);
    int levels = 0;
    for (int s = r; s > 4; s >>= 1) levels++;  // interior levels: node sides r .. 8
    std::vector<NodeTable> tabs(levels);
    std::vector<Level> grids(levels + 1);  // grids[levels] = leaf ids
    {
        Level& lv = grids[levels];
        lv.init(nb, B.bz0, B.bz1);
        for (size_t i = 0; i < B.m.size(); i++)
            if (B.m[i]) lv.id[i] = lt.intern(B.m[i]);
    }
    // interior levels bottom-up
    std::vector<uint64_t> cnt_leaf(lt.masks.size());
    for (size_t i = 0; i < lt.masks.size(); i++) cnt_leaf[i] = (uint64_t)__builtin_popcountll(lt.masks[i]);
    for (int lev = levels - 1; lev >= 0; lev--) {
        const Level& cg = grids[lev + 1];
        const int p = cg.n / 2;
        Level& pg = grids[lev];
        pg.init(p, cg.z0 / 2, (cg.z1 + 1) / 2);
        NodeTable& t = tabs[lev];
        t.reset(std::max<size_t>(16, pg.id.size() / 8));
        const bool leaf_children = lev == levels - 1;
        uint32_t key[10];
        for (int z = pg.z0; z < pg.z1; z++)
            for (int y = 0; y < p; y++)
                for (int x = 0; x < p; x++) {
                    uint32_t mask = 0;
                    int k = 2;
                    uint64_t c = 0;
                    for (int o = 0; o < 8; o++) {
                        const uint32_t ch = cg.get(2 * x + (o & 1), 2 * y + ((o >> 1) & 1), 2 * z + (o >> 2));
                        if (ch == NONE) continue;
                        mask |= 1u << o;
                        key[k++] = ch;
                        c += leaf_children ? cnt_leaf[ch] : tabs[lev + 1].words[ch + 1];
                    }
                    if (!mask) continue;
                    key[0] = mask;
                    key[1] = (uint32_t)c;
                    pg.at(x, y, z) = t.intern(key, k);
                }
    }
    const uint32_t root = grids[0].get(0, 0, 0);
    // breadth-first relayout: level by level from the root
    std::vector<std::vector<uint32_t>> newoff(levels);
    std::vector<uint32_t> leafnew(lt.masks.size(), NONE);
    out.nodes.clear();
    out.leaves.clear();
    std::vector<uint32_t> next;
    newoff[0].assign(tabs[0].words.size(), NONE);
    newoff[0][root] = 0;
    // first pass assigns offsets level by level, second pass writes words
    std::vector<std::vector<uint32_t>> order(levels);
    order[0] = {root};
    uint32_t woff = 2 + __builtin_popcount(tabs[0].words[root]);
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
    out.mats.reserve(tabs[0].words[root + 1]);
    int lo[3] = {r, r, r}, hi[3] = {-1, -1, -1};
    struct Frame { int lev, x, y, z, oct; };
    std::vector<Frame> st;
    st.push_back({0, 0, 0, 0, 0});
    uint8_t tmp[64];
    while (!st.empty()) {
        Frame& f = st.back();
        if (f.oct == 8) { st.pop_back(); continue; }
        int o = f.oct++;
        int cx = 2 * f.x + (o & 1), cy = 2 * f.y + ((o >> 1) & 1), cz = 2 * f.z + (o >> 2);
        uint32_t ch = grids[f.lev + 1].get(cx, cy, cz);
        if (ch == NONE) continue;
        if (f.lev + 1 < levels) {
            st.push_back({f.lev + 1, cx, cy, cz, 0});
        } else {
            uint64_t m = lt.masks[ch];
            const uint8_t* mt = matb(B, cx, cy, cz, m, tmp);
            uint32_t e[3];
            block_extent(m, e);
            const int c4[3] = {4 * cx, 4 * cy, 4 * cz};
            for (int a = 0; a < 3; a++) {
                lo[a] = std::min(lo[a], c4[a] + __builtin_ctz(e[a]));
                hi[a] = std::max(hi[a], c4[a] + 31 - __builtin_clz(e[a]));
            }
            while (m) {
                const int bit = __builtin_ctzll(m);
                m &= m - 1;
                out.mats.push_back(mt[bit]);
            }
        }
    }
    for (int a = 0; a < 3; a++) { out.lo[a] = lo[a]; out.hi[a] = hi[a] + 1; }
}

// One LOD step (Sec. 3.4): a voxel exists iff >= 2 of its 8 children exist; its
// material is the rounded mean of the existing children's.  Coarse block
// (X, Y, Z) takes its 2x2x2 voxel octants from the 8 fine blocks
// (2X + i, 2Y + j, 2Z + k).
template <class MatBlock>
void aggregate(const Blocks& F, MatBlock matb, Blocks& C) {
    C.init(F.r / 2, F.bz0 / 2, (F.bz1 + 1) / 2, true);
    const int nc = C.nb;
    uint8_t tmp[64], cm8[64];
    for (int Z = C.bz0; Z < C.bz1; Z++)
        for (int Y = 0; Y < nc; Y++)
            for (int X = 0; X < nc; X++) {
                uint64_t fm[8], any = 0;
                for (int o = 0; o < 8; o++) {
                    fm[o] = F.mask(2 * X + (o & 1), 2 * Y + ((o >> 1) & 1), 2 * Z + (o >> 2));
                    any |= fm[o];
                }
                if (!any) continue;
                uint64_t cm = 0;
                for (int o = 0; o < 8; o++) {
                    if (!fm[o]) continue;
                    const uint8_t* fmat = matb(F, 2 * X + (o & 1), 2 * Y + ((o >> 1) & 1), 2 * Z + (o >> 2), fm[o], tmp);
                    for (int s = 0; s < 8; s++) {
                        const int a = s & 1, b = (s >> 1) & 1, c = s >> 2;
                        uint64_t sub = fm[o] & (0x330033ull << (2 * a + 8 * b + 32 * c));
                        const int cnt = __builtin_popcountll(sub);
                        if (cnt < 2) continue;
                        int sum = 0;
                        while (sub) {
                            sum += fmat[__builtin_ctzll(sub)];
                            sub &= sub - 1;
                        }
                        const int q = (2 * (o & 1) + a) + 4 * (2 * ((o >> 1) & 1) + b) + 16 * (2 * (o >> 2) + c);
                        cm |= 1ull << q;
                        cm8[q] = (uint8_t)((sum + cnt / 2) / cnt);
                    }
                }
                if (!cm) continue;
                const size_t i = C.index(X, Y, Z);
                C.m[i] = cm;
                C.slot[i] = (uint32_t)(C.mat.size() / 64);
                C.mat.insert(C.mat.end(), cm8, cm8 + 64);
            }
}

void build_chunk(const sg_scene* w, int M, int L, int cx, int cy, int cz, Blob* out /* [L] */,
                 uint32_t lod_mask = 0xFFFFFFFFu) {
    static thread_local FillScratch g;
    int last = -1;
    for (int l = 0; l < L; l++)
        if ((lod_mask >> l) & 1u) last = l;
    for (int l = 0; l < L; l++) out[l] = Blob();
    if (last < 0) return;
    uint64_t* bits = g.prepare(M);
    int zr[2] = {0, 0};
    const int ox = cx * M, oy = cy * M, oz = cz * M;
    if (M % 64 == 0) {
        if (sg_fill_bits_z(w, ox, oy, oz, M, M, M, bits, zr) <= 0) return;
    } else {
        std::vector<uint8_t> b((size_t)M * M * M);
        if (!sg_fill_bytes(w, ox, oy, oz, M, M, M, b.data())) return;
        zr[0] = M;
        for (int z = 0; z < M; z++)
            for (int y = 0; y < M; y++)
                for (int x = 0; x < M; x++)
                    if (b[(size_t)x + (size_t)M * ((size_t)y + (size_t)M * z)]) {
                        bits[(size_t)(x >> 6) + (size_t)g.w64 * ((size_t)y + (size_t)M * z)] |= 1ull << (x & 63);
                        zr[0] = std::min(zr[0], z);
                        zr[1] = z + 1;
                    }
    }
    g.dz0 = zr[0];
    g.dz1 = zr[1];
    // LOD 0 materials straight from the generator; coarser LODs from their blocks' slots
    auto mat0 = [&](const Blocks&, int bx, int by, int bz, uint64_t m, uint8_t* tmp) -> const uint8_t* {
        sg_materials_block4(w, ox + 4 * bx, oy + 4 * by, oz + 4 * bz, m, tmp);
        return tmp;
    };
    auto matl = [](const Blocks& B, int bx, int by, int bz, uint64_t, uint8_t*) -> const uint8_t* {
        return &B.mat[(size_t)64 * B.slot[B.index(bx, by, bz)]];
    };
    Blocks cur, next;
    blocks_from_bits(g, zr[0], zr[1], cur);
    for (int l = 0; l <= last; l++) {
        if ((lod_mask >> l) & 1u) {
            if (l == 0) build_dag(cur, mat0, out[l]);
            else build_dag(cur, matl, out[l]);
            for (int a = 0; a < 3; a++) {  // AABB to chunk-local LOD-0 units
                out[l].lo[a] <<= l;
                out[l].hi[a] <<= l;
            }
        }
        if (l + 1 <= last) {
            if (l == 0) aggregate(cur, mat0, next);
            else aggregate(cur, matl, next);
            std::swap(cur, next);
        }
    }
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
// aokb_source_release.  With a cache (aokb_source_set_cache) a build also
// makes the region's coarser LODs (their aggregation is a small part of the
// work), and recently built blobs are kept in host memory up to a byte
// budget, least recently used out first: a (chunk, LOD) asked for again --
// a region leaving and re-entering the view, or its LOD switching back --
// costs no second build.
struct aokb_source {
    const sg_scene* w;
    int M, L;
    int64_t gx, gy, gz;
    std::mutex mu;
    size_t cap = 0, bytes = 0;
    uint64_t hits = 0, misses = 0;
    std::list<int64_t> lru;  // most recently used first
    struct Entry {
        std::shared_ptr<const Blob> blob;
        size_t bytes;
        std::list<int64_t>::iterator pos;
    };
    std::unordered_map<int64_t, Entry> cache;  // key chunk * L + lod

    void evict_to(size_t limit) {
        while (bytes > limit && !lru.empty()) {
            auto it = cache.find(lru.back());
            bytes -= it->second.bytes;
            cache.erase(it);
            lru.pop_back();
        }
    }
};

namespace {
size_t blob_bytes(const Blob& b) { return b.nodes.size() * 4 + b.leaves.size() * 8 + b.mats.size() + sizeof(Blob); }

void fill_blob(const Blob& b, aok_chunk_blob* out) {
    out->nodes = b.nodes.data();
    out->n_node_words = b.nodes.size();
    out->leaves = b.leaves.data();
    out->n_leaves = b.leaves.size();
    out->mats = b.mats.data();
    out->n_mats = b.mats.size();
    out->root = b.root;
    for (int a = 0; a < 3; a++) { out->aabb_lo[a] = b.lo[a]; out->aabb_hi[a] = b.hi[a]; }
}
}  // namespace

aokb_source* aokb_source_create(const sg_scene* w, int32_t M, int32_t L) {
    const sg_params* p = sg_get_params(w);
    if (M < 8 || (M & (M - 1)) || L < 1 || L > 8 || (M >> (L - 1)) < 8 || p->wx % M || p->wy % M || p->wz % M)
        return nullptr;
    aokb_source* s = new aokb_source();
    s->w = w;
    s->M = M;
    s->L = L;
    s->gx = p->wx / M;
    s->gy = p->wy / M;
    s->gz = p->wz / M;
    return s;
}

void aokb_source_destroy(aokb_source* s) { delete s; }

// Host-memory budget of the blob cache in bytes (0, the default: no cache;
// blobs still held by a handle outlive their eviction).
void aokb_source_set_cache(aokb_source* s, uint64_t bytes) {
    if (!s) return;
    std::lock_guard<std::mutex> lk(s->mu);
    s->cap = (size_t)bytes;
    s->evict_to(s->cap);
}

// [0] cache hits, [1] builds, [2] cached bytes, [3] cached blobs
void aokb_source_stats(aokb_source* s, uint64_t out[4]) {
    std::lock_guard<std::mutex> lk(s->mu);
    out[0] = s->hits;
    out[1] = s->misses;
    out[2] = s->bytes;
    out[3] = s->cache.size();
}

int aokb_source_build(void* user, int32_t cx, int32_t cy, int32_t cz, uint32_t lod, aok_chunk_blob* out,
                      void** handle) {
    aokb_source* s = (aokb_source*)user;
    if (!s || !out || !handle || cx < 0 || cy < 0 || cz < 0 || cx >= s->gx || cy >= s->gy || cz >= s->gz ||
        (int)lod >= s->L)
        return -1;
    const int64_t chunk = (int64_t)cx + s->gx * ((int64_t)cy + s->gy * (int64_t)cz);
    const int64_t key = chunk * s->L + lod;
    bool cached;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        cached = s->cap > 0;
        auto it = s->cache.find(key);
        if (it != s->cache.end()) {
            s->lru.splice(s->lru.begin(), s->lru, it->second.pos);
            s->hits++;
            auto* h = new std::shared_ptr<const Blob>(it->second.blob);
            fill_blob(**h, out);
            *handle = h;
            return 0;
        }
        s->misses++;
    }
    // without a cache only the asked LOD; with one, it and every coarser LOD
    const uint32_t mask = cached ? (0xFFu << lod) & ((1u << s->L) - 1u) : 1u << lod;
    std::vector<Blob> blobs(s->L);
    build_chunk(s->w, s->M, s->L, cx, cy, cz, blobs.data(), mask);
    auto* h = new std::shared_ptr<const Blob>(std::make_shared<const Blob>(std::move(blobs[lod])));
    if (cached) {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int l = (int)lod; l < s->L; l++) {
            const int64_t k = chunk * s->L + l;
            if (s->cache.count(k)) continue;  // another thread built it meanwhile
            std::shared_ptr<const Blob> b = l == (int)lod ? *h : std::make_shared<const Blob>(std::move(blobs[l]));
            const size_t nb = blob_bytes(*b);
            if (nb > s->cap) continue;
            s->lru.push_front(k);
            s->cache.emplace(k, aokb_source::Entry{std::move(b), nb, s->lru.begin()});
            s->bytes += nb;
        }
        s->evict_to(s->cap);
    }
    fill_blob(**h, out);
    *handle = h;
    return 0;
}

void aokb_source_release(void* user, void* handle) {
    (void)user;
    delete (std::shared_ptr<const Blob>*)handle;
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
