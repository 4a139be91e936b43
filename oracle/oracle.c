/*
 * oracle -- plain CPU reference of the chunked multi-LOD SVDAG primary-ray
 * path (Aokana, Sec. 3.2-3.5, Eq. 1).  TEST INFRASTRUCTURE ONLY: only the
 * tests, the package smoke check and the benchmark's CPU-baseline leg load it.
 * See oracle.h for the definitions and their sources.  Written for clarity:
 * dense byte grids, sort-based dedup, FP64 slab tests, recursion.
 */
#include "oracle.h"
#include <math.h>
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>

#define IDX(x, y, z, r) ((size_t)(x) + (size_t)(r) * ((size_t)(y) + (size_t)(r) * (size_t)(z)))

static int ilog2(int64_t v) { int l = 0; while (((int64_t)1 << l) < v) l++; return l; }

/* ------------------------------------------------------------------------ */
/* LOD aggregation, Sec. 3.4 (density = 2; value = rounded mean)            */
/* ------------------------------------------------------------------------ */
void or_lod_down(const uint8_t* occ, const uint8_t* mat, int32_t r, uint8_t* occ2, uint8_t* mat2) {
    int32_t h = r / 2;
    for (int32_t z = 0; z < h; z++)
        for (int32_t y = 0; y < h; y++)
            for (int32_t x = 0; x < h; x++) {
                int32_t cnt = 0, sum = 0;
                for (int32_t dz = 0; dz < 2; dz++)
                    for (int32_t dy = 0; dy < 2; dy++)
                        for (int32_t dx = 0; dx < 2; dx++) {
                            size_t i = IDX(2 * x + dx, 2 * y + dy, 2 * z + dz, r);
                            if (occ[i]) { cnt++; sum += mat[i]; }
                        }
                size_t j = IDX(x, y, z, h);
                occ2[j] = cnt >= 2;
                mat2[j] = cnt >= 2 ? (uint8_t)((sum + cnt / 2) / cnt) : 0;
            }
}

/* ------------------------------------------------------------------------ */
/* SVDAG build, Sec. 3.2: bottom-up, one dedup (sort) per level             */
/* ------------------------------------------------------------------------ */
typedef struct { uint32_t key[9]; int64_t pos; } rec_t;  /* key = mask, child ids */
static int rec_cmp(const void* a, const void* b) {
    return memcmp(((const rec_t*)a)->key, ((const rec_t*)b)->key, sizeof(uint32_t) * 9);
}
typedef struct { uint64_t m; int64_t pos; } lrec_t;
static int lrec_cmp(const void* a, const void* b) {
    uint64_t x = ((const lrec_t*)a)->m, y = ((const lrec_t*)b)->m;
    return x < y ? -1 : x > y;
}

/* depth-first material order: ascending octant, then ascending leaf bit */
static void dfs_mats(const uint8_t* occ, const uint8_t* mat, int32_t r, int32_t x0, int32_t y0, int32_t z0,
                     int32_t size, uint8_t* out, uint64_t* n) {
    if (size == 4) {
        for (int bit = 0; bit < 64; bit++) {
            int32_t x = x0 + (bit & 3), y = y0 + ((bit >> 2) & 3), z = z0 + (bit >> 4);
            size_t i = IDX(x, y, z, r);
            if (occ[i]) out[(*n)++] = mat[i];
        }
        return;
    }
    int32_t h = size / 2;
    for (int oct = 0; oct < 8; oct++)
        dfs_mats(occ, mat, r, x0 + (oct & 1) * h, y0 + ((oct >> 1) & 1) * h, z0 + ((oct >> 2) & 1) * h, h, out, n);
}

int or_dag_build(const uint8_t* occ, const uint8_t* mat, int32_t res, or_dag* g) {
    memset(g, 0, sizeof(*g));
    if (res < 8 || (res & (res - 1))) return -1;
    g->res = res;
    g->n_int = ilog2(res) - 2;
    int32_t nb = res / 4;
    size_t nblk = (size_t)nb * nb * nb;
    /* 4x4x4 leaf masks, bit x + 4y + 16z */
    uint64_t* bm = (uint64_t*)malloc(nblk * sizeof(uint64_t));
    size_t n_nonzero = 0;
    for (int32_t bz = 0; bz < nb; bz++)
        for (int32_t by = 0; by < nb; by++)
            for (int32_t bx = 0; bx < nb; bx++) {
                uint64_t m = 0;
                for (int bit = 0; bit < 64; bit++)
                    if (occ[IDX(4 * bx + (bit & 3), 4 * by + ((bit >> 2) & 3), 4 * bz + (bit >> 4), res)])
                        m |= 1ULL << bit;
                bm[IDX(bx, by, bz, nb)] = m;
                n_nonzero += m != 0;
            }
    /* unique leaves */
    lrec_t* lr = (lrec_t*)malloc((n_nonzero + 1) * sizeof(lrec_t));
    size_t k = 0;
    for (size_t i = 0; i < nblk; i++) if (bm[i]) { lr[k].m = bm[i]; lr[k].pos = (int64_t)i; k++; }
    qsort(lr, k, sizeof(lrec_t), lrec_cmp);
    int64_t* cid = (int64_t*)malloc(nblk * sizeof(int64_t));
    for (size_t i = 0; i < nblk; i++) cid[i] = -1;
    g->leaves = (uint64_t*)malloc((k + 1) * sizeof(uint64_t));
    for (size_t i = 0; i < k; i++) {
        if (i == 0 || lr[i].m != lr[i - 1].m) g->leaves[g->n_leaves++] = lr[i].m;
        cid[lr[i].pos] = (int64_t)g->n_leaves - 1;
    }
    free(lr);
    free(bm);
    g->level_nodes[g->n_int] = g->n_leaves;
    /* interior levels, deepest first */
    size_t cap = 1024, nw = 0;
    uint32_t* pool = (uint32_t*)malloc(cap * sizeof(uint32_t));
    int32_t n = nb;
    int child_is_leaf = 1;
    for (int level = g->n_int - 1; level >= 0; level--) {
        int32_t p = n / 2;
        size_t np = (size_t)p * p * p;
        rec_t* rc = (rec_t*)malloc((np + 1) * sizeof(rec_t));
        size_t nr = 0;
        int64_t* pid = (int64_t*)malloc(np * sizeof(int64_t));
        for (size_t i = 0; i < np; i++) pid[i] = -1;
        for (int32_t z = 0; z < p; z++)
            for (int32_t y = 0; y < p; y++)
                for (int32_t x = 0; x < p; x++) {
                    rec_t r;
                    memset(&r, 0xFF, sizeof(r));
                    uint32_t mask = 0, c = 0;
                    for (int oct = 0; oct < 8; oct++) {
                        int64_t ch = cid[IDX(2 * x + (oct & 1), 2 * y + ((oct >> 1) & 1), 2 * z + ((oct >> 2) & 1), n)];
                        if (ch >= 0) { mask |= 1u << oct; r.key[1 + c++] = (uint32_t)ch; }
                    }
                    if (!mask) continue;
                    r.key[0] = mask;
                    r.pos = (int64_t)IDX(x, y, z, p);
                    rc[nr++] = r;
                }
        qsort(rc, nr, sizeof(rec_t), rec_cmp);
        uint64_t uniq = 0;
        int64_t last = -1;
        for (size_t i = 0; i < nr; i++) {
            if (i == 0 || rec_cmp(&rc[i], &rc[i - 1]) != 0) {
                uint32_t mask = rc[i].key[0];
                int nc = __builtin_popcount(mask);
                while (nw + 2 + (size_t)nc > cap) { cap *= 2; pool = (uint32_t*)realloc(pool, cap * sizeof(uint32_t)); }
                uint64_t cnt = 0;
                for (int c = 0; c < nc; c++) {
                    uint32_t ch = rc[i].key[1 + c];
                    cnt += child_is_leaf ? (uint64_t)__builtin_popcountll(g->leaves[ch]) : pool[ch + 1];
                }
                last = (int64_t)nw;
                pool[nw++] = mask;
                pool[nw++] = (uint32_t)cnt;
                for (int c = 0; c < nc; c++) pool[nw++] = rc[i].key[1 + c];
                uniq++;
            }
            pid[rc[i].pos] = last;
        }
        g->level_nodes[level] = uniq;
        free(rc);
        free(cid);
        cid = pid;
        n = p;
        child_is_leaf = 0;
    }
    g->nodes = pool;
    if (cid[0] >= 0) {
        g->n_words = nw;
        g->root = (uint32_t)cid[0];
    } else {
        g->n_words = 0;
        g->root = 0;
    }
    free(cid);
    /* materials in DFS order */
    uint64_t nsolid = 0;
    size_t nv = (size_t)res * res * res;
    for (size_t i = 0; i < nv; i++) nsolid += occ[i] != 0;
    g->mats = (uint8_t*)malloc(nsolid + 1);
    g->n_mats = 0;
    if (nsolid) dfs_mats(occ, mat, res, 0, 0, 0, res, g->mats, &g->n_mats);
    return 0;
}

void or_dag_free(or_dag* g) {
    free(g->nodes);
    free(g->leaves);
    free(g->mats);
    memset(g, 0, sizeof(*g));
}

static void decode_rec(const or_dag* g, uint32_t node, int32_t x0, int32_t y0, int32_t z0, int32_t size,
                       uint8_t* occ, uint8_t* mat, uint64_t* counter) {
    uint32_t mask = g->nodes[node] & 0xFFu;
    uint32_t p = node + 2;
    int32_t h = size / 2;
    for (int oct = 0; oct < 8; oct++) {
        if (!((mask >> oct) & 1)) continue;
        uint32_t ch = g->nodes[p++];
        int32_t cx = x0 + (oct & 1) * h, cy = y0 + ((oct >> 1) & 1) * h, cz = z0 + ((oct >> 2) & 1) * h;
        if (h == 4) {
            uint64_t m = g->leaves[ch];
            for (int bit = 0; bit < 64; bit++)
                if ((m >> bit) & 1) {
                    size_t i = IDX(cx + (bit & 3), cy + ((bit >> 2) & 3), cz + (bit >> 4), g->res);
                    occ[i] = 1;
                    mat[i] = g->mats[(*counter)++];
                }
        } else {
            decode_rec(g, ch, cx, cy, cz, h, occ, mat, counter);
        }
    }
}

void or_dag_decode(const or_dag* g, uint8_t* occ, uint8_t* mat) {
    size_t nv = (size_t)g->res * g->res * g->res;
    memset(occ, 0, nv);
    memset(mat, 0, nv);
    if (!g->n_words) return;
    uint64_t counter = 0;
    decode_rec(g, g->root, 0, 0, 0, g->res, occ, mat, &counter);
}

/* Sec. 3.3: index = sum over the root path of earlier siblings' leaf counts,
 * plus the solid voxels before the hit bit inside its 4x4x4 block. */
int64_t or_dag_dfs_index(const or_dag* g, int32_t x, int32_t y, int32_t z) {
    if (!g->n_words || x < 0 || y < 0 || z < 0 || x >= g->res || y >= g->res || z >= g->res) return -1;
    uint32_t node = g->root;
    int32_t size = g->res;
    int64_t idx = 0;
    for (;;) {
        int32_t h = size / 2;
        int oct = ((x & h) ? 1 : 0) | ((y & h) ? 2 : 0) | ((z & h) ? 4 : 0);
        uint32_t mask = g->nodes[node] & 0xFFu;
        if (!((mask >> oct) & 1)) return -1;
        uint32_t p = node + 2, ch = 0;
        for (int o = 0; o < 8; o++) {
            if (!((mask >> o) & 1)) continue;
            uint32_t c = g->nodes[p++];
            if (o < oct) idx += (h == 4) ? __builtin_popcountll(g->leaves[c]) : g->nodes[c + 1];
            if (o == oct) ch = c;
        }
        if (h == 4) {
            uint64_t m = g->leaves[ch];
            int bit = (x & 3) + 4 * (y & 3) + 16 * (z & 3);
            if (!((m >> bit) & 1)) return -1;
            return idx + __builtin_popcountll(m & ((1ULL << bit) - 1));
        }
        node = ch;
        size = h;
    }
}

/* ------------------------------------------------------------------------ */
/* Colour blocks, Sec. 3.3                                                  */
/* ------------------------------------------------------------------------ */
uint64_t or_color_blocks(const uint8_t* v, uint64_t n, double e_c, uint64_t* start, uint8_t* color) {
    if (n == 0) return 0;
    const double tol = e_c * 255.0;
    uint64_t nb = 0, sum = 0, cnt = 0;
    uint8_t cur = 0;
    for (uint64_t i = 0; i < n; i++) {
        const double dist = fabs((double)v[i] - (double)cur);
        if (cnt > 0 && dist <= tol) {
            /* merge: the block's colour becomes the average of its entries */
            sum += v[i];
            cnt++;
            cur = (uint8_t)((sum + cnt / 2) / cnt);
        } else {
            /* close the current block (if any) and open one at i */
            if (cnt > 0) color[nb - 1] = cur;
            start[nb++] = i;
            sum = v[i];
            cnt = 1;
            cur = v[i];
        }
    }
    color[nb - 1] = cur;
    return nb;
}

uint8_t or_color_lookup(const uint64_t* start, const uint8_t* color, uint64_t n_blocks, uint64_t idx) {
    /* largest j with start[j] <= idx */
    uint64_t lo = 0, hi = n_blocks;
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (start[mid] <= idx) lo = mid;
        else hi = mid;
    }
    return color[lo];
}

/* ------------------------------------------------------------------------ */
/* LOD selection, Sec. 3.4, Eq. 1                                           */
/* ------------------------------------------------------------------------ */
double or_streaming_factor(int32_t H, float tan_half_fovy, double tau, int32_t M) {
    double f = (double)H / (2.0 * (double)tan_half_fovy);
    return f / (tau * (double)M);
}

int or_lod_loads(int32_t n, const int32_t b[3], int32_t M, const float o[3], double sf) {
    /* LODError = ChunkSize * SF - |ChunkCenter - Camera| <= 0, compared squared */
    double S = (double)((int64_t)M << n);
    double e2 = 0.0;
    for (int a = 0; a < 3; a++) {
        double c = (double)b[a] * S + 0.5 * S;
        double dd = c - (double)o[a];
        e2 = e2 + dd * dd;
    }
    double thr = S * sf;
    return e2 >= thr * thr;
}

void or_select_closed(int32_t gx, int32_t gy, int32_t gz, int32_t M, int32_t L,
                      const float o[3], double sf, int8_t* lod_out) {
    for (int32_t cz = 0; cz < gz; cz++)
        for (int32_t cy = 0; cy < gy; cy++)
            for (int32_t cx = 0; cx < gx; cx++) {
                int8_t sel = 0;
                for (int32_t n = L - 1; n >= 1; n--) {
                    int32_t b[3] = { cx >> n, cy >> n, cz >> n };
                    if (or_lod_loads(n, b, M, o, sf)) { sel = (int8_t)n; break; }
                }
                lod_out[(size_t)cx + (size_t)gx * ((size_t)cy + (size_t)gy * cz)] = sel;
            }
}

typedef struct { int32_t gx, gy, gz, M, L; const float* o; double sf; int8_t* out; } sel_ctx;

static void sel_rec(const sel_ctx* s, int32_t level, int32_t bx, int32_t by, int32_t bz) {
    int32_t span = 1 << level;
    if (bx * span >= s->gx || by * span >= s->gy || bz * span >= s->gz) return; /* no chunk here */
    int32_t b[3] = { bx, by, bz };
    if (level <= s->L - 1 && (level == 0 || or_lod_loads(level, b, s->M, s->o, s->sf))) {
        for (int32_t z = bz * span; z < (bz + 1) * span && z < s->gz; z++)
            for (int32_t y = by * span; y < (by + 1) * span && y < s->gy; y++)
                for (int32_t x = bx * span; x < (bx + 1) * span && x < s->gx; x++)
                    s->out[(size_t)x + (size_t)s->gx * ((size_t)y + (size_t)s->gy * z)] = (int8_t)level;
        return;
    }
    /* no LOD chunk at this octree level, or LODError > 0: subdivide */
    for (int oct = 0; oct < 8; oct++)
        sel_rec(s, level - 1, 2 * bx + (oct & 1), 2 * by + ((oct >> 1) & 1), 2 * bz + ((oct >> 2) & 1));
}

void or_select_recursive(int32_t gx, int32_t gy, int32_t gz, int32_t M, int32_t L,
                         const float o[3], double sf, int8_t* lod_out) {
    int32_t g = gx > gy ? gx : gy;
    if (gz > g) g = gz;
    int32_t T = ilog2(g);
    if (T < L - 1) T = L - 1;
    sel_ctx s = { gx, gy, gz, M, L, o, sf, lod_out };
    sel_rec(&s, T, 0, 0, 0);
}

/* ------------------------------------------------------------------------ */
/* Rays                                                                     */
/* ------------------------------------------------------------------------ */
void or_ray_dir(const or_cam* cam, int32_t px, int32_t py, float d[3]) {
    /* each statement is one IEEE binary32 operation, round to nearest */
    float fW = (float)cam->W, fH = (float)cam->H;
    float a = (float)(2 * px + 1);
    float b = a / fW;
    float c = b - 1.0f;
    float e = c * cam->tan_half_fovy;
    float aspect = fW / fH;
    float u = e * aspect;
    float a2 = (float)(2 * py + 1);
    float b2 = a2 / fH;
    float c2 = 1.0f - b2;
    float v = c2 * cam->tan_half_fovy;
    for (int i = 0; i < 3; i++) {
        float p = cam->R[3 * i + 0] * u;
        float q = cam->R[3 * i + 1] * v;
        float s = p + q;
        d[i] = s - cam->R[3 * i + 2];
    }
}

/* ------------------------------------------------------------------------ */
/* Scene: per (chunk, LOD) DAGs built on demand                             */
/* ------------------------------------------------------------------------ */
struct or_scene {
    const sg_scene* w;
    int32_t M, L, gx, gy, gz;
    double color_tol;   /* < 0: exact colour arrays */
    or_dag* dags;       /* [chunk * L + lod] */
    uint8_t* built;     /* 0: not built, 1: being built by a thread, 2: built */
    int32_t* aabb;      /* [chunk * L + lod][6] */
};

or_scene* or_scene_create(const sg_scene* world, int32_t M, int32_t L) {
    const sg_params* p = sg_get_params(world);
    if (M < 8 || (M & (M - 1)) || L < 1 || (M >> (L - 1)) < 8) return NULL;
    if (p->wx % M || p->wy % M || p->wz % M) return NULL;
    or_scene* s = (or_scene*)calloc(1, sizeof(or_scene));
    s->w = world;
    s->M = M;
    s->L = L;
    s->gx = p->wx / M;
    s->gy = p->wy / M;
    s->gz = p->wz / M;
    size_t n = (size_t)s->gx * s->gy * s->gz * L;
    s->dags = (or_dag*)calloc(n, sizeof(or_dag));
    s->built = (uint8_t*)calloc(n, 1);
    s->aabb = (int32_t*)calloc(n * 6, sizeof(int32_t));
    s->color_tol = -1.0;
    return s;
}

void or_scene_set_color_tol(or_scene* s, double e_c) { s->color_tol = e_c; }

/* Replace a DAG's colour array by what the colour-block resolve returns for
 * every DFS index. */
static void apply_color_blocks(or_dag* g, double e_c) {
    if (!g->n_mats) return;
    uint64_t* start = (uint64_t*)malloc(g->n_mats * sizeof(uint64_t));
    uint8_t* color = (uint8_t*)malloc(g->n_mats);
    uint64_t nb = or_color_blocks(g->mats, g->n_mats, e_c, start, color);
    for (uint64_t i = 0; i < g->n_mats; i++) g->mats[i] = or_color_lookup(start, color, nb, i);
    free(start);
    free(color);
}

void or_scene_destroy(or_scene* s) {
    if (!s) return;
    size_t n = (size_t)s->gx * s->gy * s->gz * s->L;
    for (size_t i = 0; i < n; i++) if (s->built[i]) or_dag_free(&s->dags[i]);
    free(s->dags);
    free(s->built);
    free(s->aabb);
    free(s);
}

void or_chunk_dense(const sg_scene* world, int32_t M, int32_t cx, int32_t cy, int32_t cz, int32_t n,
                    uint8_t* occ, uint8_t* mat) {
    size_t nv = (size_t)M * M * M;
    uint8_t* o0 = (uint8_t*)malloc(nv);
    uint8_t* m0 = (uint8_t*)malloc(nv);
    if (sg_fill_bytes(world, cx * M, cy * M, cz * M, M, M, M, o0) == 0) {
        /* no solid voxel: empty at every LOD */
        size_t r = (size_t)(M >> n);
        memset(occ, 0, r * r * r);
        memset(mat, 0, r * r * r);
        free(o0);
        free(m0);
        return;
    }
    for (int32_t z = 0; z < M; z++)
        for (int32_t y = 0; y < M; y++)
            for (int32_t x = 0; x < M; x++) {
                size_t i = IDX(x, y, z, M);
                m0[i] = o0[i] ? sg_material(world, cx * M + x, cy * M + y, cz * M + z) : 0;
            }
    int32_t r = M;
    for (int32_t k = 0; k < n; k++) {
        size_t nh = (size_t)(r / 2) * (r / 2) * (r / 2);
        uint8_t* o1 = (uint8_t*)malloc(nh);
        uint8_t* m1 = (uint8_t*)malloc(nh);
        or_lod_down(o0, m0, r, o1, m1);
        free(o0);
        free(m0);
        o0 = o1;
        m0 = m1;
        r /= 2;
    }
    memcpy(occ, o0, (size_t)r * r * r);
    memcpy(mat, m0, (size_t)r * r * r);
    free(o0);
    free(m0);
}

typedef struct {
    or_scene* s;
    int64_t* jobs;
    int64_t n_jobs;
    atomic_llong next;
} prep_ctx;

static void build_one(or_scene* s, int64_t key) {
    int32_t L = s->L, M = s->M;
    int64_t chunk = key / L;
    int32_t lod = (int32_t)(key % L);
    int32_t cx = (int32_t)(chunk % s->gx), cy = (int32_t)((chunk / s->gx) % s->gy), cz = (int32_t)(chunk / ((int64_t)s->gx * s->gy));
    int32_t r = M >> lod;
    size_t nv = (size_t)r * r * r;
    uint8_t* occ = (uint8_t*)malloc(nv);
    uint8_t* mat = (uint8_t*)malloc(nv);
    or_chunk_dense(s->w, M, cx, cy, cz, lod, occ, mat);
    or_dag_build(occ, mat, r, &s->dags[key]);
    if (s->color_tol >= 0.0) apply_color_blocks(&s->dags[key], s->color_tol);
    int32_t lo[3] = { r, r, r }, hi[3] = { -1, -1, -1 };
    for (int32_t z = 0; z < r; z++)
        for (int32_t y = 0; y < r; y++)
            for (int32_t x = 0; x < r; x++)
                if (occ[IDX(x, y, z, r)]) {
                    int32_t v[3] = { x, y, z };
                    for (int a = 0; a < 3; a++) { if (v[a] < lo[a]) lo[a] = v[a]; if (v[a] > hi[a]) hi[a] = v[a]; }
                }
    int32_t org[3] = { cx * M, cy * M, cz * M };
    int32_t* bb = &s->aabb[key * 6];
    for (int a = 0; a < 3; a++) {
        bb[a] = hi[a] >= 0 ? org[a] + (lo[a] << lod) : 0;
        bb[3 + a] = hi[a] >= 0 ? org[a] + ((hi[a] + 1) << lod) : 0;
    }
    free(occ);
    free(mat);
    __atomic_store_n(&s->built[key], (uint8_t)2, __ATOMIC_RELEASE);
}

/* Build (chunk, LOD) `key` unless it is built; a thread that finds another
 * building it waits until it is done.  Safe to call from several threads. */
static void ensure_built(or_scene* s, int64_t key) {
    if (__atomic_load_n(&s->built[key], __ATOMIC_ACQUIRE) == 2) return;
    uint8_t expect = 0;
    if (__atomic_compare_exchange_n(&s->built[key], &expect, (uint8_t)1, 0, __ATOMIC_ACQ_REL, __ATOMIC_ACQUIRE)) {
        build_one(s, key);
        return;
    }
    while (__atomic_load_n(&s->built[key], __ATOMIC_ACQUIRE) != 2) sched_yield();
}

static void* prep_worker(void* arg) {
    prep_ctx* c = (prep_ctx*)arg;
    for (;;) {
        int64_t i = atomic_fetch_add(&c->next, 1);
        if (i >= c->n_jobs) break;
        ensure_built(c->s, c->jobs[i]);
    }
    return NULL;
}

int or_scene_prepare(or_scene* s, const int8_t* lod_sel, int n_threads) {
    int64_t nc = (int64_t)s->gx * s->gy * s->gz;
    int64_t* jobs = (int64_t*)malloc((size_t)(nc + 1) * sizeof(int64_t));
    int64_t nj = 0;
    for (int64_t c = 0; c < nc; c++) {
        int l = lod_sel[c];
        if (l < 0 || l >= s->L) continue;
        int64_t key = c * s->L + l;
        if (__atomic_load_n(&s->built[key], __ATOMIC_ACQUIRE) != 2) jobs[nj++] = key;
    }
    if (n_threads < 1) n_threads = 1;
    prep_ctx ctx;
    ctx.s = s;
    ctx.jobs = jobs;
    ctx.n_jobs = nj;
    atomic_init(&ctx.next, 0);
    pthread_t th[256];
    int nt = n_threads > 256 ? 256 : n_threads;
    for (int t = 0; t < nt; t++) pthread_create(&th[t], NULL, prep_worker, &ctx);
    for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
    free(jobs);
    return 0;
}

const or_dag* or_scene_dag(const or_scene* s, int32_t chunk, int32_t lod, int32_t aabb[6]) {
    int64_t key = (int64_t)chunk * s->L + lod;
    if (__atomic_load_n(&s->built[key], __ATOMIC_ACQUIRE) != 2) return NULL;
    if (aabb) memcpy(aabb, &s->aabb[key * 6], 6 * sizeof(int32_t));
    return &s->dags[key];
}

/* ------------------------------------------------------------------------ */
/* Casting: FP64 slab tests over the exact float ray o + t d                */
/* ------------------------------------------------------------------------ */
/* closed box [lo, hi]; returns 1 and (tn, tf, entry axis) when the line meets
 * the box with tf >= 0 */
static int slab(const double o[3], const double d[3], const double lo[3], const double hi[3],
                double* tn_out, double* tf_out, int* axis_out) {
    double tn = -INFINITY, tf = INFINITY;
    int ax = -1;
    for (int a = 0; a < 3; a++) {
        if (d[a] == 0.0) {
            if (o[a] < lo[a] || o[a] > hi[a]) return 0;
        } else {
            double t1 = (lo[a] - o[a]) / d[a], t2 = (hi[a] - o[a]) / d[a];
            if (t1 > t2) { double t = t1; t1 = t2; t2 = t; }
            if (t1 > tn) { tn = t1; ax = a; }
            if (t2 < tf) tf = t2;
        }
    }
    if (tn > tf || tf < 0.0) return 0;
    *tn_out = tn;
    *tf_out = tf;
    *axis_out = ax;
    return 1;
}

static int box_slab(const double o[3], const double d[3], const int32_t lo[3], int32_t size, double grow,
                    double* tn, double* tf, int* ax) {
    double l[3], h[3];
    for (int a = 0; a < 3; a++) { l[a] = (double)lo[a] - grow; h[a] = (double)lo[a] + (double)size + grow; }
    return slab(o, d, l, h, tn, tf, ax);
}

typedef struct {
    const or_scene* s;
    const int8_t* sel;
    double o[3], d[3];
    /* best hit */
    int found;
    double bt;
    int32_t chunk, lod, axis;
    int32_t vlo[3];          /* hit voxel min corner, world LOD-0 units */
    /* ambiguity pass */
    double tseg;
    int amb, hit_valid;
    /* visit counting */
    uint32_t v_int, v_leaf;
} cast_t;

typedef struct { double tn; uint32_t child; int32_t lo[3]; } cand_t;

static void sort_cands(cand_t* c, int n) {
    for (int i = 1; i < n; i++) {
        cand_t k = c[i];
        int j = i - 1;
        while (j >= 0 && c[j].tn > k.tn) { c[j + 1] = c[j]; j--; }
        c[j + 1] = k;
    }
}

static void first_hit_node(cast_t* ct, const or_dag* g, uint32_t node, int32_t size, const int32_t lo[3],
                           int32_t vs, int32_t chunk, int32_t lod) {
    uint32_t mask = g->nodes[node] & 0xFFu;
    uint32_t p = node + 2;
    int32_t h = size / 2;
    cand_t c[8];
    int nc = 0;
    for (int oct = 0; oct < 8; oct++) {
        if (!((mask >> oct) & 1)) continue;
        uint32_t ch = g->nodes[p++];
        int32_t clo[3] = { lo[0] + (oct & 1) * h, lo[1] + ((oct >> 1) & 1) * h, lo[2] + ((oct >> 2) & 1) * h };
        double tn, tf;
        int ax;
        if (!box_slab(ct->o, ct->d, clo, h, 0.0, &tn, &tf, &ax)) continue;
        c[nc].tn = tn > 0.0 ? tn : 0.0;
        c[nc].child = ch;
        memcpy(c[nc].lo, clo, sizeof(clo));
        nc++;
    }
    sort_cands(c, nc);
    for (int i = 0; i < nc; i++) {
        if (ct->found && c[i].tn > ct->bt) break;
        if (h == 4 * vs) {
            uint64_t m = g->leaves[c[i].child];
            for (int bit = 0; bit < 64; bit++) {
                if (!((m >> bit) & 1)) continue;
                int32_t vlo[3] = { c[i].lo[0] + (bit & 3) * vs, c[i].lo[1] + ((bit >> 2) & 3) * vs,
                                   c[i].lo[2] + (bit >> 4) * vs };
                double tn, tf;
                int ax;
                if (!box_slab(ct->o, ct->d, vlo, vs, 0.0, &tn, &tf, &ax)) continue;
                double e = tn > 0.0 ? tn : 0.0;
                if (!ct->found || e < ct->bt) {
                    ct->found = 1;
                    ct->bt = e;
                    ct->chunk = chunk;
                    ct->lod = lod;
                    ct->axis = tn >= 0.0 ? ax : -1;
                    memcpy(ct->vlo, vlo, sizeof(vlo));
                }
            }
        } else {
            first_hit_node(ct, g, c[i].child, h, c[i].lo, vs, chunk, lod);
        }
    }
}

/* any solid voxel other than the hit whose eps-grown box meets [0, tseg] */
static void amb_node(cast_t* ct, const or_dag* g, uint32_t node, int32_t size, const int32_t lo[3],
                     int32_t vs, double eps) {
    uint32_t mask = g->nodes[node] & 0xFFu;
    uint32_t p = node + 2;
    int32_t h = size / 2;
    for (int oct = 0; oct < 8 && !ct->amb; oct++) {
        if (!((mask >> oct) & 1)) continue;
        uint32_t ch = g->nodes[p++];
        int32_t clo[3] = { lo[0] + (oct & 1) * h, lo[1] + ((oct >> 1) & 1) * h, lo[2] + ((oct >> 2) & 1) * h };
        double tn, tf;
        int ax;
        if (!box_slab(ct->o, ct->d, clo, h, eps, &tn, &tf, &ax) || tn > ct->tseg) continue;
        if (h == 4 * vs) {
            uint64_t m = g->leaves[ch];
            for (int bit = 0; bit < 64 && !ct->amb; bit++) {
                if (!((m >> bit) & 1)) continue;
                int32_t vlo[3] = { clo[0] + (bit & 3) * vs, clo[1] + ((bit >> 2) & 3) * vs, clo[2] + (bit >> 4) * vs };
                if (ct->hit_valid && vlo[0] == ct->vlo[0] && vlo[1] == ct->vlo[1] && vlo[2] == ct->vlo[2]) continue;
                if (box_slab(ct->o, ct->d, vlo, vs, eps, &tn, &tf, &ax) && tn <= ct->tseg) ct->amb = 1;
            }
        } else {
            amb_node(ct, g, ch, h, clo, vs, eps);
        }
    }
}

/* occupied cells met by [0, tseg]: interior visits and leaf-block visits */
static void count_node(cast_t* ct, const or_dag* g, uint32_t node, int32_t size, const int32_t lo[3], int32_t vs) {
    uint32_t mask = g->nodes[node] & 0xFFu;
    uint32_t p = node + 2;
    int32_t h = size / 2;
    for (int oct = 0; oct < 8; oct++) {
        if (!((mask >> oct) & 1)) continue;
        uint32_t ch = g->nodes[p++];
        int32_t clo[3] = { lo[0] + (oct & 1) * h, lo[1] + ((oct >> 1) & 1) * h, lo[2] + ((oct >> 2) & 1) * h };
        double tn, tf;
        int ax;
        if (!box_slab(ct->o, ct->d, clo, h, 0.0, &tn, &tf, &ax) || tn > ct->tseg) continue;
        if (h == 4 * vs) {
            ct->v_leaf++;
        } else {
            ct->v_int++;
            count_node(ct, g, ch, h, clo, vs);
        }
    }
}

typedef struct { double tn; int64_t chunk; } ccand_t;
static int ccand_cmp(const void* a, const void* b) {
    double x = ((const ccand_t*)a)->tn, y = ((const ccand_t*)b)->tn;
    return x < y ? -1 : x > y;
}

static void chunk_origin(const or_scene* s, int64_t c, int32_t org[3]) {
    org[0] = (int32_t)(c % s->gx) * s->M;
    org[1] = (int32_t)((c / s->gx) % s->gy) * s->M;
    org[2] = (int32_t)(c / ((int64_t)s->gx * s->gy)) * s->M;
}

static void cast_one(or_scene* s, const int8_t* sel, const or_cam* cam, double view_dist,
                     int32_t px, int32_t py, ccand_t* cbuf, or_result* r) {
    cast_t ct;
    memset(&ct, 0, sizeof(ct));
    ct.s = s;
    ct.sel = sel;
    float df[3];
    or_ray_dir(cam, px, py, df);
    for (int a = 0; a < 3; a++) { ct.o[a] = (double)cam->o[a]; ct.d[a] = (double)df[a]; }
    double dn = sqrt(ct.d[0] * ct.d[0] + ct.d[1] * ct.d[1] + ct.d[2] * ct.d[2]);
    double tlim = view_dist > 0.0 ? view_dist / dn : INFINITY;
    /* chunk cells met by the ray, by entry parameter (their DAGs are built
     * when the ray reaches them; empty ones are skipped there) */
    int64_t nc = (int64_t)s->gx * s->gy * s->gz, k = 0;
    for (int64_t c = 0; c < nc; c++) {
        int l = sel[c];
        if (l < 0 || l >= s->L) continue;
        int32_t org[3];
        chunk_origin(s, c, org);
        double tn, tf;
        int ax;
        if (!box_slab(ct.o, ct.d, org, s->M, 0.0, &tn, &tf, &ax)) continue;
        cbuf[k].tn = tn > 0.0 ? tn : 0.0;
        cbuf[k].chunk = c;
        k++;
    }
    qsort(cbuf, (size_t)k, sizeof(ccand_t), ccand_cmp);
    double tprune = isinf(tlim) ? INFINITY : tlim * (1.0 + 1e-3) + 1.0;
    for (int64_t i = 0; i < k; i++) {
        if (ct.found && cbuf[i].tn > ct.bt) break;
        if (cbuf[i].tn > tprune) break;
        int64_t c = cbuf[i].chunk;
        int l = sel[c];
        ensure_built(s, c * s->L + l);
        const or_dag* g = &s->dags[c * s->L + l];
        if (!g->n_words) continue;
        int32_t org[3];
        chunk_origin(s, c, org);
        first_hit_node(&ct, g, g->root, s->M, org, 1 << l, (int32_t)c, l);
    }
    int hit = ct.found && ct.bt <= tlim;
    double eps_hit = ct.found ? 1e-5 * (double)(1 << ct.lod) : 0.0;
    /* ambiguity: (a) another solid voxel within eps of [0, tseg]; every chunk
     * whose eps-grown cell meets the segment is searched */
    ct.tseg = hit ? ct.bt : tlim;
    ct.hit_valid = hit;
    for (int64_t c = 0; c < nc && !ct.amb; c++) {
        int l = sel[c];
        if (l < 0 || l >= s->L) continue;
        int32_t org[3];
        chunk_origin(s, c, org);
        double eps = 1e-5 * (double)(1 << l), tn, tf;
        int ax;
        if (!box_slab(ct.o, ct.d, org, s->M, eps, &tn, &tf, &ax) || tn > ct.tseg) continue;
        ensure_built(s, c * s->L + l);
        const or_dag* g = &s->dags[c * s->L + l];
        if (!g->n_words) continue;
        amb_node(&ct, g, g->root, s->M, org, 1 << l, eps);
    }
    if (hit) {
        /* (b) the ray must meet the hit voxel shrunk by eps */
        double tn, tf;
        int ax;
        double lo[3], hi[3];
        int32_t vs = 1 << ct.lod;
        for (int a = 0; a < 3; a++) { lo[a] = ct.vlo[a] + eps_hit; hi[a] = ct.vlo[a] + vs - eps_hit; }
        if (!slab(ct.o, ct.d, lo, hi, &tn, &tf, &ax)) ct.amb = 1;
    }
    /* (c) hit distance within eps of the view distance */
    if (ct.found && view_dist > 0.0 && fabs(ct.bt * dn - view_dist) < eps_hit) ct.amb = 1;
    /* visits along [0, tseg], chunks entered through their valid-voxel AABB */
    for (int64_t i = 0; i < k; i++) {
        if (cbuf[i].tn > ct.tseg) break;
        int64_t c = cbuf[i].chunk;
        int l = sel[c];
        int64_t key = c * s->L + l;
        ensure_built(s, key);
        const or_dag* g = &s->dags[key];
        if (!g->n_words) continue;
        const int32_t* bb = &s->aabb[key * 6];
        double blo[3], bhi[3], tn, tf;
        int ax;
        for (int a = 0; a < 3; a++) { blo[a] = bb[a]; bhi[a] = bb[3 + a]; }
        if (!slab(ct.o, ct.d, blo, bhi, &tn, &tf, &ax) || tn > ct.tseg) continue;
        int32_t org[3];
        chunk_origin(s, c, org);
        ct.v_int++;
        count_node(&ct, g, g->root, s->M, org, 1 << l);
    }
    r->v_int = ct.v_int;
    r->v_leaf = ct.v_leaf;
    r->amb = ct.amb;
    r->pad = 0;
    if (!hit) {
        r->x = r->y = r->z = 0;
        r->lod = 255;
        r->mat = 0;
        r->normal = 7;
        r->hit = 0;
        r->dist = INFINITY;
        r->resolve_bytes = 0;
        return;
    }
    r->x = ct.vlo[0];
    r->y = ct.vlo[1];
    r->z = ct.vlo[2];
    r->lod = ct.lod;
    r->hit = 1;
    r->dist = ct.bt * dn;
    r->normal = ct.axis < 0 ? 7 : 2 * ct.axis + (ct.d[ct.axis] < 0.0 ? 1 : 0);
    /* material through the DFS index (Sec. 3.3 / colour resolve, Sec. 3.5) */
    const or_dag* g = &s->dags[(int64_t)ct.chunk * s->L + ct.lod];
    int32_t org[3];
    chunk_origin(s, ct.chunk, org);
    int32_t lx = (ct.vlo[0] - org[0]) >> ct.lod, ly = (ct.vlo[1] - org[1]) >> ct.lod, lz = (ct.vlo[2] - org[2]) >> ct.lod;
    int64_t idx = or_dag_dfs_index(g, lx, ly, lz);
    r->mat = idx >= 0 ? g->mats[idx] : -1;
    /* resolve bytes: earlier siblings' counts on the path (4 B node count, 8 B leaf mask) + 1 B */
    uint32_t rb = 1, node = g->root;
    int32_t size = g->res;
    for (;;) {
        int32_t h = size / 2;
        int oct = ((lx & h) ? 1 : 0) | ((ly & h) ? 2 : 0) | ((lz & h) ? 4 : 0);
        uint32_t mask = g->nodes[node] & 0xFFu;
        rb += (uint32_t)__builtin_popcount(mask & ((1u << oct) - 1)) * (h == 4 ? 8u : 4u);
        if (h == 4) break;
        node = g->nodes[node + 2 + __builtin_popcount(mask & ((1u << oct) - 1))];
        size = h;
    }
    r->resolve_bytes = rb;
}

typedef struct {
    or_scene* s;
    const int8_t* sel;
    const or_cam* cam;
    double vd;
    const int32_t* pix;
    int64_t n;
    or_result* out;
    atomic_llong next;
    /* brute mode */
    int brute;
    const sg_scene* world;
    int32_t M, L, gx, gy, gz;
    uint8_t** docc;
    uint8_t** dmat;
} cast_ctx;

static void brute_one(const cast_ctx* c, int32_t px, int32_t py, or_result* r);

static void* cast_worker(void* arg) {
    cast_ctx* c = (cast_ctx*)arg;
    ccand_t* cbuf = NULL;
    if (!c->brute) cbuf = (ccand_t*)malloc(((size_t)c->s->gx * c->s->gy * c->s->gz + 1) * sizeof(ccand_t));
    for (;;) {
        int64_t i0 = atomic_fetch_add(&c->next, 16);
        if (i0 >= c->n) break;
        int64_t i1 = i0 + 16 < c->n ? i0 + 16 : c->n;
        for (int64_t i = i0; i < i1; i++) {
            if (c->brute) brute_one(c, c->pix[2 * i], c->pix[2 * i + 1], &c->out[i]);
            else cast_one(c->s, c->sel, c->cam, c->vd, c->pix[2 * i], c->pix[2 * i + 1], cbuf, &c->out[i]);
        }
    }
    free(cbuf);
    return NULL;
}

static void run_threads(cast_ctx* c, int n_threads) {
    atomic_init(&c->next, 0);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, cast_worker, c);
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
}

int or_cast(or_scene* s, const int8_t* lod_sel, const or_cam* cam, double view_dist,
            const int32_t* pix, int64_t n, or_result* out, int n_threads) {
    cast_ctx c;
    memset(&c, 0, sizeof(c));
    c.s = s;
    c.sel = lod_sel;
    c.cam = cam;
    c.vd = view_dist;
    c.pix = pix;
    c.n = n;
    c.out = out;
    run_threads(&c, n_threads);
    return 0;
}

/* ---- brute force: every voxel of every chunk's dense LOD grid ----------- */
static void brute_one(const cast_ctx* c, int32_t px, int32_t py, or_result* r) {
    float df[3];
    or_ray_dir(c->cam, px, py, df);
    double o[3], d[3];
    for (int a = 0; a < 3; a++) { o[a] = (double)c->cam->o[a]; d[a] = (double)df[a]; }
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double tlim = c->vd > 0.0 ? c->vd / dn : INFINITY;
    int64_t nc = (int64_t)c->gx * c->gy * c->gz;
    int found = 0, axis = -1;
    double bt = 0.0;
    int32_t blo[3] = { 0, 0, 0 }, blod = 0, bmat = 0;
    for (int pass = 0; pass < 2; pass++) {
        for (int64_t ch = 0; ch < nc; ch++) {
            int l = c->sel[ch];
            if (l < 0 || l >= c->L) continue;
            int32_t r0 = c->M >> l, vs = 1 << l;
            int32_t org[3] = { (int32_t)(ch % c->gx) * c->M, (int32_t)((ch / c->gx) % c->gy) * c->M,
                               (int32_t)(ch / ((int64_t)c->gx * c->gy)) * c->M };
            const uint8_t* occ = c->docc[ch];
            double eps = 1e-5 * vs;
            for (int32_t z = 0; z < r0; z++)
                for (int32_t y = 0; y < r0; y++)
                    for (int32_t x = 0; x < r0; x++) {
                        size_t i = IDX(x, y, z, r0);
                        if (!occ[i]) continue;
                        int32_t vlo[3] = { org[0] + x * vs, org[1] + y * vs, org[2] + z * vs };
                        double tn, tf;
                        int ax;
                        if (pass == 0) {
                            if (!box_slab(o, d, vlo, vs, 0.0, &tn, &tf, &ax)) continue;
                            double e = tn > 0.0 ? tn : 0.0;
                            if (!found || e < bt) {
                                found = 1; bt = e; axis = tn >= 0.0 ? ax : -1;
                                memcpy(blo, vlo, sizeof(vlo)); blod = l; bmat = c->dmat[ch][i];
                            }
                        } else {
                            if (found && bt <= tlim && vlo[0] == blo[0] && vlo[1] == blo[1] && vlo[2] == blo[2]) continue;
                            double tseg = (found && bt <= tlim) ? bt : tlim;
                            if (box_slab(o, d, vlo, vs, eps, &tn, &tf, &ax) && tn <= tseg) r->amb = 1;
                        }
                    }
        }
        if (pass == 0) r->amb = 0;
    }
    int hit = found && bt <= tlim;
    if (hit) {
        double eps = 1e-5 * (1 << blod), lo[3], hi[3], tn, tf;
        int ax;
        for (int a = 0; a < 3; a++) { lo[a] = blo[a] + eps; hi[a] = blo[a] + (1 << blod) - eps; }
        if (!slab(o, d, lo, hi, &tn, &tf, &ax)) r->amb = 1;
    }
    if (found && c->vd > 0.0 && fabs(bt * dn - c->vd) < 1e-5 * (1 << blod)) r->amb = 1;
    r->v_int = r->v_leaf = r->resolve_bytes = r->pad = 0;
    if (!hit) {
        r->x = r->y = r->z = 0; r->lod = 255; r->mat = 0; r->normal = 7; r->hit = 0; r->dist = INFINITY;
        return;
    }
    r->x = blo[0]; r->y = blo[1]; r->z = blo[2];
    r->lod = blod; r->mat = bmat; r->hit = 1; r->dist = bt * dn;
    r->normal = axis < 0 ? 7 : 2 * axis + (d[axis] < 0.0 ? 1 : 0);
}

int or_cast_brute(const sg_scene* world, int32_t M, int32_t L, const int8_t* lod_sel,
                  const or_cam* cam, double view_dist, const int32_t* pix, int64_t n,
                  or_result* out, int n_threads) {
    const sg_params* p = sg_get_params(world);
    cast_ctx c;
    memset(&c, 0, sizeof(c));
    c.brute = 1;
    c.world = world;
    c.M = M;
    c.L = L;
    c.gx = p->wx / M;
    c.gy = p->wy / M;
    c.gz = p->wz / M;
    c.sel = lod_sel;
    c.cam = cam;
    c.vd = view_dist;
    c.pix = pix;
    c.n = n;
    c.out = out;
    int64_t nc = (int64_t)c.gx * c.gy * c.gz;
    c.docc = (uint8_t**)calloc((size_t)nc, sizeof(uint8_t*));
    c.dmat = (uint8_t**)calloc((size_t)nc, sizeof(uint8_t*));
    for (int64_t ch = 0; ch < nc; ch++) {
        int l = lod_sel[ch];
        if (l < 0 || l >= L) continue;
        int32_t r0 = M >> l;
        c.docc[ch] = (uint8_t*)malloc((size_t)r0 * r0 * r0);
        c.dmat[ch] = (uint8_t*)malloc((size_t)r0 * r0 * r0);
        or_chunk_dense(world, M, (int32_t)(ch % c.gx), (int32_t)((ch / c.gx) % c.gy),
                       (int32_t)(ch / ((int64_t)c.gx * c.gy)), l, c.docc[ch], c.dmat[ch]);
    }
    run_threads(&c, n_threads);
    for (int64_t ch = 0; ch < nc; ch++) { free(c.docc[ch]); free(c.dmat[ch]); }
    free(c.docc);
    free(c.dmat);
    return 0;
}
