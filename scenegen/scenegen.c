/*
 * scenegen -- seeded synthetic voxel-world generator (input data only).
 * See scenegen.h for the world model.  Integer arithmetic only.
 */
#include "scenegen.h"
#include <stdlib.h>
#include <string.h>

#define BIN 256  /* box bin size over (x, y) */

struct sg_scene {
    sg_params p;
    uint64_t noise_seed, mat_seed;
    sg_box* boxes;
    int32_t nbx, nby;        /* bins over (x, y) */
    int32_t* bin_start;      /* CSR: nbx*nby + 1 */
    int32_t* bin_items;      /* box indices */
};

uint64_t sg_mix64(uint64_t z) {
    /* SplitMix64 output function (Steele, Lea, Flood 2014). */
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s; } rng_t;
static uint64_t rng_next(rng_t* r) { r->s += 0x9E3779B97F4A7C15ULL; return sg_mix64(r->s); }
static int32_t rng_uniform(rng_t* r, int32_t a, int32_t b) {  /* inclusive */
    if (b <= a) return a;
    return a + (int32_t)(rng_next(r) % (uint64_t)(b - a + 1));
}

static int32_t floor_div(int32_t x, int32_t p) { return x >= 0 ? x / p : -((-x + p - 1) / p); }

static uint32_t lattice(const sg_scene* s, int32_t i, int32_t j, int32_t o) {
    uint64_t k = sg_mix64((uint64_t)(uint32_t)i ^ ((uint64_t)(uint32_t)j << 32));
    return (uint32_t)(sg_mix64(k ^ (s->noise_seed + (uint64_t)(o + 1) * 0x9E3779B97F4A7C15ULL)) & 0xFFFFu);
}

static int64_t smooth_q16(int64_t t) {  /* t in [0, 65536): t^2 (3 - 2t) in Q16 */
    int64_t t2 = (t * t) >> 16;
    return (t2 * (3 * 65536 - 2 * t)) >> 16;
}

int32_t sg_height(const sg_scene* s, int32_t x, int32_t y) {
    const sg_params* p = &s->p;
    int64_t total = 0, wsum = 0;
    int32_t K = p->octaves - 1;
    for (int32_t o = 0; o < p->octaves; o++) {
        int32_t P = p->period0 >> o;
        if (P < 1) P = 1;
        int32_t i = floor_div(x, P), j = floor_div(y, P);
        int64_t fx = (int64_t)(x - i * P), fy = (int64_t)(y - j * P);
        int64_t tx = (fx << 16) / P, ty = (fy << 16) / P;
        int64_t sx = smooth_q16(tx), sy = smooth_q16(ty);
        int64_t v00 = lattice(s, i, j, o), v10 = lattice(s, i + 1, j, o);
        int64_t v01 = lattice(s, i, j + 1, o), v11 = lattice(s, i + 1, j + 1, o);
        int64_t a = (v00 * (65536 - sx) + v10 * sx) >> 16;
        int64_t b = (v01 * (65536 - sx) + v11 * sx) >> 16;
        int64_t n = (a * (65536 - sy) + b * sy) >> 16;
        total += n << (K - o);
        wsum += (int64_t)1 << (K - o);
    }
    int64_t nq = total / wsum; /* [0, 65535] */
    return p->h_min + (int32_t)(((int64_t)(p->h_max - p->h_min) * nq) >> 16);
}

/* Same values as sg_height over a rectangle, with the per-octave lattice values
 * and interpolation weights computed once per cell / column / row. */
void sg_heights(const sg_scene* s, int32_t x0, int32_t y0, int32_t nx, int32_t ny, int32_t* out) {
    const sg_params* p = &s->p;
    const int32_t K = p->octaves - 1;
    int64_t* acc = (int64_t*)calloc((size_t)nx * ny, sizeof(int64_t));
    int32_t* ix = (int32_t*)malloc((size_t)nx * sizeof(int32_t));
    int32_t* iy = (int32_t*)malloc((size_t)ny * sizeof(int32_t));
    int64_t* sx = (int64_t*)malloc((size_t)nx * sizeof(int64_t));
    int64_t* sy = (int64_t*)malloc((size_t)ny * sizeof(int64_t));
    int64_t* ta = (int64_t*)malloc((size_t)nx * sizeof(int64_t));
    int64_t* tb = (int64_t*)malloc((size_t)nx * sizeof(int64_t));
    for (int32_t o = 0; o < p->octaves; o++) {
        int32_t P = p->period0 >> o;
        if (P < 1) P = 1;
        for (int32_t x = 0; x < nx; x++) {
            const int32_t i = floor_div(x0 + x, P);
            ix[x] = i;
            sx[x] = smooth_q16(((int64_t)(x0 + x - i * P) << 16) / P);
        }
        for (int32_t y = 0; y < ny; y++) {
            const int32_t j = floor_div(y0 + y, P);
            iy[y] = j;
            sy[y] = smooth_q16(((int64_t)(y0 + y - j * P) << 16) / P);
        }
        const int32_t i0 = ix[0], j0 = iy[0];
        const int32_t ci = ix[nx - 1] - i0 + 2, cj = iy[ny - 1] - j0 + 2;
        int64_t* lat = (int64_t*)malloc((size_t)ci * cj * sizeof(int64_t));
        for (int32_t j = 0; j < cj; j++)
            for (int32_t i = 0; i < ci; i++) lat[(size_t)j * ci + i] = lattice(s, i0 + i, j0 + j, o);
        for (int32_t y = 0; y < ny; y++) {
            if (y == 0 || iy[y] != iy[y - 1]) {
                /* the x interpolation of this lattice row pair, shared by the rows up to the next pair */
                const int64_t* r0 = lat + (size_t)(iy[y] - j0) * ci;
                const int64_t* r1 = r0 + ci;
                for (int32_t x = 0; x < nx; x++) {
                    const int32_t c = ix[x] - i0;
                    const int64_t wx = sx[x];
                    ta[x] = (r0[c] * (65536 - wx) + r0[c + 1] * wx) >> 16;
                    tb[x] = (r1[c] * (65536 - wx) + r1[c + 1] * wx) >> 16;
                }
            }
            const int64_t wy = sy[y];
            int64_t* a = acc + (size_t)y * nx;
            for (int32_t x = 0; x < nx; x++) a[x] += ((ta[x] * (65536 - wy) + tb[x] * wy) >> 16) << (K - o);
        }
        free(lat);
    }
    /* the weight sum is 2^octaves - 1; a literal divisor per case lets the
     * compiler divide by multiplication (the same quotients) */
    const size_t n = (size_t)nx * ny;
    const int64_t span = (int64_t)(p->h_max - p->h_min);
#define SG_HEIGHTS_OUT(d) \
    for (size_t k = 0; k < n; k++) out[k] = p->h_min + (int32_t)((span * (acc[k] / (d))) >> 16); \
    break;
    switch (p->octaves) {
    case 1: SG_HEIGHTS_OUT(1)
    case 2: SG_HEIGHTS_OUT(3)
    case 3: SG_HEIGHTS_OUT(7)
    case 4: SG_HEIGHTS_OUT(15)
    case 5: SG_HEIGHTS_OUT(31)
    case 6: SG_HEIGHTS_OUT(63)
    case 7: SG_HEIGHTS_OUT(127)
    case 8: SG_HEIGHTS_OUT(255)
    case 9: SG_HEIGHTS_OUT(511)
    case 10: SG_HEIGHTS_OUT(1023)
    case 11: SG_HEIGHTS_OUT(2047)
    case 12: SG_HEIGHTS_OUT(4095)
    case 13: SG_HEIGHTS_OUT(8191)
    case 14: SG_HEIGHTS_OUT(16383)
    case 15: SG_HEIGHTS_OUT(32767)
    default: SG_HEIGHTS_OUT(65535)
    }
#undef SG_HEIGHTS_OUT
    free(acc);
    free(ta);
    free(tb);
    free(ix);
    free(iy);
    free(sx);
    free(sy);
}

const sg_params* sg_get_params(const sg_scene* s) { return &s->p; }
int32_t sg_num_boxes(const sg_scene* s) { return s->p.n_boxes; }
void sg_get_box(const sg_scene* s, int32_t i, sg_box* out) { *out = s->boxes[i]; }

static sg_scene* create(const sg_params* p, const sg_box* given) {
    if (!p || p->wx <= 0 || p->wy <= 0 || p->wz <= 0 || p->octaves < 1 || p->octaves > 16 ||
        p->period0 < 1 || p->h_max < p->h_min || p->n_boxes < 0 || p->crust < 0 || p->mat_mode < 0 ||
        p->mat_mode > 1)
        return NULL;
    if (given) {
        for (int32_t b = 0; b < p->n_boxes; b++) {
            const sg_box* g = &given[b];
            if (g->sx < 1 || g->sy < 1 || g->sz < 1 || g->x0 < 0 || g->y0 < 0 || g->z0 < 0 ||
                g->x0 + g->sx > p->wx || g->y0 + g->sy > p->wy || g->z0 + g->sz > p->wz)
                return NULL;
        }
    }
    sg_scene* s = (sg_scene*)calloc(1, sizeof(sg_scene));
    s->p = *p;
    s->noise_seed = sg_mix64(p->seed ^ 0x6E6F697365ULL);
    s->mat_seed = sg_mix64(p->seed ^ 0x6D6174ULL);
    s->boxes = (sg_box*)calloc((size_t)(p->n_boxes > 0 ? p->n_boxes : 1), sizeof(sg_box));
    rng_t r = { sg_mix64(p->seed ^ 0x626F786573ULL) };
    for (int32_t b = 0; b < p->n_boxes && given; b++) s->boxes[b] = given[b];
    for (int32_t b = 0; b < p->n_boxes && !given; b++) {
        sg_box* bx = &s->boxes[b];
        bx->sx = rng_uniform(&r, p->box_min, p->box_max);
        bx->sy = rng_uniform(&r, p->box_min, p->box_max);
        bx->sz = rng_uniform(&r, p->box_min, p->box_max);
        if (bx->sx > p->wx) bx->sx = p->wx;
        if (bx->sy > p->wy) bx->sy = p->wy;
        if (bx->sz > p->wz) bx->sz = p->wz;
        bx->x0 = rng_uniform(&r, 0, p->wx - bx->sx);
        bx->y0 = rng_uniform(&r, 0, p->wy - bx->sy);
        if (p->box_hollow) {
            /* city block standing on the terrain at its centre, sunk one voxel */
            int32_t z0 = sg_height(s, bx->x0 + bx->sx / 2, bx->y0 + bx->sy / 2) - 1;
            if (z0 < 0) z0 = 0;
            if (z0 > p->wz - bx->sz) z0 = p->wz - bx->sz;
            bx->z0 = z0;
            bx->hollow = 1;
        } else {
            bx->z0 = rng_uniform(&r, 0, p->wz - bx->sz);
            bx->hollow = 0;
        }
    }
    /* bin boxes over (x, y) */
    s->nbx = (p->wx + BIN - 1) / BIN;
    s->nby = (p->wy + BIN - 1) / BIN;
    size_t nb = (size_t)s->nbx * s->nby;
    s->bin_start = (int32_t*)calloc(nb + 1, sizeof(int32_t));
    for (int pass = 0; pass < 2; pass++) {
        int32_t* fill = pass ? (int32_t*)calloc(nb, sizeof(int32_t)) : NULL;
        for (int32_t b = 0; b < p->n_boxes; b++) {
            const sg_box* bx = &s->boxes[b];
            int32_t bx0 = bx->x0 / BIN, bx1 = (bx->x0 + bx->sx - 1) / BIN;
            int32_t by0 = bx->y0 / BIN, by1 = (bx->y0 + bx->sy - 1) / BIN;
            for (int32_t j = by0; j <= by1; j++)
                for (int32_t i = bx0; i <= bx1; i++) {
                    size_t k = (size_t)j * s->nbx + i;
                    if (!pass) s->bin_start[k + 1]++;
                    else s->bin_items[s->bin_start[k] + fill[k]++] = b;
                }
        }
        if (!pass) {
            for (size_t k = 0; k < nb; k++) s->bin_start[k + 1] += s->bin_start[k];
            s->bin_items = (int32_t*)calloc((size_t)s->bin_start[nb] + 1, sizeof(int32_t));
        } else {
            free(fill);
        }
    }
    return s;
}

sg_scene* sg_create(const sg_params* p) { return create(p, NULL); }

sg_scene* sg_create_with_boxes(const sg_params* p, const sg_box* boxes) { return boxes ? create(p, boxes) : NULL; }

void sg_destroy(sg_scene* s) {
    if (!s) return;
    free(s->boxes);
    free(s->bin_start);
    free(s->bin_items);
    free(s);
}

static int in_box(const sg_box* b, int32_t x, int32_t y, int32_t z) {
    if (x < b->x0 || y < b->y0 || z < b->z0) return 0;
    if (x >= b->x0 + b->sx || y >= b->y0 + b->sy || z >= b->z0 + b->sz) return 0;
    if (!b->hollow) return 1;
    return x == b->x0 || y == b->y0 || z == b->z0 ||
           x == b->x0 + b->sx - 1 || y == b->y0 + b->sy - 1 || z == b->z0 + b->sz - 1;
}

static int32_t crust_lo(const sg_scene* s, int32_t x, int32_t y, int32_t h) {
    int32_t m = h, t;
    t = sg_height(s, x - 1, y); if (t < m) m = t;
    t = sg_height(s, x + 1, y); if (t < m) m = t;
    t = sg_height(s, x, y - 1); if (t < m) m = t;
    t = sg_height(s, x, y + 1); if (t < m) m = t;
    m -= s->p.crust;
    return m < 0 ? 0 : m;
}

int sg_solid(const sg_scene* s, int32_t x, int32_t y, int32_t z) {
    const sg_params* p = &s->p;
    if (x < 0 || y < 0 || z < 0 || x >= p->wx || y >= p->wy || z >= p->wz) return 0;
    int32_t h = sg_height(s, x, y);
    if (z < h) {
        if (p->crust == 0) return 1;
        if (z >= crust_lo(s, x, y, h)) return 1;
    }
    size_t k = (size_t)(y / BIN) * s->nbx + (size_t)(x / BIN);
    for (int32_t i = s->bin_start[k]; i < s->bin_start[k + 1]; i++)
        if (in_box(&s->boxes[s->bin_items[i]], x, y, z)) return 1;
    return 0;
}

static inline uint8_t material_at(const sg_scene* s, int32_t x, int32_t y, int32_t z) {
    uint64_t key = ((uint64_t)(uint32_t)x & 0x1FFFFFULL) | (((uint64_t)(uint32_t)y & 0x1FFFFFULL) << 21) |
                   (((uint64_t)(uint32_t)z & 0x1FFFFFULL) << 42);
    const uint64_t h = sg_mix64(key ^ s->mat_seed);
    if (s->p.mat_mode == 0) return (uint8_t)(h & 0xFFu);
    if ((h & 63u) == 0) return (uint8_t)((h >> 8) & 0xFFu);
    const uint32_t stratum = (uint32_t)z >> 3;
    const uint32_t cell = (((uint32_t)x >> 6) * 7u + ((uint32_t)y >> 6) * 13u) & 31u;
    return (uint8_t)((stratum * 5u + cell * 3u + (uint32_t)(s->mat_seed & 63u)) & 0xFFu);
}

uint8_t sg_material(const sg_scene* s, int32_t x, int32_t y, int32_t z) { return material_at(s, x, y, z); }

void sg_materials_block4(const sg_scene* s, int32_t x0, int32_t y0, int32_t z0, uint64_t mask, uint8_t* out) {
    while (mask) {
        const int b = __builtin_ctzll(mask);
        mask &= mask - 1;
        out[b] = material_at(s, x0 + (b & 3), y0 + ((b >> 2) & 3), z0 + (b >> 4));
    }
}

void sg_materials(const sg_scene* s, const int32_t* xyz, size_t n, uint8_t* out) {
    for (size_t i = 0; i < n; i++) out[i] = sg_material(s, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]);
}

/* ---- dense fills ------------------------------------------------------- */

typedef struct {
    uint8_t* bytes; uint64_t* bits;
    int32_t x0, y0, z0, nx, ny, nz;
    int32_t zlo, zhi;  /* world z range of the rows written (zlo >= zhi: none) */
} region_t;

static inline void touch_z(region_t* r, int32_t z0, int32_t z1) {
    if (z0 >= z1) return;
    if (z0 < r->zlo) r->zlo = z0;
    if (z1 > r->zhi) r->zhi = z1;
}

static inline void set_voxel(region_t* r, int32_t x, int32_t y, int32_t z) {
    /* region-local coordinates, already clipped */
    size_t row = (size_t)y + (size_t)r->ny * (size_t)z;
    if (r->bytes) r->bytes[(size_t)x + (size_t)r->nx * row] = 1;
    else r->bits[(size_t)(x >> 6) + (size_t)(r->nx >> 6) * row] |= 1ULL << (x & 63);
}

static void fill_region(const sg_scene* s, region_t* r) {
    const sg_params* p = &s->p;
    /* world-clipped region */
    int32_t ax0 = r->x0 < 0 ? 0 : r->x0, ay0 = r->y0 < 0 ? 0 : r->y0, az0 = r->z0 < 0 ? 0 : r->z0;
    int32_t ax1 = r->x0 + r->nx, ay1 = r->y0 + r->ny, az1 = r->z0 + r->nz;
    if (ax1 > p->wx) ax1 = p->wx;
    if (ay1 > p->wy) ay1 = p->wy;
    if (az1 > p->wz) az1 = p->wz;
    if (ax0 >= ax1 || ay0 >= ay1 || az0 >= az1) return;
    /* terrain: heights with a one-voxel border for the crust rule */
    int32_t hx = ax1 - ax0 + 2, hy = ay1 - ay0 + 2;
    int32_t* h = (int32_t*)malloc((size_t)hx * hy * sizeof(int32_t));
    sg_heights(s, ax0 - 1, ay0 - 1, hx, hy, h);
    /* per row y and 64-column word of the bit layout: each column's first and
     * one-past-last solid z are marked in ev[] and a running XOR over z gives
     * the word of every row (bytes: one voxel at a time) */
    uint64_t* ev = r->bits ? (uint64_t*)calloc((size_t)(az1 - az0 + 1), sizeof(uint64_t)) : NULL;
    const int32_t w64 = r->nx >> 6;
    for (int32_t y = ay0; y < ay1; y++) {
        int32_t x = ax0;
        while (x < ax1) {
            /* columns [x, xe): one word of the bit layout */
            const int32_t xe0 = r->x0 + (((x - r->x0) >> 6) + 1) * 64;
            const int32_t xe = r->bits && xe0 < ax1 ? xe0 : ax1;
            int32_t zmn = az1, zmx = az0;
            for (; x < xe; x++) {
                size_t c = (size_t)(y - ay0 + 1) * hx + (size_t)(x - ax0 + 1);
                int32_t top = h[c];
                int32_t lo = 0;
                if (p->crust > 0) {
                    int32_t m = top;
                    if (h[c - 1] < m) m = h[c - 1];
                    if (h[c + 1] < m) m = h[c + 1];
                    if (h[c - hx] < m) m = h[c - hx];
                    if (h[c + hx] < m) m = h[c + hx];
                    lo = m - p->crust;
                    if (lo < 0) lo = 0;
                }
                int32_t z0 = lo > az0 ? lo : az0, z1 = top < az1 ? top : az1;
                if (z0 >= z1) continue;
                touch_z(r, z0, z1);
                if (!r->bits) {
                    for (int32_t z = z0; z < z1; z++) set_voxel(r, x - r->x0, y - r->y0, z - r->z0);
                    continue;
                }
                const uint64_t bit = 1ULL << ((x - r->x0) & 63);
                ev[z0 - az0] ^= bit;
                ev[z1 - az0] ^= bit;
                if (z0 < zmn) zmn = z0;
                if (z1 > zmx) zmx = z1;
            }
            if (zmn >= zmx) continue;
            /* x - 1 is the word's last column */
            uint64_t* col = r->bits + (size_t)((x - 1 - r->x0) >> 6) + (size_t)w64 * (size_t)(y - r->y0);
            const size_t zstride = (size_t)w64 * (size_t)r->ny;
            uint64_t cur = 0;
            for (int32_t z = zmn; z < zmx; z++) {
                cur ^= ev[z - az0];
                ev[z - az0] = 0;
                col[zstride * (size_t)(z - r->z0)] |= cur;
            }
            ev[zmx - az0] = 0;
        }
    }
    free(ev);
    free(h);
    /* boxes: visit each box overlapping the region once */
    int32_t bi0 = ax0 / BIN, bi1 = (ax1 - 1) / BIN, bj0 = ay0 / BIN, bj1 = (ay1 - 1) / BIN;
    for (int32_t bj = bj0; bj <= bj1; bj++)
        for (int32_t bi = bi0; bi <= bi1; bi++) {
            size_t k = (size_t)bj * s->nbx + bi;
            for (int32_t it = s->bin_start[k]; it < s->bin_start[k + 1]; it++) {
                const sg_box* b = &s->boxes[s->bin_items[it]];
                /* the box is visited from its first bin overlapping the region only */
                int32_t fbi = b->x0 / BIN, fbj = b->y0 / BIN;
                if (fbi < bi0) fbi = bi0;
                if (fbj < bj0) fbj = bj0;
                if (fbi != bi || fbj != bj) continue;
                int32_t x0 = b->x0 > ax0 ? b->x0 : ax0, x1 = b->x0 + b->sx < ax1 ? b->x0 + b->sx : ax1;
                int32_t y0 = b->y0 > ay0 ? b->y0 : ay0, y1 = b->y0 + b->sy < ay1 ? b->y0 + b->sy : ay1;
                int32_t z0 = b->z0 > az0 ? b->z0 : az0, z1 = b->z0 + b->sz < az1 ? b->z0 + b->sz : az1;
                for (int32_t z = z0; z < z1; z++)
                    for (int32_t y = y0; y < y1; y++) {
                        int shell_row = !b->hollow || z == b->z0 || z == b->z0 + b->sz - 1 ||
                                        y == b->y0 || y == b->y0 + b->sy - 1;
                        if (shell_row) {
                            if (x0 < x1) touch_z(r, z, z + 1);
                            for (int32_t x = x0; x < x1; x++) set_voxel(r, x - r->x0, y - r->y0, z - r->z0);
                        } else {
                            int32_t xe = b->x0 + b->sx - 1;
                            if (b->x0 >= x0 && b->x0 < x1) {
                                touch_z(r, z, z + 1);
                                set_voxel(r, b->x0 - r->x0, y - r->y0, z - r->z0);
                            }
                            if (xe >= x0 && xe < x1) {
                                touch_z(r, z, z + 1);
                                set_voxel(r, xe - r->x0, y - r->y0, z - r->z0);
                            }
                        }
                    }
            }
        }
}

uint64_t sg_fill_bytes(const sg_scene* s, int32_t x0, int32_t y0, int32_t z0,
                       int32_t nx, int32_t ny, int32_t nz, uint8_t* out) {
    size_t n = (size_t)nx * ny * nz;
    memset(out, 0, n);
    region_t r = { out, NULL, x0, y0, z0, nx, ny, nz, 0, 0 };
    fill_region(s, &r);
    uint64_t cnt = 0;
    for (size_t i = 0; i < n; i++) cnt += out[i];
    return cnt;
}

uint64_t sg_fill_bits(const sg_scene* s, int32_t x0, int32_t y0, int32_t z0,
                      int32_t nx, int32_t ny, int32_t nz, uint64_t* out) {
    if (nx % 64) return 0;
    size_t nw = (size_t)(nx / 64) * ny * nz;
    memset(out, 0, nw * sizeof(uint64_t));
    region_t r = { NULL, out, x0, y0, z0, nx, ny, nz, 0, 0 };
    fill_region(s, &r);
    uint64_t cnt = 0;
    for (size_t i = 0; i < nw; i++) cnt += (uint64_t)__builtin_popcountll(out[i]);
    return cnt;
}

int sg_fill_bits_z(const sg_scene* s, int32_t x0, int32_t y0, int32_t z0,
                   int32_t nx, int32_t ny, int32_t nz, uint64_t* out, int32_t* zr) {
    zr[0] = zr[1] = 0;
    if (nx % 64) return -1;
    region_t r = { NULL, out, x0, y0, z0, nx, ny, nz, 0x7FFFFFFF, -0x7FFFFFFF };
    fill_region(s, &r);
    if (r.zlo >= r.zhi) return 0;
    zr[0] = r.zlo - z0;
    zr[1] = r.zhi - z0;
    return 1;
}
