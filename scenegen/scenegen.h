/*
 * scenegen -- seeded synthetic voxel-world generator (input data only).
 *
 * This module produces the LOD-0 input scene that both the CPU oracle and the
 * GPU library consume: occupancy of every LOD-0 voxel and its uint8 material.
 * It contains none of the rendering method's arithmetic (no DAG building, no
 * LOD aggregation, no ray casting).  All arithmetic here is integer, so every
 * platform (x86-64, aarch64) produces bit-identical worlds.
 *
 * The paper evaluates on voxelised San Miguel / Sponza / Greenfield scenes
 * (Sec. 4); those datasets are not available, so procedural open worlds with
 * the same character (terrain plus city blocks, up to tens of billions of
 * voxels) stand in for them.
 *
 * World model (up axis = z, LOD-0 voxel units, voxel k covers [k, k+1)):
 *   height  h(x,y) = h_min + ((h_max-h_min) * n(x,y)) >> 16, where n is a
 *           sum of `octaves` octaves of Q16 value noise.  Octave o has period
 *           period0 >> o and weight 2^-o; lattice values come from the
 *           SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014) of
 *           (i, j, o, seed); interpolation is bilinear with the smoothstep
 *           weight s = t^2 (3 - 2t), all in Q16 fixed point.
 *   terrain filled (crust == 0): solid iff 0 <= z < h(x,y)
 *           crust  (crust  > 0): solid iff lo(x,y) <= z < h(x,y), with
 *           lo = max(0, min(h(x,y), h(x+-1,y), h(x,y+-1)) - crust); every
 *           exposed side face of a column is therefore backed by solid voxels.
 *   boxes   axis-aligned boxes, either solid or hollow (1-voxel shell).
 *   solid   = terrain OR any box; material(x,y,z) = hash(x,y,z,seed) & 0xFF
 *   (mat_mode 0), or (mat_mode 1) spatially coherent: a stratum of 8 voxels
 *   in z combined with a 64x64 column cell, plus a hashed value on 1 voxel
 *   in 64 -- long runs of equal values in depth-first order, as colours of
 *   real scenes have.
 */
#ifndef SCENEGEN_H
#define SCENEGEN_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_box {
    int32_t x0, y0, z0;   /* min corner (LOD-0 voxels) */
    int32_t sx, sy, sz;   /* side lengths */
    int32_t hollow;       /* 1: only the 1-voxel shell is solid */
} sg_box;

typedef struct sg_params {
    uint64_t seed;
    int32_t wx, wy, wz;        /* world extent in LOD-0 voxels */
    int32_t octaves;           /* value-noise octaves */
    int32_t period0;           /* period of octave 0 (voxels) */
    int32_t h_min, h_max;      /* terrain height range */
    int32_t crust;             /* 0: filled terrain, >0: crust thickness */
    int32_t n_boxes;           /* number of seeded boxes */
    int32_t box_min, box_max;  /* box side range (inclusive) */
    int32_t box_hollow;        /* 1: hollow city boxes on the terrain; 0: solid floating boxes */
    int32_t mat_mode;          /* 0: material = hash per voxel; 1: layered (coherent) materials */
} sg_params;

typedef struct sg_scene sg_scene;

/* Create a scene (draws the box list from the seed).  Returns NULL on bad params. */
sg_scene* sg_create(const sg_params* p);
/* The same with the box list given instead of drawn: p->n_boxes entries of
 * `boxes`, each inside the world (NULL otherwise).  For hand-made test scenes. */
sg_scene* sg_create_with_boxes(const sg_params* p, const sg_box* boxes);
void sg_destroy(sg_scene* s);
const sg_params* sg_get_params(const sg_scene* s);
int32_t sg_num_boxes(const sg_scene* s);
void sg_get_box(const sg_scene* s, int32_t i, sg_box* out);

/* SplitMix64 finaliser (public) -- exposed so that seeded camera poses can use
 * the same integer stream on every platform. */
uint64_t sg_mix64(uint64_t z);

/* Terrain height at integer column (x, y); defined for every integer x, y. */
int32_t sg_height(const sg_scene* s, int32_t x, int32_t y);
/* Heights of a rectangle: out[(y-y0)*nx + (x-x0)]. */
void sg_heights(const sg_scene* s, int32_t x0, int32_t y0, int32_t nx, int32_t ny, int32_t* out);

/* Point queries. Outside [0,w) on any axis the world is empty. */
int sg_solid(const sg_scene* s, int32_t x, int32_t y, int32_t z);
uint8_t sg_material(const sg_scene* s, int32_t x, int32_t y, int32_t z);

/* Dense occupancy of the box region [x0,x0+nx) x [y0,y0+ny) x [z0,z0+nz).
 * Byte layout: out[x + nx*(y + ny*z)] in {0,1}.  Returns the solid count. */
uint64_t sg_fill_bytes(const sg_scene* s, int32_t x0, int32_t y0, int32_t z0,
                       int32_t nx, int32_t ny, int32_t nz, uint8_t* out);
/* Bit layout (nx a multiple of 64): bit (x & 63) of word
 * out[(x >> 6) + (nx >> 6) * (y + ny*z)].  Returns the solid count. */
uint64_t sg_fill_bits(const sg_scene* s, int32_t x0, int32_t y0, int32_t z0,
                      int32_t nx, int32_t ny, int32_t nz, uint64_t* out);

/* Materials of the listed voxels: out[i] = material(xyz[3i], xyz[3i+1], xyz[3i+2]). */
void sg_materials(const sg_scene* s, const int32_t* xyz, size_t n, uint8_t* out);
/* Materials of the solid voxels of one 4x4x4 block with corner (x0, y0, z0):
 * out[b] = material(x0 + (b & 3), y0 + ((b >> 2) & 3), z0 + (b >> 4)) for every
 * set bit b of `mask`; the other entries of out[64] are left as they are. */
void sg_materials_block4(const sg_scene* s, int32_t x0, int32_t y0, int32_t z0, uint64_t mask, uint8_t* out);

/* sg_fill_bits into a buffer the caller has zeroed (nothing is cleared here),
 * without the count: returns 1 if any voxel of the region is solid, else 0.
 * zr[0], zr[1] (region-local z) are the lowest z holding a solid voxel and one
 * past the highest, so every row outside [zr[0], zr[1]) is left untouched
 * (zr = {0, 0} when nothing is solid).  Returns -1 (nothing written) unless nx
 * is a multiple of 64. */
int sg_fill_bits_z(const sg_scene* s, int32_t x0, int32_t y0, int32_t z0,
                   int32_t nx, int32_t ny, int32_t nz, uint64_t* out, int32_t* zr);

#ifdef __cplusplus
}
#endif
#endif
