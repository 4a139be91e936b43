/*
 * oracle -- plain, slow CPU reference of the chunked multi-LOD SVDAG
 * primary-ray path of "Aokana: A GPU-Driven Voxel Rendering Framework for
 * Open World Games" (Fang, Wang, Wang, PACMCGIT 8(1), 2025).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code
 * with the GPU library; both read their input worlds from scenegen.
 *
 * What it computes, and where the paper defines it:
 *   or_lod_down      LOD aggregation, Sec. 3.4: a voxel of LOD n exists iff at
 *                    least density = 2 of its 8 LOD n-1 voxels exist; its value
 *                    is the average of theirs (applied to uint8 materials,
 *                    rounded to nearest integer).
 *   or_dag_build     geometry compression, Sec. 3.2 (and Fig. 2): an octree whose
 *                    isomorphic subtrees are merged; node = 32-bit header whose
 *                    low 8 bits are the child mask, 32-bit subtree leaf count,
 *                    then one 32-bit child pointer per set mask bit; the three
 *                    deepest levels are a 4x4x4 block stored as a 64-bit mask.
 *                    Built bottom-up with one dedup table per level.
 *   materials        colour decoupling, Sec. 3.3: one value per solid voxel in
 *                    depth-first order; the DFS index of a voxel is the sum,
 *                    along its root path, of the leaf counts of earlier
 *                    siblings (or_dag_dfs_index).
 *   or_select_*      LOD selection, Sec. 3.4 Eq. 1, recursive (as described in
 *                    the paper) and per-chunk closed form.
 *   or_cast          first solid voxel along each pixel's ray in the LOD-cut
 *                    scene (every chunk region shown at its selected LOD),
 *                    traced in FP64 over the oracle's own DAGs, with the
 *                    material resolved through the DFS index (Sec. 3.5 colour
 *                    resolve) and an ambiguity flag.
 *   or_cast_brute    the same first hit by testing every voxel of the dense
 *                    LOD-cut grid (no DAG) -- used to pin or_cast.
 *
 * Readings where the paper is silent (listed with reasons in the design notes):
 *   bit order in a leaf block x + 4y + 16z; child octant x | y<<1 | z<<2;
 *   "leaf nodes" counted by or_dag leaf counts are solid voxels; LOD tie
 *   LODError == 0 loads (does not subdivide); Eq. 1 is evaluated as a squared
 *   comparison in IEEE FP64 with a fixed operation order; rays are generated
 *   in FP32 with a fixed operation order and no contraction.
 */
#ifndef AOK_ORACLE_H
#define AOK_ORACLE_H
#include <stdint.h>
#include <stddef.h>
#include "../scenegen/scenegen.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- LOD aggregation (Sec. 3.4) ---------------------------------------- */
/* occ/mat: dense side r (index x + r*(y + r*z)); outputs of side r/2. */
void or_lod_down(const uint8_t* occ, const uint8_t* mat, int32_t r, uint8_t* occ2, uint8_t* mat2);

/* ---- SVDAG (Sec. 3.2, 3.3) --------------------------------------------- */
typedef struct or_dag {
    uint32_t* nodes; uint64_t n_words;     /* node pool (words)                 */
    uint64_t* leaves; uint64_t n_leaves;   /* 4x4x4 leaf masks                  */
    uint8_t* mats; uint64_t n_mats;        /* materials in DFS order            */
    uint32_t root;                         /* word index of the root; n_words==0 => empty */
    int32_t res;                           /* voxels per axis (power of 2, >= 8) */
    int32_t n_int;                         /* interior levels = log2(res) - 2   */
    uint64_t level_nodes[16];              /* unique nodes per interior level (0 = root level) */
} or_dag;

/* Build from a dense grid of side res (occ in {0,1}; mat read where occ). 0 on success. */
int or_dag_build(const uint8_t* occ, const uint8_t* mat, int32_t res, or_dag* out);
void or_dag_free(or_dag* g);
/* Decompress to dense occupancy and materials (mat = 0 where empty). */
void or_dag_decode(const or_dag* g, uint8_t* occ, uint8_t* mat);
/* DFS index of voxel (x,y,z) (chunk-local voxel units at the DAG's LOD); -1 if empty. */
int64_t or_dag_dfs_index(const or_dag* g, int32_t x, int32_t y, int32_t z);

/* ---- colour blocks (Sec. 3.3, colour compression) ---------------------- */
/* The DFS colour array v[0..n) cut into blocks of consecutive entries, left
 * to right: an entry joins the current block when its distance to the
 * block's colour is within e_c (on the 0..1 scale of v / 255), and the
 * block's colour becomes the average of its entries (rounded mean of the
 * uint8 values, (sum + count/2) / count); otherwise it opens a new block.
 * Writes each block's first index and colour; returns the block count.
 * e_c = 0 gives the runs of equal values. */
uint64_t or_color_blocks(const uint8_t* v, uint64_t n, double e_c, uint64_t* start, uint8_t* color);
/* Colour of entry idx: the block with the largest start <= idx (Sec. 3.5,
 * colour resolve by binary search over the block array). */
uint8_t or_color_lookup(const uint64_t* start, const uint8_t* color, uint64_t n_blocks, uint64_t idx);

/* ---- LOD selection (Sec. 3.4, Eq. 1) ------------------------------------ */
/* StreamingFactor equivalent to a pixel threshold tau: a voxel of LOD n at
 * distance d covers 2^n H / (2 tan(fovy/2) d) pixels, so Eq. 1's cut-off
 * ChunkSize*SF = distance with ChunkSize = 2^n M is the tau-pixel cut-off
 * when SF = (H / (2 tan_half_fovy)) / (tau M). */
double or_streaming_factor(int32_t H, float tan_half_fovy, double tau, int32_t M);
/* Eq. 1 for the octree block at level n (2^n chunks per side) with block
 * coordinate b: returns 1 when the block is loaded at this level
 * (LODError <= 0), 0 when it subdivides (LODError > 0). */
int or_lod_loads(int32_t n, const int32_t b[3], int32_t M, const float o[3], double sf);
/* Closed form per chunk: first n from L-1 down to 0 with LODError_n <= 0, else 0. */
void or_select_closed(int32_t gx, int32_t gy, int32_t gz, int32_t M, int32_t L,
                      const float o[3], double sf, int8_t* lod_out);
/* Recursive implicit-octree search as described in Sec. 3.4. */
void or_select_recursive(int32_t gx, int32_t gy, int32_t gz, int32_t M, int32_t L,
                         const float o[3], double sf, int8_t* lod_out);

/* ---- rays --------------------------------------------------------------- */
typedef struct or_cam {
    float o[3];          /* origin, LOD-0 voxel units */
    float R[9];          /* row-major 3x3; columns = right, up, back */
    float tan_half_fovy;
    int32_t W, H;
} or_cam;
/* Pixel (px, py) direction, FP32, fixed op order, no contraction:
 * u = (((2px+1)/W) - 1) * t * (W/H); v = (1 - (2py+1)/H) * t;
 * d_i = ((R_i0 u) + (R_i1 v)) - R_i2. */
void or_ray_dir(const or_cam* cam, int32_t px, int32_t py, float d[3]);

/* ---- scene + cast --------------------------------------------------------- */
typedef struct or_scene or_scene;
or_scene* or_scene_create(const sg_scene* world, int32_t M, int32_t L);
void or_scene_destroy(or_scene* s);
/* Colour-block tolerance e_c of the scene's DAGs (< 0: exact colour arrays,
 * the default).  With e_c >= 0 every DAG built afterwards resolves colours
 * through or_color_blocks / or_color_lookup of its DFS colour array. */
void or_scene_set_color_tol(or_scene* s, double e_c);
/* Build the DAGs for every (chunk, lod_sel[chunk]) not yet built (threads > 0). */
int or_scene_prepare(or_scene* s, const int8_t* lod_sel, int n_threads);
/* Access a built DAG (NULL if not built). aabb: lo[3], hi[3] world LOD-0 units, [lo, hi). */
const or_dag* or_scene_dag(const or_scene* s, int32_t chunk, int32_t lod, int32_t aabb[6]);
/* Dense LOD-n occupancy + material of one chunk region (side M >> n), from the
 * world's LOD-0 voxels aggregated n times with or_lod_down. */
void or_chunk_dense(const sg_scene* world, int32_t M, int32_t cx, int32_t cy, int32_t cz, int32_t n,
                    uint8_t* occ, uint8_t* mat);

typedef struct or_result {
    int32_t x, y, z;       /* min corner of the hit voxel, LOD-0 world units */
    int32_t lod;           /* LOD of the hit voxel's chunk; 255 on miss */
    int32_t mat;           /* material; 0 on miss */
    int32_t normal;        /* 2*axis + (d_axis < 0); 7 = origin inside a voxel; 7 on miss */
    int32_t hit;           /* 1 hit, 0 miss */
    int32_t amb;           /* 1 if the pixel is ambiguous at eps = 1e-5 LOD voxel */
    double dist;           /* t* |d| in LOD-0 units; +inf on miss */
    uint32_t v_int;        /* interior-node visits (root included) along [0, t_end] */
    uint32_t v_leaf;       /* leaf-block visits along [0, t_end] */
    uint32_t resolve_bytes;/* sibling-count reads + 1 material byte (0 on miss) */
    uint32_t pad;
} or_result;

/* Trace n pixels (pix = px0,py0,px1,py1,...).  view_dist <= 0 means unlimited.
 * Chunks whose lod_sel is negative are treated as empty.  A (chunk, LOD) DAG is
 * built the first time a ray's segment reaches its chunk cell (or_scene_prepare
 * builds them ahead instead); the results do not depend on which were built. */
int or_cast(or_scene* s, const int8_t* lod_sel, const or_cam* cam, double view_dist,
            const int32_t* pix, int64_t n, or_result* out, int n_threads);
/* Same first hit by testing every voxel of every chunk's dense LOD grid.  Tiny scenes only. */
int or_cast_brute(const sg_scene* world, int32_t M, int32_t L, const int8_t* lod_sel,
                  const or_cam* cam, double view_dist, const int32_t* pix, int64_t n,
                  or_result* out, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
