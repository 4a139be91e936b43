/*
 * aok.h -- C ABI of the GB300 primary-ray library for chunked multi-LOD
 * sparse voxel DAG scenes (after "Aokana: A GPU-Driven Voxel Rendering
 * Framework for Open World Games", Fang, Wang, Wang, PACMCGIT 8(1), 2025).
 *
 * A scene is a grid of chunk regions, each M^3 LOD-0 voxels (Sec. 3.1), each
 * stored at n_lods levels of detail (Sec. 3.4) as one sparse voxel DAG per
 * (chunk, LOD) (Sec. 3.2) with a depth-first material array (Sec. 3.3).  A
 * frame selects one LOD per chunk region with Eq. 1, culls chunks to the
 * view, and casts one primary ray per pixel to its first solid voxel,
 * returning voxel coordinate, LOD, material and hit distance (the ray
 * marching and colour-resolve passes of Sec. 3.5).
 *
 * Conventions common to every call:
 *  - Every call returns an aok_status (int); no C++ exception or abort
 *    crosses this boundary.  AOK_E_CUDA means a CUDA error was observed; a
 *    sticky device error leaves the context unusable.
 *  - Host pointers are read during the call only; the caller keeps ownership.
 *  - "device" pointers are CUDA global-memory addresses on the context's
 *    device, owned by the caller unless stated otherwise.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls taking a stream only enqueue work; they return before
 *    the GPU finishes.
 *  - Coordinates are LOD-0 voxel units, up axis z; voxel k covers [k, k+1).
 *  - A context is used by one host thread at a time, except the serving
 *    calls (aok_serve_*), which are thread-safe.
 */
#ifndef AOK_H
#define AOK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum aok_status {
    AOK_OK = 0,
    AOK_PENDING = 1,          /* serving: request not finished yet */
    AOK_E_INVALID = -1,       /* bad argument (null, out of range, misaligned) */
    AOK_E_OOM = -2,           /* HBM budget or pool capacity exceeded */
    AOK_E_NOT_RESIDENT = -3,  /* chunk/LOD or scene not present */
    AOK_E_TIMEOUT = -4,       /* a bounded wait ran out */
    AOK_E_CUDA = -5,          /* CUDA runtime error */
    AOK_E_BUSY = -6,          /* serving: no free slot, retry later */
    AOK_E_CORRUPT = -7        /* chunk blob failed validation */
} aok_status;

typedef struct aok_ctx aok_ctx;

/* ------------------------------------------------------------------ */
/* Context                                                            */
/* ------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  All device memory the library
 * allocates (scene pools, per-frame tables, serving slots) is charged
 * against `hbm_budget_bytes` (0 = 90% of the device's free memory at
 * creation).  Returns AOK_E_INVALID for a bad device, AOK_E_CUDA on
 * initialisation failure. */
int aok_create(aok_ctx** out, int device, size_t hbm_budget_bytes);
/* Wait for the context's work, free every allocation, stop serving. */
void aok_destroy(aok_ctx* ctx);
/* Bytes currently charged against the budget / the budget itself. */
int aok_memory(aok_ctx* ctx, size_t* used_bytes, size_t* budget_bytes);
const char* aok_status_str(int status);

/* ------------------------------------------------------------------ */
/* Scenes and chunk residency (Sec. 3.1-3.4)                          */
/* ------------------------------------------------------------------ */

typedef struct aok_scene_desc {
    int32_t grid[3];          /* chunk regions per axis (>= 1); grid*chunk_res <= 131072 per axis */
    int32_t chunk_res;        /* M: LOD-0 voxels per chunk side, power of two in [8, 512] */
    int32_t n_lods;           /* LODs per chunk, 1 <= n_lods and (chunk_res >> (n_lods-1)) >= 8 */
    float view_dist;          /* > 0: hits farther than this (LOD-0 units) are misses; 0 = none */
    uint64_t node_words;      /* pool capacities: DAG node words (uint32, blob format; the device
                                 layout stores a prefix count beside every child pointer and
                                 reserves twice this many words) ... */
    uint64_t leaf_count;      /* ... 4x4x4 leaf masks (uint64) ... */
    uint64_t mat_bytes;       /* ... material bytes */
} aok_scene_desc;

/* Allocate a scene's device pools (charged to the budget; AOK_E_OOM if they
 * do not fit).  *scene_id receives a handle. */
int aok_scene_create(aok_ctx* ctx, const aok_scene_desc* desc, uint32_t* scene_id);
/* Free a scene (waits for the context's streams first). */
int aok_scene_destroy(aok_ctx* ctx, uint32_t scene);

/* One (chunk, LOD) as produced offline (Sec. 3.2, Sec. 3.3, Fig. 2).
 *  nodes  : uint32 words.  A node is [header, leaf_count, child_0 .. child_{k-1}]:
 *           header bits 0..7 = child mask (bit o set <=> octant o non-empty;
 *           octant o = x | y<<1 | z<<2), bits 8..31 zero; leaf_count = solid
 *           voxels in the subtree; k = popcount(mask) child pointers in octant
 *           order.  A node covering 8x8x8 voxels of its LOD points into
 *           `leaves`; every other node points to node word indices.  Pointers
 *           are relative to this blob.
 *  leaves : uint64 masks of 4x4x4 voxel blocks, bit x + 4y + 16z.
 *  mats   : one uint8 per solid voxel in depth-first order (ascending octant,
 *           then ascending leaf bit); n_mats = leaf_count of the root.
 *  root   : word index of the root node (covers the whole chunk region at
 *           resolution chunk_res >> lod).  n_node_words == 0 => empty chunk.
 *  aabb   : bounding box of the solid voxels, chunk-local LOD-0 units, [lo, hi). */
typedef struct aok_chunk_blob {
    const uint32_t* nodes;
    uint64_t n_node_words;
    const uint64_t* leaves;
    uint64_t n_leaves;
    const uint8_t* mats;
    uint64_t n_mats;
    uint32_t root;
    int32_t aabb_lo[3];
    int32_t aabb_hi[3];
} aok_chunk_blob;

/* Validate a host blob, rebase its pointers and copy it into the scene's
 * device pools (synchronously on the context's copy stream).  Replaces a
 * previous upload of the same (chunk, lod).  The validator walks every node
 * reachable from the root and returns AOK_E_CORRUPT (uploading nothing) for
 * an out-of-range pointer, a zero or reserved-bit header, a node reached at
 * two depths, a leaf count that is not the sum of its children's, a root
 * count different from n_mats, or an AABB outside the chunk; a rejected
 * blob changes nothing.  When the pools cannot hold the new blob next to the
 * previous upload of the same (chunk, lod), the previous one is evicted
 * first; AOK_E_OOM if the blob still does not fit (the chunk is then
 * non-resident).  AOK_E_INVALID for a bad chunk/lod. */
int aok_scene_upload_chunk(aok_ctx* ctx, uint32_t scene, int32_t cx, int32_t cy, int32_t cz,
                           uint32_t lod, const aok_chunk_blob* blob);
/* Host-only check of a blob against the rules aok_scene_upload_chunk applies
 * (no device work, no context needed): AOK_OK, AOK_E_CORRUPT, or
 * AOK_E_INVALID for a bad chunk_res / lod. */
int aok_validate_chunk(const aok_chunk_blob* blob, int32_t chunk_res, uint32_t lod);
/* Make a (chunk, lod) non-resident (it renders as empty).  Pool space of the
 * evicted chunk is reused by later uploads of at most the same size. */
int aok_scene_evict_chunk(aok_ctx* ctx, uint32_t scene, int32_t cx, int32_t cy, int32_t cz, uint32_t lod);
/* Colour-block compression of the scene's colour (material) arrays (Sec. 3.3):
 * chunks uploaded after this call store their DFS colour array as blocks of
 * consecutive entries -- an entry within e_c (on the 0..1 scale of value/255)
 * of the current block's colour joins it and the block's colour becomes the
 * rounded mean (sum + count/2) / count of its entries; any other entry opens a
 * new block -- and the casting kernels resolve a hit's colour by binary search
 * for the last block whose first index is <= the DFS index (Sec. 3.5).
 * e_c = 0 is lossless (runs of equal values); e_c > 0 is lossy; e_c < 0
 * (the default) stores raw arrays.  Blocks take 5 bytes each plus a 4-byte
 * search hint per 128 entries; a chunk whose blocks would not be smaller than
 * its array stores one byte per entry instead,
 * holding the colour its block gives (the same rendered colours).
 * AOK_E_INVALID for e_c > 1 or NaN. */
int aok_scene_set_color_blocks(aok_ctx* ctx, uint32_t scene, double e_c);
/* Device pool usage of the scene's resident (chunk, LOD)s: usage[0] node
 * bytes, [1] leaf bytes, [2] colour bytes (blocks or raw arrays), [3] resident
 * (chunk, LOD) count. */
int aok_scene_usage(aok_ctx* ctx, uint32_t scene, uint64_t* usage);

/* ------------------------------------------------------------------ */
/* Cameras and frames                                                 */
/* ------------------------------------------------------------------ */

/* Pinhole camera.  origin components must be multiples of 2^-12 with
 * |origin| < 2^17 (exact fixed-point traversal; AOK_E_INVALID otherwise).
 * R is row-major 3x3 whose columns are right, up and back (= -forward).
 * The ray of pixel (px, py) is origin + t d with d computed in IEEE binary32,
 * one rounding per operation, no contraction:
 *   u = (((2px+1)/W) - 1) * tan_half_fovy * (W/H),  v = (1 - (2py+1)/H) * tan_half_fovy,
 *   d_i = ((R_i0 u) + (R_i1 v)) - R_i2.
 * width, height >= 1, height <= 524280 (65535 rows of 8-pixel casting blocks)
 * and width * height < 2^31 (AOK_E_INVALID otherwise). */
typedef struct aok_camera {
    float origin[3];
    float R[9];
    float tan_half_fovy;
    int32_t width, height;
} aok_camera;

/* Per-pixel output, caller-owned device buffers, row-major (py*W + px):
 *  hit  : 4 x uint32 per pixel, 16-byte aligned: x, y, z = min corner of the
 *         first-hit voxel (LOD-0 units, multiples of 2^lod) and meta =
 *         lod (bits 0..7) | material << 8 | normal << 16 (3 bits:
 *         2*axis + (d_axis < 0) for the voxel face the ray enters through,
 *         the lowest such axis when it enters through an edge or a corner;
 *         7 = origin inside a voxel) | 1 << 19 (hit).
 *         A miss writes x = y = z = 0, meta = 0xFF | 7 << 16.
 *  t    : float per pixel, 4-byte aligned: hit distance |t* d| in LOD-0
 *         units (+inf on a miss). */
typedef struct aok_frame {
    void* hit;
    float* t;
} aok_frame;

/* ------------------------------------------------------------------ */
/* Per-frame LOD selection and visibility (Sec. 3.4 Eq. 1, Sec. 3.5)  */
/* ------------------------------------------------------------------ */

/* Select one LOD per chunk region with Eq. 1,
 *   LODError = ChunkSize * StreamingFactor - |ChunkCenter - CameraPos|,
 * over the implicit chunk octree (level n block = (2^n)^3 chunk regions,
 * ChunkSize = 2^n M, centre = the block's centre): a chunk takes the first
 * level n from n_lods-1 down to 0 whose LODError <= 0, else 0.  The pixel
 * threshold tau maps to StreamingFactor = (H / (2 tan_half_fovy)) / (tau M),
 * i.e. an LOD-n voxel at the cut-off distance covers tau pixels.  Evaluated
 * in IEEE FP64 with a fixed operation order.  When the selected (chunk, LOD)
 * has not been uploaded (it may still be streaming in) but another LOD of
 * the region has, that LOD stands in: the nearest coarser one, else the
 * nearest finer one.  Then culls chunks whose DAG is empty or not resident,
 * whose AABB lies outside the view pyramid, or (view_dist > 0) beyond the
 * view distance.
 *  lod_per_chunk_dev : optional device int8[grid x*y*z] (x fastest) receiving
 *                      every chunk region's LOD: Eq. 1's, or the stand-in
 *                      actually used.
 *  visible_dev       : optional device uint8[grid x*y*z]: 1 if the chunk is
 *                      kept for casting, 0 if empty, not resident or culled.
 *  n_visible_out     : optional host pointer; if given the call synchronises
 *                      the stream and returns the number of visible chunks.
 * Enqueued on `stream`; writes the scene's per-frame chunk table used by the
 * next aok_render of this scene on the same stream. */
int aok_select_chunks(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double lod_threshold_px,
                      int8_t* lod_per_chunk_dev, uint8_t* visible_dev, uint32_t* n_visible_out, void* stream);

/* ------------------------------------------------------------------ */
/* Asynchronous streaming (Sec. 3.4)                                  */
/* ------------------------------------------------------------------ */

/* Produces the blob of one (chunk, LOD) on the calling (worker) thread:
 * returns 0 and fills *out (pointers valid until release(user, *handle)),
 * non-zero on failure. */
typedef int (*aok_chunk_source_fn)(void* user, int32_t cx, int32_t cy, int32_t cz, uint32_t lod,
                                   aok_chunk_blob* out, void** handle);
typedef void (*aok_chunk_release_fn)(void* user, void* handle);

typedef struct aok_stream aok_stream;

/* Background loader that keeps the (chunk, LOD)s a camera needs resident in
 * a scene's device pools (Sec. 3.4).  n_threads worker threads take load
 * requests in the paper's order -- coarser LODs first, then the regions
 * nearest the camera -- build each blob with `source`, validate it and copy
 * it into free pool space (copy stream), while frames keep rendering.  A
 * loaded (chunk, LOD) becomes visible to rendering only at the next
 * aok_stream_update, which installs every change with one small kernel on
 * the rendering stream, so a frame sees a consistent descriptor table.  Pool
 * space of an evicted (chunk, LOD) is reused only after the rendering work
 * enqueued before its eviction has finished.  While a region's selected LOD
 * is not resident yet, frames render the nearest resident LOD of the region
 * (coarser first; see aok_select_chunks' lod output).  The scene's pools
 * (aok_scene_desc capacities) are the HBM budget: a load that does not fit
 * waits for evictions and is retried.  The streamer owns the residency of
 * its scene: do not upload or evict its chunks by other calls meanwhile.
 * Destroy it before the scene; destroying the scene (or its context) first
 * stops it -- its workers are joined, its loads freed -- after which
 * aok_stream_update, _wait and _set_prefetch return AOK_E_NOT_RESIDENT and
 * aok_stream_destroy only frees the object. */
int aok_stream_create(aok_ctx* ctx, uint32_t scene, aok_chunk_source_fn source, aok_chunk_release_fn release,
                      void* user, int32_t n_threads, aok_stream** out);
/* Between frames, on the rendering thread: plan the camera's residency (as
 * aok_plan_residency), install the loads finished since the last update and
 * the evictions of LODs no longer needed (a region keeps its old LOD until
 * the new one is installed) on `stream`, cancel queued requests the new plan
 * no longer wants, queue the missing ones, free quarantined pool space whose
 * frames are done.  Does not wait for loads.  Frames must render on `stream`
 * (or streams ordered after it). */
int aok_stream_update(aok_stream* s, const aok_camera* cam, double lod_threshold_px, void* stream);
/* Block until no load is queued or running (AOK_E_TIMEOUT after timeout_ms;
 * < 0 waits without limit).  The finished loads are installed by the next
 * aok_stream_update.  A wait under way when the scene is destroyed returns
 * AOK_E_NOT_RESIDENT. */
int aok_stream_wait(aok_stream* s, int32_t timeout_ms);
/* Load ahead of need along the camera's motion (not in the paper, which
 * plans for the current camera only).  From its second update on, each
 * aok_stream_update also plans `samples` cameras moved on from the current
 * one by frames * k / samples (k = 1 .. samples) times the displacement
 * since the previous update (same orientation and projection).  LODs those
 * plans want are queued after the current plan's (the nearest in time
 * first) and are not evicted while an extrapolated plan still wants them;
 * the current plan's loads, evictions and stand-ins are as without
 * prefetch.  frames = 0 (the default) turns it off.  frames in [0, 1000],
 * samples in [1, 16] when frames > 0, else AOK_E_INVALID.  Takes effect at
 * the next update; costs `samples` more residency plans per update. */
int aok_stream_set_prefetch(aok_stream* s, int32_t frames, int32_t samples);
/* stats[0] installed (chunk, LOD)s, [1] their device bytes, [2] / [3] the
 * maxima of both so far, [4] queued requests, [5] loads running, [6] loads
 * finished but not installed, [7] installed in total, [8] evicted in total,
 * [9] requests cancelled, [10] loads that failed (source or validation),
 * [11] loads deferred for lack of pool space, [12] planned regions whose
 * planned LOD was not installed at the last update (0: the frame after it
 * renders exactly the Eq. 1 selection), [13] regions that update planned,
 * [14] installs of LODs that only an extrapolated plan wanted (prefetch).
 * stats holds 15 entries. */
int aok_stream_stats(aok_stream* s, uint64_t* stats);
/* Per chunk region (x fastest) the bitmask of installed LODs (bit l = LOD l). */
int aok_stream_resident(aok_stream* s, uint8_t* lod_masks);
/* Stop the workers (running loads finish), free loads not installed and
 * quarantined pool space (waits for their frames).  Installed chunks stay. */
int aok_stream_destroy(aok_stream* s);

/* ------------------------------------------------------------------ */
/* Chunk-blob files (the on-disk chunks the paper streams from)       */
/* ------------------------------------------------------------------ */

/* A file of (chunk, LOD) blobs of one chunking (chunk_res, n_lods, grid),
 * versioned and checksummed (64-bit FNV-1a over header, index and every
 * entry).  Written once -- create, add each blob (pointers read during the
 * call; one blob per (chunk, LOD), AOK_E_INVALID for a duplicate or an
 * out-of-range chunk), finish (writes index and header, syncs, frees the
 * handle) -- then opened for reading by any number of threads.  Host only. */
typedef struct aok_blobfile aok_blobfile;
int aok_blobfile_create(const char* path, int32_t chunk_res, int32_t n_lods, const int32_t grid[3],
                        aok_blobfile** out);
int aok_blobfile_add(aok_blobfile* f, int64_t chunk, uint32_t lod, const aok_chunk_blob* blob);
int aok_blobfile_finish(aok_blobfile* f);
/* Open for reading: AOK_E_CORRUPT for a wrong magic or version, a header or
 * index checksum mismatch, or sizes that do not match the file. */
int aok_blobfile_open(const char* path, aok_blobfile** out);
int aok_blobfile_info(const aok_blobfile* f, int32_t* chunk_res, int32_t* n_lods, int32_t grid[3],
                      uint64_t* n_entries);
/* Read one blob (chunk index x fastest): *out points into a buffer owned by
 * *handle until aok_blobfile_release(NULL, *handle).  AOK_E_NOT_RESIDENT if
 * the file holds no such entry, AOK_E_CORRUPT on a checksum mismatch. */
int aok_blobfile_read(aok_blobfile* f, int64_t chunk, uint32_t lod, aok_chunk_blob* out, void** handle);
void aok_blobfile_release(void* user, void* handle);
/* aok_chunk_source_fn over an open file (user = the aok_blobfile*): a
 * (chunk, LOD) the file does not hold is an empty chunk; a corrupt entry
 * fails the load.  Pair with aok_blobfile_release. */
int aok_blobfile_source(void* user, int32_t cx, int32_t cy, int32_t cz, uint32_t lod, aok_chunk_blob* out,
                        void** handle);
int aok_blobfile_close(aok_blobfile* f);

/* Residency plan for one camera, on the host (the streaming side of
 * Sec. 3.4): for every chunk region, the LOD that Eq. 1 selects -- the same
 * FP64 arithmetic as aok_select_chunks, so the GPU selection finds exactly
 * these (chunk, LOD) -- if the region's cell lies within the scene's view
 * distance of the camera (all regions when view_dist is 0), else 0xFF.
 * lod_out: host uint8[grid x*y*z] (x fastest).  Returns the number of
 * regions kept in *n_kept (optional). */
int aok_plan_residency(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double lod_threshold_px,
                       uint8_t* lod_out, uint32_t* n_kept);

/* One frame of the paper's per-frame work: the LOD selection of Eq. 1 and
 * the chunk culling (Sec. 3.4, Sec. 3.5 chunk selection pass), then the ray
 * marching pass (Sec. 3.5: every pixel's primary ray through the chunk grid
 * and the selected DAGs to its first solid voxel) with the colour-resolve
 * step (Sec. 3.3 depth-first index, Sec. 3.5) fused at the hit.  Selects as
 * aok_select_chunks and writes `frame` (layout above) on `stream`.  The
 * scene's per-frame chunk table is shared: aok_render calls on one scene that
 * overlap on the GPU (different streams) race; use aok_render_batch for
 * concurrent views.  AOK_E_INVALID for a bad camera, threshold or misaligned
 * frame, AOK_E_NOT_RESIDENT for an unknown scene, AOK_E_CUDA when a launch
 * fails (the context's last CUDA error then holds its code). */
int aok_render(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double lod_threshold_px,
               const aok_frame* frame, void* stream);

/* Tile-chunk pipeline (Sec. 3.5, Fig. 7): the same frame as aok_render,
 * computed the way the paper organises its GPU passes -- 8x8-pixel tiles
 * paired with the selected chunks whose AABB they may see (pair depth = the
 * distance from the camera to the AABB), Hi-Z occlusion culling of the pairs
 * against the previous frame's per-tile depth, ray marching of each pair
 * through its chunk's DAG into a visibility buffer (a 64-bit key and a
 * 64-bit payload per pixel, installed by a 128-bit compare-and-swap when the
 * key is the smallest), this frame's Hi-Z, a second culling + marching pass
 * over the pairs the first pass culled, and a resolve pass that writes the
 * output from the payloads.
 * The output equals aok_render's (see the one exception documented in the
 * implementation: rays entering the world box exactly on an interior chunk
 * plane).  The previous frame's Hi-Z only saves work; it is kept per context
 * for the last scene and resolution rendered.
 * Buffers (visibility records 16 B per pixel, per-tile and per-region arrays)
 * are allocated on first use and when the resolution or grid changes,
 * charged to the budget.  Not for concurrent calls on one context.
 * AOK_E_INVALID for scenes of more than AOK_TILES_MAX_CHUNKS regions (the key
 * holds a 16-bit region index) or a misaligned frame. */
#define AOK_TILES_MAX_CHUNKS 65536
int aok_render_tiles(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double lod_threshold_px,
                     const aok_frame* frame, void* stream);
/* Counters of the last aok_render_tiles frame (synchronises the device):
 * stats[0] chunk regions with pairs, [1] / [2] half-tile items marched /
 * culled by Hi-Z in pass 1, [3] / [4] the same in pass 2, [5] pixel rays
 * traced through a chunk, [6] pixel rays skipped because the pixel already
 * held a nearer hit, [7] records not installed because the compare-and-swap
 * loop ran out of attempts (0 unless the implementation is wrong).
 * AOK_E_INVALID before the first aok_render_tiles. */
int aok_tiles_stats(aok_ctx* ctx, uint64_t* stats);
/* Drop the Hi-Z history: the next aok_render_tiles runs its first pass
 * without occlusion culling (as on a scene's first frame). */
int aok_tiles_forget(aok_ctx* ctx);

/* Cast with the chunk table written by the last aok_select_chunks of this
 * scene (same camera), so that the two passes can be enqueued and timed
 * separately.  Same output contract as aok_render. */
int aok_cast_selected(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, const aok_frame* frame, void* stream);

/* aok_render into host memory: renders into library-owned device buffers,
 * then copies the frame into the caller's host buffers (hit_host: 16 bytes
 * per pixel, t_host: 4 bytes per pixel; pinned memory gives asynchronous
 * copies) and synchronises `stream` before returning.  The device buffers
 * are kept for the next call (grown on demand, charged to the budget). */
int aok_render_host(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double lod_threshold_px,
                    void* hit_host, float* t_host, void* stream);
/* Pipelined aok_render_host for frame loops: enqueues the render into one of
 * three library-owned device frames on a context stream and the copy into
 * the caller's host buffers (pinned) on a second stream, and returns at once
 * with a ticket, so that a frame's render overlaps the previous frame's copy.
 * The host buffers must stay valid and untouched until
 * aok_host_frame_wait(ticket) returns.  With three frames in flight, a new
 * call first waits for the oldest one's copy.  Frames of one context are
 * rendered in call order on the context's own stream: other renders of the
 * same scene must not overlap them (aok_render's rule). */
int aok_render_host_async(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double lod_threshold_px,
                          void* hit_host, float* t_host, uint64_t* ticket);
/* Block until the frame `ticket` is complete in host memory (AOK_E_INVALID
 * for a ticket never issued). */
int aok_host_frame_wait(aok_ctx* ctx, uint64_t ticket);

/* ------------------------------------------------------------------ */
/* Batched multi-view rendering                                       */
/* ------------------------------------------------------------------ */

typedef struct aok_view {
    uint32_t scene;
    aok_camera cam;
    double lod_threshold_px;
    aok_frame frame;
} aok_view;

/* Render n views (any scenes, uneven resolutions) with one selection launch
 * and one casting launch per group of up to 128 views: by default a grid
 * over the block tiles (2x2 warp tiles) of all views, scheduled by the
 * hardware; optionally (aok_set_batch_kernel) a persistent kernel whose warps
 * pull warp tiles from a global counter.  With the grid launch and the beam
 * pass on, one beam pass (a cooperative launch) per group serves all of the
 * group's views large enough for it, between the selection and the cast.
 * The launches of one list shape (n, scenes, sizes) -- selections, beam
 * passes with their counter resets, casts -- form a CUDA graph built on first
 * use and updated in place (aok_set_batch_graph(ctx, 0) launches them one by
 * one instead).  Results equal n separate aok_render calls.  Calls on one
 * context are serialised by the caller (one stream).  AOK_E_INVALID if n is 0
 * or above 4096. */
int aok_render_batch(aok_ctx* ctx, const aok_view* views, uint32_t n, void* stream);

/* 0: batches use the grid launch (default); 1: the persistent kernel. */
int aok_set_batch_kernel(aok_ctx* ctx, int persistent);
/* 1 (default): aok_render_batch replays a CUDA graph of its launches; 0: it
 * launches them one by one (same results). */
int aok_set_batch_graph(aok_ctx* ctx, int on);
/* Launch shape of the persistent casting kernel (0 = keep current):
 * CTAs per SM, threads per CTA (multiple of 32), rays per packet (multiple
 * of 32).  aok_autotune times grid launches (three warp tiles) and
 * persistent shapes on the given views and keeps the fastest; *best_ms
 * receives its time per batch.  aok_get_launch reports 0 CTAs per SM while
 * the grid launch is selected. */
int aok_set_launch(aok_ctx* ctx, uint32_t ctas_per_sm, uint32_t threads_per_cta, uint32_t packet_rays);
int aok_get_launch(aok_ctx* ctx, uint32_t* ctas_per_sm, uint32_t* threads_per_cta, uint32_t* packet_rays);
int aok_autotune(aok_ctx* ctx, const aok_view* views, uint32_t n, void* stream, float* best_ms);
/* Warp tile of the persistent kernel: tile_w x (32 / tile_w) pixels, tile_w in
 * {4, 8, 16, 32} (default 8).  aok_autotune also picks it. */
int aok_set_tile(aok_ctx* ctx, uint32_t tile_w);
/* Kernel used by aok_render / aok_cast_selected for one view: 0 = one thread
 * per pixel over a grid of 16x8 tiles (default), 1 = the persistent kernel of
 * aok_render_batch with this context's launch shape.  Results are identical. */
int aok_set_single_view_kernel(aok_ctx* ctx, int persistent);

/* ------------------------------------------------------------------ */
/* Continuous-batching serving                                        */
/* ------------------------------------------------------------------ */

typedef struct aok_request {
    uint32_t scene;
    aok_camera cam;
    double lod_threshold_px;
} aok_request;

/* Start the serving loop: a host thread admits submitted requests into at
 * most `max_slots` in-flight slots when their framebuffers fit in the HBM
 * budget, groups the admitted ones into batches of at most `max_batch`
 * views, and launches each batch on one of `n_streams` streams, so that new
 * arrivals overlap with batches already on the GPU. */
int aok_serve_start(aok_ctx* ctx, uint32_t max_slots, uint32_t max_batch, uint32_t n_streams);
/* Stop admitting, finish in-flight work, join the loop. */
int aok_serve_stop(aok_ctx* ctx);
/* Queue a request; *ticket identifies it.  AOK_E_BUSY when the submit queue
 * is full, AOK_E_NOT_RESIDENT for an unknown scene. */
int aok_serve_submit(aok_ctx* ctx, const aok_request* req, uint64_t* ticket);
/* AOK_PENDING while queued or running; AOK_OK when done, with out_view
 * pointing at library-owned device buffers valid until aok_serve_release. */
int aok_serve_poll(aok_ctx* ctx, uint64_t ticket, aok_frame* out_view);
/* Block until done or `timeout_ms` passes (AOK_E_TIMEOUT). */
int aok_serve_wait(aok_ctx* ctx, uint64_t ticket, uint32_t timeout_ms, aok_frame* out_view);
/* Return the ticket's buffers to the pool (cancels it if not started);
 * AOK_E_BUSY while its batch is on the GPU. */
int aok_serve_release(aok_ctx* ctx, uint64_t ticket);
/* Host steady-clock times (ns) at which the ticket was submitted and at which
 * the serving loop saw its batch complete (0 while not complete). */
int aok_serve_times(aok_ctx* ctx, uint64_t ticket, uint64_t* submit_ns, uint64_t* done_ns);

/* ------------------------------------------------------------------ */
/* Rendering without device allocation                                */
/* ------------------------------------------------------------------ */

/* Largest chunk grid (x*y*z chunk regions) aok_render_noalloc accepts. */
#define AOK_NOALLOC_MAX_CHUNKS 65536

/* aok_render for callers that must not allocate device memory while they
 * render -- for example an engine frame loop that reserved all of its device
 * memory up front, or code running under an allocator that forbids
 * cudaMalloc/cudaFree at that point.  (The paper has no counterpart: its
 * renderer is a set of engine passes.)  The result equals aok_render's.
 * The call allocates nothing and calls no cudaMalloc or cudaFree: the
 * per-frame chunk table that aok_render keeps in scene memory lives instead
 * in one static device array of AOK_NOALLOC_MAX_CHUNKS entries (2 MiB) that
 * every GPU loading this library holds until the process exits.
 *  - Scenes with more than AOK_NOALLOC_MAX_CHUNKS chunk regions are rejected
 *    with AOK_E_INVALID before any work is enqueued.
 *  - The first call on a device looks up the array's device address (with
 *    that device current) and caches it; make that first call before any
 *    CUDA stream capture.  The cached address belongs to the device's
 *    current context: do not call this function again in a process that has
 *    reset the device (cudaDeviceReset) after its first call there.
 *  - With aok_set_checked(ctx, 1) it launches the checked casting kernel, as
 *    aok_render does; the error word is context memory, so this allocates
 *    nothing either.
 *  - All calls share the one array and each call overwrites the entries it
 *    uses, so calls whose GPU work overlaps (different streams, or no
 *    ordering between them) race and may return wrong pixels; order them on
 *    one stream or synchronise between them.
 * The scene, camera and frame are passed as for aok_render. */
int aok_render_noalloc(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double lod_threshold_px,
                       const aok_frame* frame, void* stream);

/* Beam pass (ESVO's beam optimisation, which the paper's traversal builds on,
 * Sec. 2; here exact): with on = 1, aok_render, aok_render_counted,
 * aok_render_host(_async), aok_cast_selected, aok_render_batch (grid
 * launch) and the render server of this context first compute, for every 8 x 4 pixel tile of each
 * frame of at least 1.5 M pixels (aok_beam_tune), a lower bound on the
 * L-infinity distance from the camera origin of every solid voxel of the
 * frame's LOD-cut scene that the tile's rays can meet: a level-by-level walk
 * of the selected DAGs (all views of a batch in one launch), refining a node
 * while its screen rectangle spans more than R tiles and its side is above
 * 2^L voxels, each node scattering its distance over its rectangle with an
 * atomic minimum.  The casting kernels then restart each ray's march at the
 * last integer plane of its dominant axis that the ray crosses before that
 * distance.  Output records are identical with the pass on or off.  Buffers
 * (about 11 B per 8 x 4 pixel tile, grown to the largest frame or batch seen,
 * and two 16 MiB node queues) are charged to the budget when first needed.
 * The render server runs it for its batches too (per-request pyramids).
 * Not used by the persistent single-view and batch kernels,
 * aok_render_noalloc or the tile pipeline; with checked casting it runs with
 * its node and leaf indices checked.  Default on.  The pass's
 * buffers belong to the context: with it on, renders of one context on
 * different streams must be ordered (an event or a synchronisation between
 * them).  The passes of all contexts of a process run one after another on a
 * device (each waits for the previous one's launch to finish). */
int aok_set_beam(aok_ctx* ctx, int on);
/* Refinement of the beam pass's walk: a node is refined while its rectangle
 * spans more than refine_tiles tiles and its side is above 2^min_node_log2
 * LOD-0 voxels (defaults 8 and 2: down to the 4^3 leaves); frames of fewer
 * than min_pixels pixels cast without the pass (default 1,500,000: below
 * that the pass's fixed cost, some tens of microseconds, outweighs what it
 * saves); queue_nodes caps the nodes one level of the walk may queue
 * (0: the allocated 2^20; past the cap a node stands for its children).
 * Any setting gives the same output records.  AOK_E_INVALID for
 * min_node_log2 outside [2, 16]. */
int aok_beam_tune(aok_ctx* ctx, uint32_t refine_tiles, int32_t min_node_log2, uint64_t min_pixels,
                  uint32_t queue_nodes);
/* The beam pass alone, for the frame table the last aok_select_chunks (or
 * render) of this scene selected and this camera: the next
 * aok_cast_selected of the same scene and camera then casts with these
 * bounds instead of computing them again (so that the pass and the cast can
 * be timed apart).  Runs whether or not aok_set_beam is on.  Stream rules as
 * for aok_cast_selected. */
int aok_beam_selected(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, void* stream);
/* Selection and beam pass in one launch (Eq. 1 and visibility, Sec. 3.4-3.5,
 * then the bounds): the beam pass selects this camera's frame table as the
 * first step of its walk, as aok_render does when the pass runs.  Without
 * the pass for this frame (aok_set_beam off, a frame below the beam_tune
 * pixel floor, or a camera without a usable projection) it is
 * aok_select_chunks without outputs.  The next aok_cast_selected of the same
 * scene and camera casts the selection with these bounds.  Arguments and
 * stream rules as for aok_select_chunks and aok_cast_selected. */
int aok_select_beam(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double lod_threshold_px, void* stream);
/* The last beam pass of this context (synchronises the device): bounds
 * (nullable, n_bounds >= tiles_x * tiles_y entries, row-major, numerator
 * units of 2^-12 LOD-0 voxels, INT32_MAX = no solid voxel reachable; 0
 * everywhere if the camera matrix has no usable inverse), level_counts
 * (nullable, 16 entries: nodes walked at each depth below the region roots,
 * depth 0 the selected regions; a queue holds 2^20 nodes per level, past
 * that parents stand in for their children) and tiles_xy (nullable, 2).
 * AOK_E_INVALID before the first beam pass or if n_bounds is too small. */
int aok_beam_info(aok_ctx* ctx, int32_t* bounds, uint64_t n_bounds, uint32_t* level_counts, int32_t* tiles_xy);

/* ------------------------------------------------------------------ */
/* Diagnostics                                                        */
/* ------------------------------------------------------------------ */

/* Like aok_render, but also writes per-pixel traversal counts to the device
 * buffer counts (3 x uint32 per pixel: interior-node visits including chunk
 * roots, leaf-block visits, material-resolve bytes).  Slower; used to derive
 * the algorithmic bytes of a frame. */
int aok_render_counted(aok_ctx* ctx, uint32_t scene, const aok_camera* cam, double lod_threshold_px,
                       const aok_frame* frame, uint32_t* counts, void* stream);
/* Checked casting (no counterpart in the paper; the stand-in for a device
 * memory checker): with on = 1, aok_render / aok_cast_selected /
 * aok_render_noalloc of this context test every node, leaf and colour index against the scene's pool
 * sizes before loading it; an index out of range ends that chunk's traversal
 * as a miss and ORs a code into the context's error word (1 node word, 2
 * leaf, 4 colour).  The beam pass of aok_render and aok_select_beam keeps
 * running and tests its node and leaf indices too: one out of range ORs its
 * code and bounds the whole view by 0 (no ray skips anything).  Slower;
 * batches, serving, the pipelined host frames and the tile pipeline are not
 * checked. */
int aok_set_checked(aok_ctx* ctx, int on);
/* Read and clear the error word (synchronises the device); 0 = no index was
 * ever out of range. */
int aok_checked_errors(aok_ctx* ctx, uint32_t* errors);
/* Write every pixel's FP32 ray direction (3 floats per pixel) to the device
 * buffer dirs, as the casting kernel computes it. */
int aok_ray_dirs(aok_ctx* ctx, const aok_camera* cam, float* dirs, void* stream);
/* Read-bandwidth microbenchmark (no counterpart in the paper; the yardstick
 * for traversal kernels whose working set sits in L2).  Allocates a device
 * buffer of `bytes` (rounded down to 16; charged to the budget while the call
 * runs), reads it `reps` times with 16-byte L2 loads in one launch of one
 * resident grid after a warm-up launch of two passes, and writes the achieved
 * GB/s (1e9 B/s) of the timed launch to *gbs.
 * bytes below the L2 size measure L2, larger ones HBM.  Synchronous.
 * AOK_E_INVALID for bytes < 16 or reps < 1, AOK_E_OOM if the buffer does not fit. */
int aok_read_bandwidth(aok_ctx* ctx, uint64_t bytes, int reps, double* gbs);

#ifdef __cplusplus
}
#endif
#endif /* AOK_H */
