"""GB300 primary-ray casting through chunked multi-LOD sparse voxel DAGs.

Thin ctypes binding of the C ABI in include/aok.h (argument marshalling only:
every step of the path runs in the native library's CUDA kernels).  PyTorch
supplies device memory and streams.  There is no CPU fallback: importing the
binding raises if libaok.so cannot be built or loaded.

Method: "Aokana: A GPU-Driven Voxel Rendering Framework for Open World Games"
(Fang, Wang, Wang, PACMCGIT 8(1), 2025), Sec. 3.1-3.5 and Eq. 1.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _native

AOK_OK, AOK_PENDING = 0, 1
AOK_E_INVALID, AOK_E_OOM, AOK_E_NOT_RESIDENT, AOK_E_TIMEOUT = -1, -2, -3, -4
AOK_E_CUDA, AOK_E_BUSY, AOK_E_CORRUPT = -5, -6, -7


class AokError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {lib().aok_status_str(status).decode()} ({status})")


# ---------------------------------------------------------------------------
# ctypes mirrors of include/aok.h
# ---------------------------------------------------------------------------
class SceneDesc(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32 * 3), ("chunk_res", ctypes.c_int32), ("n_lods", ctypes.c_int32),
                ("view_dist", ctypes.c_float), ("node_words", ctypes.c_uint64), ("leaf_count", ctypes.c_uint64),
                ("mat_bytes", ctypes.c_uint64)]


class ChunkBlob(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_void_p), ("n_node_words", ctypes.c_uint64), ("leaves", ctypes.c_void_p),
                ("n_leaves", ctypes.c_uint64), ("mats", ctypes.c_void_p), ("n_mats", ctypes.c_uint64),
                ("root", ctypes.c_uint32), ("aabb_lo", ctypes.c_int32 * 3), ("aabb_hi", ctypes.c_int32 * 3)]


class Camera(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("R", ctypes.c_float * 9), ("tan_half_fovy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class Frame(ctypes.Structure):
    _fields_ = [("hit", ctypes.c_void_p), ("t", ctypes.c_void_p)]


class View(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_uint32), ("cam", Camera), ("lod_threshold_px", ctypes.c_double),
                ("frame", Frame)]


class Request(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_uint32), ("cam", Camera), ("lod_threshold_px", ctypes.c_double)]


_lib = None
_blib = None


def lib() -> ctypes.CDLL:
    """libaok.so with typed signatures (built in-tree on first use)."""
    global _lib
    if _lib is None:
        _native.build()
        L = ctypes.CDLL(_native.LIBAOK)
        vp, u32, i32, u64, dbl = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        P = ctypes.POINTER
        sig = {
            "aok_create": [P(vp), ctypes.c_int, ctypes.c_size_t],
            "aok_memory": [vp, P(ctypes.c_size_t), P(ctypes.c_size_t)],
            "aok_scene_create": [vp, P(SceneDesc), P(u32)],
            "aok_scene_destroy": [vp, u32],
            "aok_scene_upload_chunk": [vp, u32, i32, i32, i32, u32, P(ChunkBlob)],
            "aok_scene_evict_chunk": [vp, u32, i32, i32, i32, u32],
            "aok_scene_set_color_blocks": [vp, u32, dbl],
            "aok_stream_create": [vp, u32, vp, vp, vp, i32, P(vp)],
            "aok_stream_update": [vp, P(Camera), dbl, vp],
            "aok_stream_wait": [vp, i32],
            "aok_stream_stats": [vp, P(u64)],
            "aok_stream_set_prefetch": [vp, i32, i32],
            "aok_stream_resident": [vp, vp],
            "aok_stream_destroy": [vp],
            "aok_blobfile_create": [ctypes.c_char_p, i32, i32, P(i32), P(vp)],
            "aok_blobfile_add": [vp, ctypes.c_int64, u32, P(ChunkBlob)],
            "aok_blobfile_finish": [vp],
            "aok_blobfile_open": [ctypes.c_char_p, P(vp)],
            "aok_blobfile_info": [vp, P(i32), P(i32), P(i32), P(u64)],
            "aok_blobfile_read": [vp, ctypes.c_int64, u32, P(ChunkBlob), P(vp)],
            "aok_blobfile_close": [vp],
            "aok_blobfile_release": [vp, vp],
            "aok_blobfile_source": [vp, i32, i32, i32, u32, P(ChunkBlob), P(vp)],
            "aok_scene_usage": [vp, u32, P(u64)],
            "aok_select_chunks": [vp, u32, P(Camera), dbl, vp, vp, P(u32), vp],
            "aok_render": [vp, u32, P(Camera), dbl, P(Frame), vp],
            "aok_render_counted": [vp, u32, P(Camera), dbl, P(Frame), vp, vp],
            "aok_render_noalloc": [vp, u32, P(Camera), dbl, P(Frame), vp],
            "aok_render_tiles": [vp, u32, P(Camera), dbl, P(Frame), vp],
            "aok_render_host_async": [vp, u32, P(Camera), dbl, vp, vp, P(u64)],
            "aok_host_frame_wait": [vp, u64],
            "aok_tiles_stats": [vp, P(u64)],
            "aok_tiles_forget": [vp],
            "aok_ray_dirs": [vp, P(Camera), vp, vp],
            "aok_read_bandwidth": [vp, ctypes.c_uint64, ctypes.c_int, P(dbl)],
            "aok_cast_selected": [vp, u32, P(Camera), P(Frame), vp],
            "aok_plan_residency": [vp, u32, P(Camera), dbl, vp, P(u32)],
            "aok_render_host": [vp, u32, P(Camera), dbl, vp, vp, vp],
            "aok_validate_chunk": [P(ChunkBlob), i32, u32],
            "aok_render_batch": [vp, P(View), u32, vp],
            "aok_set_launch": [vp, u32, u32, u32],
            "aok_get_launch": [vp, P(u32), P(u32), P(u32)],
            "aok_autotune": [vp, P(View), u32, vp, P(ctypes.c_float)],
            "aok_set_tile": [vp, u32],
            "aok_set_batch_kernel": [vp, ctypes.c_int],
            "aok_set_batch_graph": [vp, ctypes.c_int],
            "aok_set_single_view_kernel": [vp, ctypes.c_int],
            "aok_set_checked": [vp, ctypes.c_int],
            "aok_set_beam": [vp, ctypes.c_int],
            "aok_beam_tune": [vp, u32, ctypes.c_int32, u64, u32],
            "aok_beam_info": [vp, P(ctypes.c_int32), u64, P(u32), P(ctypes.c_int32)],
            "aok_beam_selected": [vp, u32, P(Camera), vp],
            "aok_select_beam": [vp, u32, P(Camera), dbl, vp],
            "aok_checked_errors": [vp, P(u32)],
            "aok_serve_start": [vp, u32, u32, u32],
            "aok_serve_stop": [vp],
            "aok_serve_submit": [vp, P(Request), P(u64)],
            "aok_serve_poll": [vp, u64, P(Frame)],
            "aok_serve_wait": [vp, u64, u32, P(Frame)],
            "aok_serve_release": [vp, u64],
            "aok_serve_times": [vp, u64, P(u64), P(u64)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.aok_destroy.argtypes = [vp]
        L.aok_destroy.restype = None
        L.aok_status_str.argtypes = [ctypes.c_int]
        L.aok_status_str.restype = ctypes.c_char_p
        _lib = L
    return _lib


def blib() -> ctypes.CDLL:
    """libaokbuild.so: offline chunk preparation over scenegen worlds."""
    global _blib
    if _blib is None:
        _native.build()
        L = ctypes.CDLL(_native.LIBBUILD)
        vp = ctypes.c_void_p
        L.aokb_build.restype = vp
        L.aokb_build.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp, ctypes.c_int64, ctypes.c_int32]
        L.aokb_build_masked.restype = vp
        L.aokb_build_masked.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp, vp, ctypes.c_int64, ctypes.c_int32]
        L.aokb_free.argtypes = [vp]
        L.aokb_count.restype = ctypes.c_int64
        L.aokb_count.argtypes = [vp]
        L.aokb_get.restype = ctypes.c_int
        L.aokb_get.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ChunkBlob)]
        L.aokb_totals.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64 * 4)]
        L.aokb_source_create.restype = vp
        L.aokb_source_create.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
        L.aokb_source_destroy.argtypes = [vp]
        L.aokb_source_set_cache.argtypes = [vp, ctypes.c_uint64]
        L.aokb_source_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64 * 4)]
        _blib = L
    return _blib


def validate_chunk(blob: ChunkBlob, chunk_res: int, lod: int) -> int:
    """Host-only blob validation (no device needed); returns the status code."""
    return int(lib().aok_validate_chunk(ctypes.byref(blob), chunk_res, lod))


def check(status: int, what: str = "aok") -> int:
    if status < 0:
        raise AokError(status, what)
    return status


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def to_camera(cam) -> Camera:
    """From a scenegen.Camera (origin, R, tan_half_fovy, W, H)."""
    c = Camera()
    for i in range(3):
        c.origin[i] = float(cam.origin[i])
    R = np.asarray(cam.R, np.float32)
    for i in range(3):
        for j in range(3):
            c.R[3 * i + j] = float(R[i, j])
    c.tan_half_fovy = float(cam.tan_half_fovy)
    c.width, c.height = int(cam.W), int(cam.H)
    return c


# ---------------------------------------------------------------------------
# context / scene / frames
# ---------------------------------------------------------------------------
class Context:
    """One aok_ctx on a CUDA device (owns all library device memory)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        h = ctypes.c_void_p()
        check(lib().aok_create(ctypes.byref(h), device, budget_bytes), "aok_create")
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            lib().aok_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def memory(self):
        u, b = ctypes.c_size_t(), ctypes.c_size_t()
        check(lib().aok_memory(self.h, ctypes.byref(u), ctypes.byref(b)))
        return u.value, b.value


class BuiltWorld:
    """Chunk blobs (all LODs) of a scenegen world, built by libaokbuild."""

    def __init__(self, world, threads: int | None = None, chunks=None, lod_masks=None):
        spec = world.spec
        self.spec = spec
        arr = None
        msk = None
        n = 0
        if chunks is not None:
            arr = np.ascontiguousarray(chunks, np.int64)
            n = len(arr)
            if lod_masks is not None:
                msk = np.ascontiguousarray(lod_masks, np.uint32)
        self.h = blib().aokb_build_masked(world.handle, spec.chunk, spec.n_lods,
                                          arr.ctypes.data if arr is not None else None,
                                          msk.ctypes.data if msk is not None else None, n,
                                          threads or os.cpu_count() or 1)
        if not self.h:
            raise ValueError("bad chunking for the builder")
        t = (ctypes.c_uint64 * 4)()
        blib().aokb_totals(self.h, ctypes.byref(t))
        self.node_words, self.leaves, self.mat_bytes, self.nonempty = (int(v) for v in t)

    def __len__(self):
        return int(blib().aokb_count(self.h))

    def blob(self, i: int, lod: int):
        b = ChunkBlob()
        c = ctypes.c_int64()
        if blib().aokb_get(self.h, i, lod, ctypes.byref(c), ctypes.byref(b)) != 0:
            raise IndexError(i)
        return int(c.value), b

    def close(self):
        if self.h:
            blib().aokb_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BlobFile:
    """A chunk-blob file (aok_blobfile_*): write() stores a BuiltWorld's
    non-empty (chunk, LOD) blobs; BlobFile(path) opens one for reading."""

    @staticmethod
    def write(path: str, built: "BuiltWorld", grid, chunk_res: int, n_lods: int) -> int:
        g = (ctypes.c_int32 * 3)(*grid)
        h = ctypes.c_void_p()
        check(lib().aok_blobfile_create(os.fsencode(path), int(chunk_res), int(n_lods), g, ctypes.byref(h)),
              "aok_blobfile_create")
        n = 0
        try:
            for i in range(len(built)):
                for lod in range(n_lods):
                    c, b = built.blob(i, lod)
                    if b.n_node_words:
                        check(lib().aok_blobfile_add(h, int(c), int(lod), ctypes.byref(b)), "aok_blobfile_add")
                        n += 1
        finally:
            check(lib().aok_blobfile_finish(h), "aok_blobfile_finish")
        return n

    def __init__(self, path: str):
        h = ctypes.c_void_p()
        check(lib().aok_blobfile_open(os.fsencode(path), ctypes.byref(h)), "aok_blobfile_open")
        self.h = h

    def info(self):
        m, nl, n = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_uint64()
        g = (ctypes.c_int32 * 3)()
        check(lib().aok_blobfile_info(self.h, ctypes.byref(m), ctypes.byref(nl), g, ctypes.byref(n)),
              "aok_blobfile_info")
        return {"chunk_res": m.value, "n_lods": nl.value, "grid": tuple(g), "entries": n.value}

    def read(self, chunk: int, lod: int) -> dict:
        """One entry as numpy copies (nodes, leaves, mats, root, aabb)."""
        b = ChunkBlob()
        hd = ctypes.c_void_p()
        check(lib().aok_blobfile_read(self.h, int(chunk), int(lod), ctypes.byref(b), ctypes.byref(hd)),
              "aok_blobfile_read")
        try:
            def arr(ptr, n, dt):
                return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(dt)), (n,)).copy() if n else \
                    np.zeros(0, np.dtype(dt))
            return {"nodes": arr(b.nodes, b.n_node_words, ctypes.c_uint32),
                    "leaves": arr(b.leaves, b.n_leaves, ctypes.c_uint64),
                    "mats": arr(b.mats, b.n_mats, ctypes.c_uint8), "root": int(b.root),
                    "aabb": (tuple(b.aabb_lo), tuple(b.aabb_hi))}
        finally:
            lib().aok_blobfile_release(None, hd)

    def close(self):
        if self.h:
            lib().aok_blobfile_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scene:
    """A scene on a Context: pools sized for `built`, every blob uploaded."""

    def __init__(self, ctx: Context, spec, node_words: int, leaves: int, mat_bytes: int):
        self.ctx = ctx
        self.spec = spec
        self.grid = (spec.wx // spec.chunk, spec.wy // spec.chunk, spec.wz // spec.chunk)
        d = SceneDesc()
        for a in range(3):
            d.grid[a] = self.grid[a]
        d.chunk_res, d.n_lods, d.view_dist = spec.chunk, spec.n_lods, float(spec.view_dist)
        d.node_words, d.leaf_count, d.mat_bytes = max(1, node_words), max(1, leaves), max(1, mat_bytes)
        sid = ctypes.c_uint32()
        check(lib().aok_scene_create(ctx.h, ctypes.byref(d), ctypes.byref(sid)), "aok_scene_create")
        self.id = sid.value

    @classmethod
    def from_world(cls, ctx: Context, world, threads: int | None = None, built: BuiltWorld | None = None,
                   color_tol: float | None = None):
        bw = built or BuiltWorld(world, threads)
        sc = cls(ctx, world.spec, bw.node_words, bw.leaves, bw.mat_bytes)
        if color_tol is not None:
            sc.set_color_blocks(color_tol)
        sc.upload_built(bw)
        return sc

    def upload_built(self, bw: BuiltWorld):
        gx, gy, _ = self.grid
        for i in range(len(bw)):
            for lod in range(self.spec.n_lods):
                c, b = bw.blob(i, lod)
                self.upload(c % gx, (c // gx) % gy, c // (gx * gy), lod, b)

    def upload(self, cx, cy, cz, lod, blob: ChunkBlob):
        return check(lib().aok_scene_upload_chunk(self.ctx.h, self.id, cx, cy, cz, lod, ctypes.byref(blob)),
                     "aok_scene_upload_chunk")

    def evict(self, cx, cy, cz, lod):
        return check(lib().aok_scene_evict_chunk(self.ctx.h, self.id, cx, cy, cz, lod), "aok_scene_evict_chunk")

    def set_color_blocks(self, e_c: float):
        """Colour-block tolerance of later uploads (aok_scene_set_color_blocks; < 0: raw arrays)."""
        return check(lib().aok_scene_set_color_blocks(self.ctx.h, self.id, float(e_c)), "aok_scene_set_color_blocks")

    def usage(self) -> dict:
        """Resident bytes per device pool (aok_scene_usage)."""
        a = (ctypes.c_uint64 * 4)()
        check(lib().aok_scene_usage(self.ctx.h, self.id, a), "aok_scene_usage")
        return {"node_bytes": int(a[0]), "leaf_bytes": int(a[1]), "color_bytes": int(a[2]), "resident": int(a[3])}

    def destroy(self):
        if self.id:
            lib().aok_scene_destroy(self.ctx.h, self.id)
            self.id = 0


def alloc_frame(W: int, H: int, device="cuda"):
    """Caller-owned device output buffers: hit int32[H, W, 4], t float32[H, W]."""
    import torch
    hit = torch.empty((H, W, 4), dtype=torch.int32, device=device)
    t = torch.empty((H, W), dtype=torch.float32, device=device)
    return hit, t


def frame_of(hit, t) -> Frame:
    f = Frame()
    f.hit = hit.data_ptr()
    f.t = t.data_ptr()
    return f


def render(ctx: Context, scene: Scene, cam, tau: float, hit, t, stream=None):
    f = frame_of(hit, t)
    c = to_camera(cam)
    return check(lib().aok_render(ctx.h, scene.id, ctypes.byref(c), float(tau), ctypes.byref(f),
                                  _stream_handle(stream)), "aok_render")


def set_checked(ctx: Context, on: bool):
    """Checked casting: every pool index tested before its load (aok_set_checked)."""
    return check(lib().aok_set_checked(ctx.h, 1 if on else 0), "aok_set_checked")


def set_beam(ctx: Context, on: bool):
    """Beam pass before single-view casting: per 8x4 tile a lower bound on the
    distance of the solid voxels its rays can meet (aok_set_beam)."""
    return check(lib().aok_set_beam(ctx.h, 1 if on else 0), "aok_set_beam")


def beam_tune(ctx: Context, refine_tiles: int = 8, min_node_log2: int = 2, min_pixels: int = 1500000,
              queue_nodes: int = 0):
    """Refinement of the beam pass's walk, the smallest frame it runs for and
    the queue capacity per level (aok_beam_tune)."""
    return check(lib().aok_beam_tune(ctx.h, refine_tiles, min_node_log2, min_pixels, queue_nodes), "aok_beam_tune")


def beam_selected(ctx: Context, scene: Scene, cam, stream=None):
    """The beam pass alone for the scene's last selection (aok_beam_selected)."""
    c = to_camera(cam)
    return check(lib().aok_beam_selected(ctx.h, scene.id, ctypes.byref(c), _stream_handle(stream)),
                 "aok_beam_selected")


def select_beam(ctx: Context, scene: Scene, cam, tau: float, stream=None):
    """Selection and beam pass in one launch (aok_select_beam); then cast_selected."""
    c = to_camera(cam)
    return check(lib().aok_select_beam(ctx.h, scene.id, ctypes.byref(c), float(tau), _stream_handle(stream)),
                 "aok_select_beam")


def beam_info(ctx: Context):
    """The last beam pass (aok_beam_info; synchronises): (bounds as an int32
    array [tiles_y, tiles_x] in 2^-12 voxel units, nodes queued per level)."""
    xy = (ctypes.c_int32 * 2)()
    lv = (ctypes.c_uint32 * 16)()
    check(lib().aok_beam_info(ctx.h, None, 0, lv, xy), "aok_beam_info")
    b = np.zeros((xy[1], xy[0]), dtype=np.int32)
    check(lib().aok_beam_info(ctx.h, b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), b.size, None, None),
          "aok_beam_info")
    return b, [int(v) for v in lv]


def checked_errors(ctx: Context) -> int:
    """Read and clear the checked-casting error word (aok_checked_errors)."""
    e = ctypes.c_uint32()
    check(lib().aok_checked_errors(ctx.h, ctypes.byref(e)), "aok_checked_errors")
    return e.value


def render_tiles(ctx: Context, scene: Scene, cam, tau: float, hit, t, stream=None):
    """The frame of render() through the tile-chunk pipeline (aok_render_tiles)."""
    f = frame_of(hit, t)
    c = to_camera(cam)
    return check(lib().aok_render_tiles(ctx.h, scene.id, ctypes.byref(c), float(tau), ctypes.byref(f),
                                        _stream_handle(stream)), "aok_render_tiles")


TILE_STATS = ("regions_with_pairs", "items_marched_1", "items_culled_1", "items_marched_2", "items_culled_2",
              "pixel_traces", "pixel_skips", "cas_exhausted")


def tiles_stats(ctx: Context) -> dict:
    """Counters of the last render_tiles frame (aok_tiles_stats; synchronises)."""
    a = (ctypes.c_uint64 * 8)()
    check(lib().aok_tiles_stats(ctx.h, a), "aok_tiles_stats")
    return dict(zip(TILE_STATS, (int(v) for v in a)))


def tiles_forget(ctx: Context):
    return check(lib().aok_tiles_forget(ctx.h), "aok_tiles_forget")


def cast_selected(ctx: Context, scene: Scene, cam, hit, t, stream=None):
    """Cast with the table of the last select_chunks on this scene."""
    f = frame_of(hit, t)
    c = to_camera(cam)
    return check(lib().aok_cast_selected(ctx.h, scene.id, ctypes.byref(c), ctypes.byref(f), _stream_handle(stream)),
                 "aok_cast_selected")


def render_host(ctx: Context, scene: Scene, cam, tau: float, hit_host, t_host, stream=None):
    """Render into host tensors (pinned for asynchronous copies); returns after the copies."""
    c = to_camera(cam)
    return check(lib().aok_render_host(ctx.h, scene.id, ctypes.byref(c), float(tau), hit_host.data_ptr(),
                                       t_host.data_ptr(), _stream_handle(stream)), "aok_render_host")


def render_host_async(ctx: Context, scene: Scene, cam, tau: float, hit_host, t_host) -> int:
    """Enqueue a frame into host tensors (pinned); returns its ticket (aok_render_host_async)."""
    c = to_camera(cam)
    tk = ctypes.c_uint64()
    check(lib().aok_render_host_async(ctx.h, scene.id, ctypes.byref(c), float(tau), hit_host.data_ptr(),
                                      t_host.data_ptr(), ctypes.byref(tk)), "aok_render_host_async")
    return tk.value


def host_frame_wait(ctx: Context, ticket: int):
    return check(lib().aok_host_frame_wait(ctx.h, int(ticket)), "aok_host_frame_wait")


def render_counted(ctx: Context, scene: Scene, cam, tau: float, hit, t, counts, stream=None):
    f = frame_of(hit, t)
    c = to_camera(cam)
    return check(lib().aok_render_counted(ctx.h, scene.id, ctypes.byref(c), float(tau), ctypes.byref(f),
                                          counts.data_ptr(), _stream_handle(stream)), "aok_render_counted")


def select_chunks(ctx: Context, scene: Scene, cam, tau: float, lod_out=None, vis_out=None, stream=None,
                  count: bool = False):
    c = to_camera(cam)
    nvis = ctypes.c_uint32()
    check(lib().aok_select_chunks(ctx.h, scene.id, ctypes.byref(c), float(tau),
                                  lod_out.data_ptr() if lod_out is not None else None,
                                  vis_out.data_ptr() if vis_out is not None else None,
                                  ctypes.byref(nvis) if count else None, _stream_handle(stream)),
          "aok_select_chunks")
    return nvis.value if count else None


def read_bandwidth(ctx: Context, nbytes: int, reps: int = 20) -> float:
    """GB/s of 16-byte L2 reads over a device buffer of nbytes (aok_read_bandwidth)."""
    g = ctypes.c_double()
    check(lib().aok_read_bandwidth(ctx.h, int(nbytes), int(reps), ctypes.byref(g)), "aok_read_bandwidth")
    return g.value


def ray_dirs(ctx: Context, cam, dirs, stream=None):
    c = to_camera(cam)
    return check(lib().aok_ray_dirs(ctx.h, ctypes.byref(c), dirs.data_ptr(), _stream_handle(stream)),
                 "aok_ray_dirs")


# ---------------------------------------------------------------------------
# batched rendering, launch shape, serving
# ---------------------------------------------------------------------------
def make_view(scene: Scene, cam, tau: float, hit, t) -> View:
    v = View()
    v.scene = scene.id
    v.cam = to_camera(cam)
    v.lod_threshold_px = float(tau)
    v.frame.hit = hit.data_ptr()
    v.frame.t = t.data_ptr()
    return v


def _view_array(views):
    arr = (View * len(views))()
    for i, v in enumerate(views):
        arr[i] = v
    return arr


def render_batch(ctx: Context, views, stream=None):
    arr = _view_array(views)
    return check(lib().aok_render_batch(ctx.h, arr, len(views), _stream_handle(stream)), "aok_render_batch")


def autotune(ctx: Context, views, stream=None) -> float:
    arr = _view_array(views)
    ms = ctypes.c_float()
    check(lib().aok_autotune(ctx.h, arr, len(views), _stream_handle(stream), ctypes.byref(ms)), "aok_autotune")
    return ms.value


def set_launch(ctx: Context, ctas_per_sm: int = 0, threads: int = 0, packet_rays: int = 0):
    return check(lib().aok_set_launch(ctx.h, ctas_per_sm, threads, packet_rays), "aok_set_launch")


def get_launch(ctx: Context):
    a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    check(lib().aok_get_launch(ctx.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "aok_get_launch")
    return a.value, b.value, c.value


def set_tile(ctx: Context, tile_w: int):
    return check(lib().aok_set_tile(ctx.h, tile_w), "aok_set_tile")


def set_batch_kernel(ctx: Context, persistent: bool):
    return check(lib().aok_set_batch_kernel(ctx.h, int(persistent)), "aok_set_batch_kernel")


def set_batch_graph(ctx: Context, on: bool):
    """aok_set_batch_graph: replay a batch's launches as one CUDA graph (default) or launch them one by one."""
    return check(lib().aok_set_batch_graph(ctx.h, int(on)), "aok_set_batch_graph")


def set_single_view_kernel(ctx: Context, persistent: bool):
    return check(lib().aok_set_single_view_kernel(ctx.h, int(persistent)), "aok_set_single_view_kernel")


class _DevArray:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": None}


class Server:
    """Continuous-batching render server on a Context (aok_serve_*)."""

    def __init__(self, ctx: Context, max_slots: int = 64, max_batch: int = 32, n_streams: int = 2):
        self.ctx = ctx
        check(lib().aok_serve_start(ctx.h, max_slots, max_batch, n_streams), "aok_serve_start")
        self.shapes = {}

    def submit(self, scene: Scene, cam, tau: float) -> int:
        r = Request()
        r.scene = scene.id
        r.cam = to_camera(cam)
        r.lod_threshold_px = float(tau)
        tk = ctypes.c_uint64()
        check(lib().aok_serve_submit(self.ctx.h, ctypes.byref(r), ctypes.byref(tk)), "aok_serve_submit")
        self.shapes[tk.value] = (int(cam.H), int(cam.W))
        return tk.value

    def poll(self, ticket: int):
        f = Frame()
        return int(lib().aok_serve_poll(self.ctx.h, ticket, ctypes.byref(f))), f

    def wait(self, ticket: int, timeout_ms: int = 60000):
        f = Frame()
        st = int(lib().aok_serve_wait(self.ctx.h, ticket, timeout_ms, ctypes.byref(f)))
        return st, f

    def result(self, ticket: int, f: Frame):
        """torch views (hit int32[H, W, 4], t float32[H, W]) of a finished ticket's buffers."""
        import torch
        H, W = self.shapes[ticket]
        hit = torch.as_tensor(_DevArray(f.hit, (H, W, 4), "<i4"), device="cuda")
        t = torch.as_tensor(_DevArray(f.t, (H, W), "<f4"), device="cuda")
        return hit, t

    def times(self, ticket: int):
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        check(lib().aok_serve_times(self.ctx.h, ticket, ctypes.byref(a), ctypes.byref(b)), "aok_serve_times")
        return a.value, b.value

    def release(self, ticket: int) -> int:
        st = int(lib().aok_serve_release(self.ctx.h, ticket))
        if st == AOK_OK:
            self.shapes.pop(ticket, None)
        return st

    def stop(self):
        if self.ctx is not None and self.ctx.h:
            lib().aok_serve_stop(self.ctx.h)
        self.ctx = None
