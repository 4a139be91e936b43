"""CPU oracle for the chunked multi-LOD SVDAG primary-ray path (Aokana).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The GPU library never
imports this package and this package never imports the GPU library; both read
their input worlds from ``scenegen``.

The C source (``oracle.c``) is a plain restatement of the paper's definitions:
LOD aggregation (Sec. 3.4), SVDAG geometry compression (Sec. 3.2), depth-first
material indexing and colour-block compression (Sec. 3.3), Eq. 1 LOD
selection (Sec. 3.4) and the first-hit
query of the ray-marching and colour-resolve passes (Sec. 3.5), traced in FP64.

Parity pins (see tests/test_oracle_*.py): DAG decompression equals the dense
grid; per-level node counts equal brute-force distinct-block counts; leaf
counts add up; the DFS order equals a sort by (octree path, leaf bit); the LOD
rule on hand-made blocks; colour blocks == runs of equal values at e_c = 0,
one block with the rounded mean for e_c >= 1, hand-worked merges and the
greedy rule's invariants; Eq. 1 recursive == closed form plus exact tie cases;
the FP64 caster equals a brute-force every-voxel caster on small worlds and
analytic single-voxel cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

import scenegen

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plus the shared input generator) with gcc.

    -ffp-contract=off keeps every FP32/FP64 operation separately rounded, as
    the ray-generation and Eq. 1 definitions require."""
    srcs = [os.path.join(_HERE, "oracle.c"), os.path.join(_ROOT, "scenegen", "scenegen.c")]
    deps = srcs + [os.path.join(_HERE, "oracle.h"), os.path.join(_ROOT, "scenegen", "scenegen.h")]
    with _lock:
        newest = max(os.path.getmtime(f) for f in deps)
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-pthread",
                               "-ffp-contract=off", "-fno-fast-math", "-fno-strict-aliasing",
                               *srcs, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Dag(ctypes.Structure):
    _fields_ = [("nodes", ctypes.POINTER(ctypes.c_uint32)), ("n_words", ctypes.c_uint64),
                ("leaves", ctypes.POINTER(ctypes.c_uint64)), ("n_leaves", ctypes.c_uint64),
                ("mats", ctypes.POINTER(ctypes.c_uint8)), ("n_mats", ctypes.c_uint64),
                ("root", ctypes.c_uint32), ("res", ctypes.c_int32), ("n_int", ctypes.c_int32),
                ("level_nodes", ctypes.c_uint64 * 16)]


class Cam(ctypes.Structure):
    _fields_ = [("o", ctypes.c_float * 3), ("R", ctypes.c_float * 9), ("tan_half_fovy", ctypes.c_float),
                ("W", ctypes.c_int32), ("H", ctypes.c_int32)]


RESULT_DTYPE = np.dtype([("x", np.int32), ("y", np.int32), ("z", np.int32), ("lod", np.int32),
                         ("mat", np.int32), ("normal", np.int32), ("hit", np.int32), ("amb", np.int32),
                         ("dist", np.float64), ("v_int", np.uint32), ("v_leaf", np.uint32),
                         ("resolve_bytes", np.uint32), ("pad", np.uint32)])


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.or_lod_down.argtypes = [vp, vp, i32, vp, vp]
        L.or_dag_build.restype = ctypes.c_int
        L.or_dag_build.argtypes = [vp, vp, i32, ctypes.POINTER(Dag)]
        L.or_dag_free.argtypes = [ctypes.POINTER(Dag)]
        L.or_dag_decode.argtypes = [ctypes.POINTER(Dag), vp, vp]
        L.or_dag_dfs_index.restype = i64
        L.or_dag_dfs_index.argtypes = [ctypes.POINTER(Dag), i32, i32, i32]
        L.or_streaming_factor.restype = f64
        L.or_streaming_factor.argtypes = [i32, ctypes.c_float, f64, i32]
        L.or_lod_loads.restype = ctypes.c_int
        L.or_lod_loads.argtypes = [i32, vp, i32, vp, f64]
        L.or_select_closed.argtypes = [i32, i32, i32, i32, i32, vp, f64, vp]
        L.or_select_recursive.argtypes = [i32, i32, i32, i32, i32, vp, f64, vp]
        L.or_ray_dir.argtypes = [ctypes.POINTER(Cam), i32, i32, vp]
        L.or_scene_create.restype = vp
        L.or_scene_create.argtypes = [vp, i32, i32]
        L.or_scene_destroy.argtypes = [vp]
        L.or_scene_prepare.restype = ctypes.c_int
        L.or_scene_prepare.argtypes = [vp, vp, ctypes.c_int]
        L.or_scene_dag.restype = ctypes.POINTER(Dag)
        L.or_scene_dag.argtypes = [vp, i32, i32, vp]
        L.or_chunk_dense.argtypes = [vp, i32, i32, i32, i32, i32, vp, vp]
        L.or_cast.restype = ctypes.c_int
        L.or_cast.argtypes = [vp, vp, ctypes.POINTER(Cam), f64, vp, i64, vp, ctypes.c_int]
        L.or_color_blocks.restype = ctypes.c_uint64
        L.or_color_blocks.argtypes = [vp, ctypes.c_uint64, f64, vp, vp]
        L.or_color_lookup.restype = ctypes.c_uint8
        L.or_color_lookup.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint64]
        L.or_scene_set_color_tol.argtypes = [vp, f64]
        L.or_cast_brute.restype = ctypes.c_int
        L.or_cast_brute.argtypes = [vp, i32, i32, vp, ctypes.POINTER(Cam), f64, vp, i64, vp, ctypes.c_int]
        _lib = L
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# LOD aggregation / DAG
# ---------------------------------------------------------------------------

def lod_down(occ: np.ndarray, mat: np.ndarray):
    """One Sec. 3.4 aggregation step on cubic [z,y,x] uint8 grids."""
    r = occ.shape[0]
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    mat = np.ascontiguousarray(mat, dtype=np.uint8)
    o2 = np.empty((r // 2,) * 3, np.uint8)
    m2 = np.empty((r // 2,) * 3, np.uint8)
    lib().or_lod_down(occ.ctypes.data, mat.ctypes.data, r, o2.ctypes.data, m2.ctypes.data)
    return o2, m2


class OracleDag:
    """SVDAG of one dense cubic grid (Sec. 3.2/3.3)."""

    def __init__(self, occ: np.ndarray, mat: np.ndarray):
        occ = np.ascontiguousarray(occ, dtype=np.uint8)
        mat = np.ascontiguousarray(mat, dtype=np.uint8)
        self.res = occ.shape[0]
        self._d = Dag()
        if lib().or_dag_build(occ.ctypes.data, mat.ctypes.data, self.res, ctypes.byref(self._d)) != 0:
            raise ValueError("resolution must be a power of two >= 8")

    def __del__(self):
        try:
            lib().or_dag_free(ctypes.byref(self._d))
        except Exception:
            pass

    @property
    def empty(self) -> bool:
        return self._d.n_words == 0

    @property
    def root(self) -> int:
        return int(self._d.root)

    @property
    def n_int(self) -> int:
        return int(self._d.n_int)

    def nodes(self) -> np.ndarray:
        return np.ctypeslib.as_array(self._d.nodes, (self._d.n_words,)).copy() if self._d.n_words else np.zeros(0, np.uint32)

    def leaves(self) -> np.ndarray:
        return np.ctypeslib.as_array(self._d.leaves, (self._d.n_leaves,)).copy() if self._d.n_leaves else np.zeros(0, np.uint64)

    def mats(self) -> np.ndarray:
        return np.ctypeslib.as_array(self._d.mats, (self._d.n_mats,)).copy() if self._d.n_mats else np.zeros(0, np.uint8)

    def level_nodes(self):
        """Unique nodes per interior level (0 = root) followed by the unique leaf count."""
        return [int(self._d.level_nodes[i]) for i in range(self._d.n_int + 1)]

    def decode(self):
        occ = np.empty((self.res,) * 3, np.uint8)
        mat = np.empty((self.res,) * 3, np.uint8)
        lib().or_dag_decode(ctypes.byref(self._d), occ.ctypes.data, mat.ctypes.data)
        return occ, mat

    def dfs_index(self, x: int, y: int, z: int) -> int:
        return int(lib().or_dag_dfs_index(ctypes.byref(self._d), x, y, z))


# ---------------------------------------------------------------------------
# Selection and rays
# ---------------------------------------------------------------------------

def streaming_factor(H: int, tan_half_fovy: float, tau: float, M: int) -> float:
    return float(lib().or_streaming_factor(H, ctypes.c_float(tan_half_fovy), tau, M))


def lod_loads(n: int, b, M: int, origin, sf: float) -> bool:
    bb = np.asarray(b, np.int32)
    o = np.asarray(origin, np.float32)
    return bool(lib().or_lod_loads(n, bb.ctypes.data, M, o.ctypes.data, sf))


def select(grid, M: int, L: int, origin, sf: float, recursive: bool = False) -> np.ndarray:
    gx, gy, gz = grid
    out = np.full(gx * gy * gz, -1, np.int8)
    o = np.ascontiguousarray(origin, np.float32)
    fn = lib().or_select_recursive if recursive else lib().or_select_closed
    fn(gx, gy, gz, M, L, o.ctypes.data, sf, out.ctypes.data)
    return out


def to_cam(cam: scenegen.Camera) -> Cam:
    c = Cam()
    for i in range(3):
        c.o[i] = float(cam.origin[i])
    R = np.asarray(cam.R, np.float32)
    for i in range(3):
        for j in range(3):
            c.R[3 * i + j] = float(R[i, j])
    c.tan_half_fovy = float(cam.tan_half_fovy)
    c.W, c.H = cam.W, cam.H
    return c


def ray_dir(cam: scenegen.Camera, px: int, py: int) -> np.ndarray:
    d = np.empty(3, np.float32)
    c = to_cam(cam)
    lib().or_ray_dir(ctypes.byref(c), px, py, d.ctypes.data)
    return d


def ray_dirs(cam: scenegen.Camera) -> np.ndarray:
    """All pixel directions, [H, W, 3] float32."""
    c = to_cam(cam)
    out = np.empty((cam.H, cam.W, 3), np.float32)
    d = np.empty(3, np.float32)
    for py in range(cam.H):
        for px in range(cam.W):
            lib().or_ray_dir(ctypes.byref(c), px, py, d.ctypes.data)
            out[py, px] = d
    return out


# ---------------------------------------------------------------------------
# Colour blocks (Sec. 3.3)
# ---------------------------------------------------------------------------

def color_blocks(values: np.ndarray, e_c: float):
    """Block starts (uint64) and colours (uint8) of a uint8 colour array."""
    v = np.ascontiguousarray(values, np.uint8)
    start = np.zeros(max(1, len(v)), np.uint64)
    color = np.zeros(max(1, len(v)), np.uint8)
    nb = int(lib().or_color_blocks(v.ctypes.data, len(v), float(e_c), start.ctypes.data, color.ctypes.data))
    return start[:nb].copy(), color[:nb].copy()


def color_lookup(start: np.ndarray, color: np.ndarray, idx: int) -> int:
    s = np.ascontiguousarray(start, np.uint64)
    c = np.ascontiguousarray(color, np.uint8)
    return int(lib().or_color_lookup(s.ctypes.data, c.ctypes.data, len(s), int(idx)))


# ---------------------------------------------------------------------------
# Scene + casting
# ---------------------------------------------------------------------------

class OracleScene:
    """Per-(chunk, LOD) oracle DAGs of a scenegen world, built on demand."""

    def __init__(self, world: scenegen.World, M: int | None = None, L: int | None = None,
                 color_tol: float | None = None):
        """color_tol: colour-block tolerance e_c of the scene's colour arrays (None: exact)."""
        self.world = world
        self.M = M or world.spec.chunk
        self.L = L or world.spec.n_lods
        self.grid = (world.spec.wx // self.M, world.spec.wy // self.M, world.spec.wz // self.M)
        self._h = lib().or_scene_create(world.handle, self.M, self.L)
        if not self._h:
            raise ValueError("bad chunking")
        if color_tol is not None:
            lib().or_scene_set_color_tol(self._h, float(color_tol))

    def __del__(self):
        try:
            lib().or_scene_destroy(self._h)
        except Exception:
            pass

    def select(self, cam: scenegen.Camera, tau: float, recursive: bool = False) -> np.ndarray:
        sf = streaming_factor(cam.H, float(cam.tan_half_fovy), tau, self.M)
        return select(self.grid, self.M, self.L, cam.origin, sf, recursive)

    def prepare(self, lod_sel: np.ndarray, threads: int | None = None):
        sel = np.ascontiguousarray(lod_sel, np.int8)
        lib().or_scene_prepare(self._h, sel.ctypes.data, threads or default_threads())

    def dag(self, chunk: int, lod: int):
        bb = np.zeros(6, np.int32)
        p = lib().or_scene_dag(self._h, chunk, lod, bb.ctypes.data)
        return (p.contents if p else None), bb

    def cast(self, cam: scenegen.Camera, lod_sel: np.ndarray, pixels: np.ndarray | None = None,
             view_dist: float = 0.0, threads: int | None = None) -> np.ndarray:
        """Trace pixels ([n,2] px,py; default all, row-major).  Returns RESULT_DTYPE records."""
        if pixels is None:
            ys, xs = np.mgrid[0:cam.H, 0:cam.W]
            pixels = np.stack([xs.ravel(), ys.ravel()], axis=1)
        pix = np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
        out = np.zeros(len(pix), RESULT_DTYPE)
        sel = np.ascontiguousarray(lod_sel, np.int8)
        c = to_cam(cam)
        lib().or_cast(self._h, sel.ctypes.data, ctypes.byref(c), float(view_dist), pix.ctypes.data,
                      len(pix), out.ctypes.data, threads or default_threads())
        return out


def chunk_dense(world: scenegen.World, M: int, cx: int, cy: int, cz: int, lod: int):
    r = M >> lod
    occ = np.empty((r, r, r), np.uint8)
    mat = np.empty((r, r, r), np.uint8)
    lib().or_chunk_dense(world.handle, M, cx, cy, cz, lod, occ.ctypes.data, mat.ctypes.data)
    return occ, mat


def cast_brute(world: scenegen.World, M: int, L: int, lod_sel: np.ndarray, cam: scenegen.Camera,
               pixels: np.ndarray | None = None, view_dist: float = 0.0, threads: int | None = None) -> np.ndarray:
    if pixels is None:
        ys, xs = np.mgrid[0:cam.H, 0:cam.W]
        pixels = np.stack([xs.ravel(), ys.ravel()], axis=1)
    pix = np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
    out = np.zeros(len(pix), RESULT_DTYPE)
    sel = np.ascontiguousarray(lod_sel, np.int8)
    c = to_cam(cam)
    lib().or_cast_brute(world.handle, M, L, sel.ctypes.data, ctypes.byref(c), float(view_dist),
                        pix.ctypes.data, len(pix), out.ctypes.data, threads or default_threads())
    return out
