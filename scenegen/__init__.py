"""Seeded synthetic voxel worlds and camera poses (input data for both sides).

This package holds only input generation: LOD-0 occupancy, uint8 materials
and camera poses.  It holds none of the rendering method's arithmetic.  Both
the CPU oracle (``oracle/``) and the GPU library consume it; neither of those
imports the other.

The paper measures on voxelised San Miguel, Sponza and Greenfield scenes
(Sec. 4), which are not available here; the procedural worlds below stand in
for them with the same character: terrain plus city blocks, open worlds up to
tens of billions of voxels.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libscenegen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile scenegen.c into an in-tree shared library (gcc, portable flags)."""
    src = os.path.join(_HERE, "scenegen.c")
    hdr = os.path.join(_HERE, "scenegen.h")
    with _lock:
        newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall",
                               "-fno-strict-aliasing", src, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("wx", ctypes.c_int32), ("wy", ctypes.c_int32),
                ("wz", ctypes.c_int32), ("octaves", ctypes.c_int32), ("period0", ctypes.c_int32),
                ("h_min", ctypes.c_int32), ("h_max", ctypes.c_int32), ("crust", ctypes.c_int32),
                ("n_boxes", ctypes.c_int32), ("box_min", ctypes.c_int32), ("box_max", ctypes.c_int32),
                ("box_hollow", ctypes.c_int32), ("mat_mode", ctypes.c_int32)]


class _Box(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_int32), ("y0", ctypes.c_int32), ("z0", ctypes.c_int32),
                ("sx", ctypes.c_int32), ("sy", ctypes.c_int32), ("sz", ctypes.c_int32),
                ("hollow", ctypes.c_int32)]


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64
        L.sg_create.restype = vp
        L.sg_create.argtypes = [ctypes.POINTER(_Params)]
        L.sg_create_with_boxes.restype = vp
        L.sg_create_with_boxes.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_Box)]
        L.sg_destroy.argtypes = [vp]
        L.sg_num_boxes.restype = i32
        L.sg_num_boxes.argtypes = [vp]
        L.sg_get_box.argtypes = [vp, i32, ctypes.POINTER(_Box)]
        L.sg_mix64.restype = u64
        L.sg_mix64.argtypes = [u64]
        L.sg_height.restype = i32
        L.sg_height.argtypes = [vp, i32, i32]
        L.sg_heights.argtypes = [vp, i32, i32, i32, i32, vp]
        L.sg_solid.restype = ctypes.c_int
        L.sg_solid.argtypes = [vp, i32, i32, i32]
        L.sg_material.restype = ctypes.c_uint8
        L.sg_material.argtypes = [vp, i32, i32, i32]
        L.sg_fill_bytes.restype = u64
        L.sg_fill_bytes.argtypes = [vp, i32, i32, i32, i32, i32, i32, vp]
        L.sg_fill_bits.restype = u64
        L.sg_fill_bits.argtypes = [vp, i32, i32, i32, i32, i32, i32, vp]
        L.sg_materials.argtypes = [vp, vp, ctypes.c_size_t, vp]
        L.sg_materials_block4.argtypes = [vp, i32, i32, i32, u64, vp]
        L.sg_fill_bits_z.argtypes = [vp, i32, i32, i32, i32, i32, i32, vp, vp]
        L.sg_fill_bits_z.restype = ctypes.c_int
        _lib = L
    return _lib


@dataclass(frozen=True)
class WorldSpec:
    """A procedural world plus its chunking (chunk side ``chunk`` in LOD-0 voxels)."""
    name: str
    seed: int
    wx: int
    wy: int
    wz: int
    chunk: int
    n_lods: int
    octaves: int
    period0: int
    h_min: int
    h_max: int
    crust: int
    n_boxes: int
    box_min: int
    box_max: int
    box_hollow: int
    view_dist: float = 0.0  # 0 = unlimited
    mat_mode: int = 0       # 0: hashed material per voxel; 1: layered, coherent materials

    @property
    def grid(self):
        return (self.wx // self.chunk, self.wy // self.chunk, self.wz // self.chunk)


class World:
    """Handle on a generated world (C object); exposes dense fills and point queries."""

    def __init__(self, spec: WorldSpec, boxes=None):
        """boxes: optional list of (x0, y0, z0, sx, sy, sz, hollow) placed instead of the
        seeded ones (hand-made test scenes; spec.n_boxes is then ignored)."""
        if boxes is not None:
            from dataclasses import replace
            spec = replace(spec, n_boxes=len(boxes))
        self.spec = spec
        p = _Params(spec.seed, spec.wx, spec.wy, spec.wz, spec.octaves, spec.period0, spec.h_min,
                    spec.h_max, spec.crust, spec.n_boxes, spec.box_min, spec.box_max, spec.box_hollow,
                    spec.mat_mode)
        if boxes is None:
            self._h = lib().sg_create(ctypes.byref(p))
        else:
            arr = (_Box * max(1, len(boxes)))(*[_Box(*b) for b in boxes])
            self._h = lib().sg_create_with_boxes(ctypes.byref(p), arr)
        if not self._h:
            raise ValueError(f"bad world spec {spec}")

    @property
    def handle(self) -> int:
        return self._h

    def close(self):
        if self._h:
            lib().sg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def boxes(self):
        out = []
        b = _Box()
        for i in range(lib().sg_num_boxes(self._h)):
            lib().sg_get_box(self._h, i, ctypes.byref(b))
            out.append((b.x0, b.y0, b.z0, b.sx, b.sy, b.sz, b.hollow))
        return out

    def height(self, x: int, y: int) -> int:
        return lib().sg_height(self._h, x, y)

    def heights(self, x0, y0, nx, ny) -> np.ndarray:
        out = np.empty((ny, nx), dtype=np.int32)
        lib().sg_heights(self._h, x0, y0, nx, ny, out.ctypes.data)
        return out

    def solid(self, x, y, z) -> bool:
        return bool(lib().sg_solid(self._h, x, y, z))

    def material(self, x, y, z) -> int:
        return int(lib().sg_material(self._h, x, y, z))

    def dense(self, x0, y0, z0, nx, ny, nz) -> np.ndarray:
        """Occupancy as uint8 array indexed [z, y, x]."""
        out = np.empty((nz, ny, nx), dtype=np.uint8)
        lib().sg_fill_bytes(self._h, x0, y0, z0, nx, ny, nz, out.ctypes.data)
        return out

    def materials(self, xyz: np.ndarray) -> np.ndarray:
        xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
        out = np.empty(len(xyz), dtype=np.uint8)
        lib().sg_materials(self._h, xyz.ctypes.data, len(xyz), out.ctypes.data)
        return out

    def materials_block4(self, x0, y0, z0, mask: int, out: np.ndarray) -> np.ndarray:
        """Materials of the set bits of a 4x4x4 block mask written into out[64]."""
        assert out.dtype == np.uint8 and out.size == 64 and out.flags.c_contiguous
        lib().sg_materials_block4(self._h, x0, y0, z0, mask, out.ctypes.data)
        return out

    def fill_bits_z(self, x0, y0, z0, nx, ny, nz, out: np.ndarray):
        """Bit-packed occupancy into a zeroed uint64 buffer; returns (any, (z_lo, z_hi))."""
        assert out.dtype == np.uint64 and out.flags.c_contiguous
        zr = np.zeros(2, np.int32)
        r = lib().sg_fill_bits_z(self._h, x0, y0, z0, nx, ny, nz, out.ctypes.data, zr.ctypes.data)
        return int(r), (int(zr[0]), int(zr[1]))

    def fill_bits(self, x0, y0, z0, nx, ny, nz) -> tuple[int, np.ndarray]:
        out = np.empty(nx // 64 * ny * nz, np.uint64)
        n = lib().sg_fill_bits(self._h, x0, y0, z0, nx, ny, nz, out.ctypes.data)
        return int(n), out


# ---------------------------------------------------------------------------
# Workload recipes.  Sizes follow the five workloads: a 128^3 single chunk,
# a 4096^3 world of 8^3 chunks x 4 LODs, a 65536x65536x1024 open world,
# 64 uneven views of the 4096^3 world, and a 4-world serving mix.
# ---------------------------------------------------------------------------

SINGLE_128 = WorldSpec("single128", seed=1, wx=128, wy=128, wz=128, chunk=128, n_lods=1,
                       octaves=4, period0=64, h_min=16, h_max=96, crust=0,
                       n_boxes=20, box_min=4, box_max=24, box_hollow=0)

CITY_4096 = WorldSpec("city4096", seed=2, wx=4096, wy=4096, wz=4096, chunk=512, n_lods=4,
                      octaves=6, period0=1024, h_min=256, h_max=1536, crust=8,
                      n_boxes=4000, box_min=4, box_max=64, box_hollow=1)

# the city world with layered (coherent) materials: the colour-block workload
CITY_4096_LAYERED = replace(CITY_4096, name="city4096_layered", mat_mode=1)

OPEN_65536 = WorldSpec("open65536", seed=3, wx=65536, wy=65536, wz=1024, chunk=512, n_lods=4,
                       octaves=6, period0=4096, h_min=64, h_max=896, crust=8,
                       n_boxes=1_024_000, box_min=4, box_max=64, box_hollow=1, view_dist=16384.0)


def city(seed: int, side: int = 4096) -> WorldSpec:
    """City-style world (terrain crust + hollow blocks), heights scaled to the side."""
    s = side / 4096
    return replace(CITY_4096, name=f"city{side}_s{seed}", seed=seed, wx=side, wy=side, wz=side,
                   period0=int(1024 * s), h_min=int(256 * s), h_max=int(1536 * s),
                   n_boxes=int(4000 * s * s))


SERVE_WORLDS = (city(2), city(5), city(6, 2048), city(7, 2048))

RESOLUTIONS = ((320, 180), (640, 360), (1280, 720), (1920, 1080), (2560, 1440))


# ---------------------------------------------------------------------------
# Camera poses (seeded, platform-identical).
# ---------------------------------------------------------------------------

@dataclass
class Camera:
    """Pinhole camera.  origin in LOD-0 voxel units (multiples of 2^-8), R columns
    (right, up, back) as float32, tan_half_fovy float32, W x H pixels."""
    origin: np.ndarray
    R: np.ndarray
    tan_half_fovy: np.float32
    W: int
    H: int
    fovy_deg: float = 60.0


class Rng:
    """SplitMix64 stream (same integers on every platform)."""

    def __init__(self, seed: int):
        self.s = int(seed) & 0xFFFFFFFFFFFFFFFF

    def next(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        return z ^ (z >> 31)

    def uniform(self, a: float, b: float) -> float:
        return a + (b - a) * ((self.next() >> 11) * (1.0 / 9007199254740992.0))

    def randint(self, a: int, b: int) -> int:
        return a + self.next() % (b - a + 1)


def _q(x: float, bits: int) -> float:
    """Round to a multiple of 2^-bits (absorbs last-ulp libm differences)."""
    return math.floor(x * (1 << bits) + 0.5) / (1 << bits)


def _frame(forward) -> np.ndarray:
    f = np.asarray(forward, dtype=np.float64)
    f = f / np.linalg.norm(f)
    r = np.cross(f, [0.0, 0.0, 1.0])
    if np.linalg.norm(r) < 1e-9:
        r = np.array([1.0, 0.0, 0.0])
    r = r / np.linalg.norm(r)
    u = np.cross(r, f)
    R = np.stack([r, u, -f], axis=1)
    return np.array([[_q(v, 20) for v in row] for row in R], dtype=np.float32)


def make_camera(origin, forward, W, H, fovy_deg=60.0) -> Camera:
    o = np.array([_q(float(v), 8) for v in origin], dtype=np.float32)
    t = np.float32(_q(math.tan(math.radians(fovy_deg) / 2.0), 20))
    return Camera(o, _frame(forward), t, int(W), int(H), fovy_deg)


def orbit_camera(spec: WorldSpec, seed: int, W: int, H: int, radius=None, center=None) -> Camera:
    """Position on a sphere around the world centre, elevation U[20,60] deg, looking at it."""
    rng = Rng(seed)
    c = np.array(center if center is not None else (spec.wx / 2, spec.wy / 2, spec.wz * 0.375))
    rad = radius if radius is not None else 1.25 * spec.wx
    el = math.radians(rng.uniform(20.0, 60.0))
    az = rng.uniform(0.0, 2 * math.pi)
    o = c + rad * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    return make_camera(o, c - o, W, H)


def ground_camera(world: World, seed: int, W: int, H: int, lo_frac=0.125, hi_frac=0.875,
                  z_lo=16, z_hi=256, pitch=(-30.0, 5.0)) -> Camera:
    """Walker pose: x,y U[lo,hi]*side, z = h + U[z_lo,z_hi], redrawn if a solid voxel
    lies within 2 voxels; yaw U[0,2pi), pitch U[pitch]."""
    spec = world.spec
    rng = Rng(seed)
    for _ in range(1000):
        x = rng.uniform(lo_frac * spec.wx, hi_frac * spec.wx)
        y = rng.uniform(lo_frac * spec.wy, hi_frac * spec.wy)
        z = world.height(int(x), int(y)) + rng.uniform(z_lo, z_hi)
        yaw = rng.uniform(0.0, 2 * math.pi)
        pit = math.radians(rng.uniform(*pitch))
        if z + 3 >= spec.wz:
            continue
        ix, iy, iz = int(math.floor(x)), int(math.floor(y)), int(math.floor(z))
        clear = True
        for dz in range(-2, 3):
            for dy in range(-2, 3):
                for dx in range(-2, 3):
                    if world.solid(ix + dx, iy + dy, iz + dz):
                        clear = False
        if clear:
            fwd = (math.cos(pit) * math.cos(yaw), math.cos(pit) * math.sin(yaw), math.sin(pit))
            return make_camera((x, y, z), fwd, W, H)
    raise RuntimeError("no clear camera position found")


def batch_cameras(world: World, seed: int, n: int):
    """n walker poses with resolutions drawn uniformly from RESOLUTIONS."""
    rng = Rng(seed)
    cams = []
    for i in range(n):
        W, H = RESOLUTIONS[rng.randint(0, len(RESOLUTIONS) - 1)]
        cams.append(ground_camera(world, rng.next(), W, H))
    return cams


def path_cameras(world: World, seed: int, n_poses: int, W: int, H: int, n_waypoints: int = 10,
                 span: float = 6000.0, z_lo: float = 32.0, z_hi: float = 512.0, pitch=(-20.0, 0.0)):
    """A flight path: n_waypoints seeded waypoints (x, y inside a span x span square
    around a seeded centre, z = terrain + U[z_lo, z_hi]), linearly interpolated to
    n_poses poses looking along the direction of travel with a seeded pitch."""
    spec = world.spec
    rng = Rng(seed)
    cx = rng.uniform(0.25 * spec.wx, 0.75 * spec.wx)
    cy = rng.uniform(0.25 * spec.wy, 0.75 * spec.wy)
    wps = []
    for _ in range(n_waypoints):
        x = min(max(cx + rng.uniform(-span / 2, span / 2), 1.0), spec.wx - 1.0)
        y = min(max(cy + rng.uniform(-span / 2, span / 2), 1.0), spec.wy - 1.0)
        z = min(world.height(int(x), int(y)) + rng.uniform(z_lo, z_hi), spec.wz - 4.0)
        wps.append(np.array([x, y, z]))
    pit = [math.radians(rng.uniform(*pitch)) for _ in range(n_waypoints)]
    cams = []
    for i in range(n_poses):
        s = i * (n_waypoints - 1) / max(1, n_poses - 1)
        k = min(int(s), n_waypoints - 2)
        f = s - k
        p = wps[k] * (1 - f) + wps[k + 1] * f
        g = max(p[2], world.height(int(p[0]), int(p[1])) + 8.0)  # stay above the ground
        d = wps[k + 1] - wps[k]
        yaw = math.atan2(d[1], d[0])
        pt = pit[k] * (1 - f) + pit[k + 1] * f
        fwd = (math.cos(pt) * math.cos(yaw), math.cos(pt) * math.sin(yaw), math.sin(pt))
        cams.append(make_camera((p[0], p[1], g), fwd, W, H))
    return cams


OPEN_8192 = replace(OPEN_65536, name="open8192", seed=31, wx=8192, wy=8192, wz=1024, period0=2048,
                    n_boxes=16000, view_dist=3000.0)
