"""Tile-chunk pipeline (Sec. 3.5, Fig. 7) through aok_render_tiles: every
frame equals the per-ray chunk march's (aok_render) bit for bit -- voxel,
LOD, material, normal, hit flag and distance -- on the first frame of a scene
(no Hi-Z history), on repeated and moving views (with history), with a view
distance and on the benchmark's 4096^3 frame; and equals the oracle on every
non-ambiguous pixel."""
import ctypes
from dataclasses import replace

import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from gpu_util import compare, decode
from worlds import MED64, MULTI16, MULTI32, TINY32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2505_02017_gb300 as aok  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = aok.Context(0)
    yield c
    c.close()


_scenes = {}


def scene_for(ctx, spec):
    key = (id(ctx), spec.name)
    if key not in _scenes:
        w = sg.World(spec)
        _scenes[key] = (w, aok.Scene.from_world(ctx, w, threads=16), orc.OracleScene(w))
    return _scenes[key]


def march(ctx, sc, cam, tau):
    hit, t = aok.alloc_frame(cam.W, cam.H)
    aok.render(ctx, sc, cam, tau, hit, t)
    return hit, t


def tiles(ctx, sc, cam, tau):
    hit, t = aok.alloc_frame(cam.W, cam.H)
    aok.render_tiles(ctx, sc, cam, tau, hit, t)
    st = aok.tiles_stats(ctx)
    assert st["cas_exhausted"] == 0, st
    return (hit, t), st


def same(a, b):
    return torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32), b[1].view(torch.int32))


CASES = [
    (TINY32, lambda w: sg.orbit_camera(TINY32, 5, 40, 30), 1.0),
    (MULTI16, lambda w: sg.ground_camera(w, 3, 40, 24, lo_frac=0.3, hi_frac=0.7, z_lo=3, z_hi=8), 2.0),
    (MULTI16, lambda w: sg.orbit_camera(MULTI16, 1, 61, 47, radius=80), 2.0),
    (MULTI32, lambda w: sg.ground_camera(w, 4, 64, 40, z_lo=4, z_hi=20), 1.0),
    (MED64, lambda w: sg.ground_camera(w, 4, 160, 90, z_lo=4, z_hi=40), 4.0),
    (MED64, lambda w: sg.ground_camera(w, 9, 203, 117, z_lo=4, z_hi=40), 1.5),
    (MED64, lambda w: sg.orbit_camera(MED64, 3, 128, 96, radius=300), 2.0),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_small_worlds_equal_march_and_oracle(ctx, case):
    spec, camf, tau = CASES[case]
    w, sc, S = scene_for(ctx, spec)
    cam = camf(w)
    ref = march(ctx, sc, cam, tau)
    aok.tiles_forget(ctx)
    first, st1 = tiles(ctx, sc, cam, tau)
    assert same(ref, first)
    assert st1["items_culled_1"] == 0  # no history: pass 1 culls nothing
    again, st2 = tiles(ctx, sc, cam, tau)  # same view: the previous frame's Hi-Z is exact
    assert same(ref, again)
    assert st2["items_marched_1"] + st2["items_marched_2"] <= st1["items_marched_1"]
    orc_ref = S.cast(cam, S.select(cam, tau), view_dist=spec.view_dist)
    compare(decode(*first), orc_ref)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_small_worlds_with_beam_bounds(ctx, case):
    """The beam pass on for every frame size: its bounds cull pairs wholly
    nearer than every voxel a half tile's rays can meet and restart the rays
    of the others; the frames still equal the march's (which restarts too)
    and the oracle's."""
    spec, camf, tau = CASES[case]
    w, sc, S = scene_for(ctx, spec)
    cam = camf(w)
    aok.beam_tune(ctx, min_pixels=0)
    try:
        ref = march(ctx, sc, cam, tau)
        aok.tiles_forget(ctx)
        first, _ = tiles(ctx, sc, cam, tau)
        again, _ = tiles(ctx, sc, cam, tau)
    finally:
        aok.beam_tune(ctx)
    assert same(ref, first) and same(ref, again)
    compare(decode(*first), S.cast(cam, S.select(cam, tau), view_dist=spec.view_dist))


def test_moving_camera_with_history(ctx):
    """Hi-Z of the previous pose culls in pass 1; pass 2 repairs what it culled wrongly."""
    spec = MED64
    w, sc, _ = scene_for(ctx, spec)
    cams = sg.path_cameras(w, 31, 8, 150, 100, n_waypoints=3, span=150.0, z_lo=4.0, z_hi=40.0)
    aok.tiles_forget(ctx)
    culled = repaired = 0
    for cam in cams:
        ref = march(ctx, sc, cam, 1.0)
        out, st = tiles(ctx, sc, cam, 1.0)
        assert same(ref, out)
        culled += st["items_culled_1"]
        repaired += st["items_marched_2"]
    assert culled > 0


def test_view_distance(ctx):
    spec = replace(MULTI32, name="multi32vd_tiles", view_dist=45.0)
    w, sc, S = scene_for(ctx, spec)
    for seed in (4, 5, 6):
        cam = sg.ground_camera(w, seed, 64, 40, z_lo=4, z_hi=20)
        ref = march(ctx, sc, cam, 1.0)
        out, _ = tiles(ctx, sc, cam, 1.0)
        assert same(ref, out)
    orc_ref = S.cast(cam, S.select(cam, 1.0), view_dist=spec.view_dist)
    compare(decode(*out), orc_ref)
    assert (orc_ref["hit"] == 0).sum() > 0


def test_axis_aligned_and_degenerate_images(ctx):
    """Rays with zero direction components and 1-pixel-wide images: equal to the
    oracle on every non-ambiguous pixel, and to the march."""
    spec = MED64
    w, sc, S = scene_for(ctx, spec)
    cams = [sg.make_camera((100.25, 130.5, 120.0), fwd, 1, 1)
            for fwd in [(0.0, 0.0, -1.0), (1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (1.0, 1.0, -1.0)]]
    cams.append(sg.make_camera((100.25, 130.5, 120.0), (0.3, 0.2, -1.0), 7, 1))
    cams.append(sg.make_camera((128.0, 64.0, 100.0), (0.0, 0.0, -1.0), 9, 9))  # origin on chunk planes
    for cam in cams:
        ref = march(ctx, sc, cam, 1.0)
        out, _ = tiles(ctx, sc, cam, 1.0)
        orc_ref = S.cast(cam, S.select(cam, 1.0))
        compare(decode(*out), orc_ref, max_amb_frac=0.5)
        ok = orc_ref["amb"] == 0
        g, m = decode(*out), decode(*ref)
        for k in ("hit", "x", "y", "z", "lod", "mat", "normal"):
            assert (g[k][ok] == m[k][ok]).all(), k


def test_city4096_1080p_equals_march(ctx):
    """The benchmark's frame: 4096^3 world, 1920x1080, tau = 1; first frame and
    steady state."""
    spec = sg.CITY_4096
    w, sc, _ = scene_for(ctx, spec)
    cam = sg.ground_camera(w, 102, 1920, 1080)
    ref = march(ctx, sc, cam, 1.0)
    aok.tiles_forget(ctx)
    out1, st1 = tiles(ctx, sc, cam, 1.0)
    assert same(ref, out1)
    out2, st2 = tiles(ctx, sc, cam, 1.0)
    assert same(ref, out2)
    assert st2["items_culled_1"] > 0
    aok.set_beam(ctx, False)  # the pipeline without the beam pass's bounds
    try:
        aok.tiles_forget(ctx)
        out3, st3 = tiles(ctx, sc, cam, 1.0)
    finally:
        aok.set_beam(ctx, True)
    assert same(ref, out3)
    assert st3["items_marched_1"] > st1["items_marched_1"]  # the bounds culled pairs
    # a far view with LOD 1-3 surfaces
    cam = sg.ground_camera(w, 8, 640, 360, z_lo=600, z_hi=900, pitch=(-20.0, -8.0))
    assert same(march(ctx, sc, cam, 1.0 / 3.0), tiles(ctx, sc, cam, 1.0 / 3.0)[0])


def test_streamed_open_world_path(ctx):
    """View distance + residency streaming: every pose of a path equals the march."""
    from paper_2505_02017_gb300.stream import Streamer
    spec = sg.OPEN_8192
    w = sg.World(spec)
    sc = aok.Scene(ctx, spec, node_words=64 << 20, leaves=16 << 20, mat_bytes=1 << 30)
    st = Streamer(ctx, w, sc, threads=16)
    for cam in sg.path_cameras(w, 77, 5, 320, 180, n_waypoints=3, span=3000.0):
        st.update(cam, 1.0 / 3.0)
        ref = march(ctx, sc, cam, 1.0 / 3.0)
        out, _ = tiles(ctx, sc, cam, 1.0 / 3.0)
        assert same(ref, out)
    sc.destroy()


def test_open_world_path_poses_equal_march(ctx):
    """Poses of the open-world benchmark path at its full resolution whose
    near chunk regions straddle the camera plane (some AABB corners behind
    it: whole-screen rectangles next to projected ones in one warp): every
    pose equals the march, with and without the previous pose's Hi-Z."""
    from paper_2505_02017_gb300.stream import Streamer
    spec = sg.OPEN_65536
    w = sg.World(spec)
    sc = aok.Scene(ctx, spec, node_words=512 << 20, leaves=256 << 20, mat_bytes=16 << 30)
    st = Streamer(ctx, w, sc, threads=16)
    cams = sg.path_cameras(w, 103, 300, 2560, 1440)
    try:
        aok.tiles_forget(ctx)
        for pose in (34, 35, 68, 72, 79):
            st.update(cams[pose], 1.0)
            ref = march(ctx, sc, cams[pose], 1.0)
            out, _ = tiles(ctx, sc, cams[pose], 1.0)
            assert same(ref, out), pose
        aok.tiles_forget(ctx)
        out, _ = tiles(ctx, sc, cams[79], 1.0)
        assert same(ref, out)
    finally:
        sc.destroy()


def test_limits_and_errors():
    c = aok.Context(0)
    L = aok.lib()
    assert L.aok_tiles_stats(c.h, (ctypes.c_uint64 * 8)()) == aok.AOK_E_INVALID  # no frame yet
    d = aok.SceneDesc()
    d.grid[0], d.grid[1], d.grid[2] = 64, 64, 17  # 69632 regions > AOK_TILES_MAX_CHUNKS
    d.chunk_res, d.n_lods = 8, 1
    d.node_words, d.leaf_count, d.mat_bytes = 1 << 16, 1 << 16, 1 << 16
    sid = ctypes.c_uint32()
    assert L.aok_scene_create(c.h, ctypes.byref(d), ctypes.byref(sid)) == aok.AOK_OK
    cam = aok.to_camera(sg.make_camera((10.0, 10.0, 100.0), (0.0, 0.0, -1.0), 8, 8))
    hit, t = aok.alloc_frame(8, 8)
    f = aok.frame_of(hit, t)
    assert L.aok_render_tiles(c.h, sid.value, ctypes.byref(cam), 1.0, ctypes.byref(f), None) == aok.AOK_E_INVALID
    assert L.aok_render_tiles(c.h, 12345, ctypes.byref(cam), 1.0, ctypes.byref(f), None) == aok.AOK_E_NOT_RESIDENT
    L.aok_scene_destroy(c.h, sid.value)
    c.close()
