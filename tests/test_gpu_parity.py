"""GPU path vs oracle, element by element, through the C ABI (libaok.so).

Small worlds (several tiles per ray, ragged image sizes, cameras inside and
outside the world, mixed LODs, a view distance) on every pixel; the 128^3
single-chunk workload on every pixel; the 4096^3 world at 1920x1080 (the
benchmark's launch) on sampled pixels the oracle computes one by one."""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from gpu_util import compare, decode
from worlds import HAND_CASES, MED64, MULTI16, MULTI32, TINY32, hand_world

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # GPU tests are collected everywhere, run only with a device
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


def run(ctx, spec, cam, tau, view_dist=None, idx=None):
    w, sc, S = scene_for(ctx, spec)
    hit, t = aok.alloc_frame(cam.W, cam.H)
    aok.render(ctx, sc, cam, tau, hit, t)
    torch.cuda.synchronize()
    g = decode(hit, t)
    sel = S.select(cam, tau)
    if idx is None:
        ref = S.cast(cam, sel, view_dist=spec.view_dist)
    else:
        pix = np.stack([idx % cam.W, idx // cam.W], 1)
        ref = S.cast(cam, sel, pixels=pix, view_dist=spec.view_dist)
    return g, ref, sel


CASES = [
    (TINY32, lambda w: sg.orbit_camera(TINY32, 5, 40, 30), 1.0),
    (TINY32, lambda w: sg.orbit_camera(TINY32, 6, 37, 23), 4.0),
    (MULTI16, lambda w: sg.ground_camera(w, 3, 40, 24, lo_frac=0.3, hi_frac=0.7, z_lo=3, z_hi=8), 2.0),
    (MULTI16, lambda w: sg.orbit_camera(MULTI16, 1, 61, 47, radius=80), 2.0),
    (MULTI32, lambda w: sg.ground_camera(w, 4, 64, 40, z_lo=4, z_hi=20), 1.0),
    (MED64, lambda w: sg.ground_camera(w, 4, 160, 90, z_lo=4, z_hi=40), 4.0),
    (MED64, lambda w: sg.ground_camera(w, 9, 203, 117, z_lo=4, z_hi=40), 1.5),
    (MED64, lambda w: sg.orbit_camera(MED64, 3, 128, 96, radius=300), 2.0),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_small_worlds_every_pixel(ctx, case):
    spec, camf, tau = CASES[case]
    w, _, _ = scene_for(ctx, spec)
    cam = camf(w)
    g, ref, _ = run(ctx, spec, cam, tau)
    checked, amb = compare(g, ref)
    assert checked > 0.99 * cam.W * cam.H


def test_single_chunk_128_every_pixel(ctx):
    spec = sg.SINGLE_128
    cam = sg.orbit_camera(spec, 101, 256, 256, radius=160, center=(64, 64, 48))
    g, ref, _ = run(ctx, spec, cam, 1.0)
    checked, amb = compare(g, ref)
    assert (ref["hit"] == 1).mean() > 0.3


def test_view_distance(ctx):
    from dataclasses import replace
    spec = replace(MULTI32, name="multi32vd", view_dist=45.0)
    w, _, _ = scene_for(ctx, spec)
    cam = sg.ground_camera(w, 4, 64, 40, z_lo=4, z_hi=20)
    g, ref, _ = run(ctx, spec, cam, 1.0)
    compare(g, ref)
    assert (ref["hit"] == 0).sum() > 0


def test_degenerate_images_and_axis_aligned_rays(ctx):
    spec = MED64
    w, _, _ = scene_for(ctx, spec)
    # 1x1 image: u = v = 0, the ray is -R[:,2]; straight down is axis-aligned (d_x = d_y = 0)
    for fwd in [(0.0, 0.0, -1.0), (1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (1.0, 1.0, -1.0)]:
        cam = sg.make_camera((100.25, 130.5, 120.0), fwd, 1, 1)
        g, ref, _ = run(ctx, spec, cam, 1.0)
        compare(g, ref)
    cam = sg.make_camera((100.25, 130.5, 120.0), (0.3, 0.2, -1.0), 7, 1)
    g, ref, _ = run(ctx, spec, cam, 1.0)
    compare(g, ref)


# Origins on voxel and chunk planes (exact on the 2^-12 grid) and directions
# along diagonals of two or three axes or in an axis plane: entry points that
# lie on several planes at once, including a chunk's upper faces, where the
# traversal's exact ties (a plane crossed no later than the entry is passed)
# and its clamp to the chunk decide the cell.
PLANE_ORIGINS = [(16.0, 16.0, 27.0), (32.0, 32.0, 29.0), (48.0, 16.0, 26.0), (24.0, 40.0, 31.0), (16.0, 24.5, 28.0)]
PLANE_DIRS = [(1.0, 1.0, -1.0), (-1.0, -1.0, -1.0), (1.0, -1.0, -0.5), (1.0, 0.0, -1.0), (0.0, 1.0, -1.0),
              (1.0, 1.0, -2.0), (2.0, -1.0, -1.0), (1.0, 1.0, 0.0)]


def test_entry_points_on_planes(ctx):
    spec = MULTI16
    checked = total = 0
    for o in PLANE_ORIGINS:
        for f in PLANE_DIRS:
            for W, H in ((1, 1), (9, 7), (33, 17)):
                for tau in (1.0, 6.0):  # LOD 0 and LOD 1 chunks
                    cam = sg.make_camera(o, f, W, H)
                    g, ref, _ = run(ctx, spec, cam, tau)
                    c, _ = compare(g, ref, max_amb_frac=0.25, min_pixels_checked=0)
                    checked += c
                    total += W * H
    assert checked > 0.95 * total


def test_ray_directions_bitwise(ctx):
    w, _, _ = scene_for(ctx, MED64)
    cam = sg.ground_camera(w, 4, 97, 61, z_lo=4, z_hi=40)
    dirs = torch.empty((cam.H, cam.W, 3), dtype=torch.float32, device="cuda")
    aok.ray_dirs(ctx, cam, dirs)
    torch.cuda.synchronize()
    ref = orc.ray_dirs(cam)
    assert (dirs.cpu().numpy().view(np.uint32) == ref.view(np.uint32)).all()


def test_selection_matches_eq1(ctx):
    for spec, camf, tau in [(MED64, lambda w: sg.ground_camera(w, 4, 160, 90, z_lo=4, z_hi=40), 4.0),
                            (MULTI32, lambda w: sg.ground_camera(w, 4, 64, 40, z_lo=4, z_hi=20), 1.0)]:
        w, sc, S = scene_for(ctx, spec)
        cam = camf(w)
        n = int(np.prod(sc.grid))
        lod = torch.full((n,), -7, dtype=torch.int8, device="cuda")
        vis = torch.zeros((n,), dtype=torch.uint8, device="cuda")
        nvis = aok.select_chunks(ctx, sc, cam, tau, lod, vis, count=True)
        ref = S.select(cam, tau)
        assert (lod.cpu().numpy() == ref).all()
        v = vis.cpu().numpy()
        assert nvis == int(v.sum())
        # visible chunks are non-empty at their LOD; hit chunks are never culled
        S.prepare(ref)
        for c in np.nonzero(v)[0]:
            d, _ = S.dag(int(c), int(ref[c]))
            assert d is not None and d.n_words > 0


def test_traversal_counts_match_oracle(ctx):
    spec = MED64
    w, sc, S = scene_for(ctx, spec)
    cam = sg.ground_camera(w, 4, 120, 70, z_lo=4, z_hi=40)
    hit, t = aok.alloc_frame(cam.W, cam.H)
    counts = torch.zeros((cam.H, cam.W, 3), dtype=torch.int32, device="cuda")
    aok.render_counted(ctx, sc, cam, 2.0, hit, t, counts)
    torch.cuda.synchronize()
    c = counts.cpu().numpy().reshape(-1, 3)
    sel = S.select(cam, 2.0)
    ref = S.cast(cam, sel)
    ok = ref["amb"] == 0
    for j, k in enumerate(("v_int", "v_leaf", "resolve_bytes")):
        bad = np.nonzero(c[ok, j] != ref[k][ok])[0]
        assert len(bad) == 0, (k, len(bad), c[ok, j][bad[:5]].tolist(), ref[k][ok][bad[:5]].tolist())
    # the counted frame equals the plain one
    g = decode(hit, t)
    compare(g, ref)


def test_counts_on_hand_counted_scenes(ctx):
    """The counting kernel's visits and resolve bytes on the hand-counted scenes
    (the oracle's counter pins): straight-down rays through a few placed voxels."""
    for voxels, size, n_lods, lod, x, y, want in HAND_CASES:
        w = hand_world(voxels, n_lods, size)
        sc = aok.Scene.from_world(ctx, w, threads=2)
        cam = sg.make_camera((x, y, 40.0), (0.0, 0.0, -1.0), 1, 1)
        assert orc.OracleScene(w).select(cam, 1.0).tolist() == [lod]
        hit, t = aok.alloc_frame(1, 1)
        counts = torch.zeros((1, 1, 3), dtype=torch.int32, device="cuda")
        aok.render_counted(ctx, sc, cam, 1.0, hit, t, counts)
        torch.cuda.synchronize()
        assert tuple(counts.view(-1).tolist()) == want, (voxels, x, y)
        sc.destroy()


def test_city4096_1080p_every_pixel(ctx):
    """The benchmark's launch: 4096^3 world (8^3 chunks of 512^3, 4 LODs), 1920x1080,
    tau = 1, every pixel against the oracle; ambiguous pixels <= 0.01% of the frame."""
    spec = sg.CITY_4096
    w, _, _ = scene_for(ctx, spec)
    cam = sg.ground_camera(w, 102, 1920, 1080)
    g, ref, sel = run(ctx, spec, cam, 1.0)
    checked, amb = compare(g, ref, max_amb_frac=1e-4)
    assert checked >= 0.9999 * cam.W * cam.H
    assert len(set(sel.tolist())) >= 2


def test_city4096_far_view_mixed_lods(ctx):
    """High camera looking across the world: many LOD-1/2 hits."""
    spec = sg.CITY_4096
    w, _, _ = scene_for(ctx, spec)
    cam = sg.ground_camera(w, 8, 320, 180, z_lo=600, z_hi=900, pitch=(-20.0, -8.0))
    g, ref, sel = run(ctx, spec, cam, 1.0 / 3.0)
    compare(g, ref, max_amb_frac=2e-4)
    lods = ref["lod"][ref["hit"] == 1]
    assert len(np.unique(lods)) >= 3  # LOD 0, 1 and 2 surfaces in one frame


def test_abi_errors(ctx):
    w, sc, _ = scene_for(ctx, TINY32)
    cam = sg.orbit_camera(TINY32, 5, 8, 8)
    hit, t = aok.alloc_frame(8, 8)
    c = aok.to_camera(cam)
    c.origin[0] = 1.0 / 3.0  # not on the 2^-12 grid
    f = aok.frame_of(hit, t)
    import ctypes
    L = aok.lib()
    s = torch.cuda.current_stream().cuda_stream
    assert L.aok_render(ctx.h, sc.id, ctypes.byref(c), 1.0, ctypes.byref(f), s) == aok.AOK_E_INVALID
    c = aok.to_camera(cam)
    assert L.aok_render(ctx.h, 999999, ctypes.byref(c), 1.0, ctypes.byref(f), s) == aok.AOK_E_NOT_RESIDENT
    assert L.aok_render(ctx.h, sc.id, ctypes.byref(c), -1.0, ctypes.byref(f), s) == aok.AOK_E_INVALID
    f2 = aok.Frame()
    f2.hit = hit.data_ptr() + 4  # misaligned
    f2.t = t.data_ptr()
    assert L.aok_render(ctx.h, sc.id, ctypes.byref(c), 1.0, ctypes.byref(f2), s) == aok.AOK_E_INVALID
    # image sizes whose casting grid could not launch (more than 65535 rows of
    # 8-pixel blocks) or with 2^31 pixels are refused before any launch
    for W, H in ((1, 600000), (4096, 524288)):
        cb = aok.to_camera(sg.make_camera((10.0, 10.0, 10.0), (1.0, 0.5, -0.2), W, H))
        assert L.aok_render(ctx.h, sc.id, ctypes.byref(cb), 1.0, ctypes.byref(f), s) == aok.AOK_E_INVALID
    # a corrupt blob is rejected by the upload and nothing changes
    aok.render(ctx, sc, cam, 1.0, hit, t)
    torch.cuda.synchronize()
    g1 = decode(hit, t)
    bw = aok.BuiltWorld(w, threads=2)
    _, b = bw.blob(0, 0)
    bad = aok.ChunkBlob.from_buffer_copy(b)
    bad.n_mats = b.n_mats + 1
    assert L.aok_scene_upload_chunk(ctx.h, sc.id, 0, 0, 0, 0, ctypes.byref(bad)) == aok.AOK_E_CORRUPT
    aok.render(ctx, sc, cam, 1.0, hit, t)
    torch.cuda.synchronize()
    g2 = decode(hit, t)
    assert all((g1[k] == g2[k]).all() for k in ("hit", "x", "y", "z", "lod", "mat"))
    # a valid re-upload into the exactly sized pools replaces the chunk in place
    assert L.aok_scene_upload_chunk(ctx.h, sc.id, 0, 0, 0, 0, ctypes.byref(b)) == aok.AOK_OK
    aok.render(ctx, sc, cam, 1.0, hit, t)
    torch.cuda.synchronize()
    g3 = decode(hit, t)
    assert all((g1[k] == g3[k]).all() for k in ("hit", "x", "y", "z", "lod", "mat"))
    # a scene larger than the budget is refused
    small = aok.Context(0, budget_bytes=1 << 20)
    d = aok.SceneDesc()
    d.grid[0] = d.grid[1] = d.grid[2] = 1
    d.chunk_res, d.n_lods = 64, 1
    d.node_words, d.leaf_count, d.mat_bytes = 1 << 20, 1 << 20, 1 << 20
    sid = ctypes.c_uint32()
    assert L.aok_scene_create(small.h, ctypes.byref(d), ctypes.byref(sid)) == aok.AOK_E_OOM
    small.close()


def test_evict_renders_as_empty(ctx):
    from dataclasses import replace
    spec = replace(TINY32, name="tiny32evict")
    w = sg.World(spec)
    sc = aok.Scene.from_world(ctx, w, threads=2)
    cam = sg.orbit_camera(spec, 5, 32, 32)
    hit, t = aok.alloc_frame(32, 32)
    aok.render(ctx, sc, cam, 1.0, hit, t)
    torch.cuda.synchronize()
    assert decode(hit, t)["hit"].sum() > 0
    for lod in range(spec.n_lods):
        sc.evict(0, 0, 0, lod)
    aok.render(ctx, sc, cam, 1.0, hit, t)
    torch.cuda.synchronize()
    assert decode(hit, t)["hit"].sum() == 0
    sc.destroy()


def test_read_bandwidth_microbenchmark(ctx):
    l2 = aok.read_bandwidth(ctx, 32 << 20, 200)
    hbm = aok.read_bandwidth(ctx, 1 << 30, 3)
    assert 100.0 < hbm < l2 < 1e6, (hbm, l2)
    for nbytes, reps in ((8, 1), (1 << 20, 0)):
        with pytest.raises(aok.AokError) as ex:
            aok.read_bandwidth(ctx, nbytes, reps)
        assert ex.value.status == aok.AOK_E_INVALID
    used, budget = ctx.memory()
    with pytest.raises(aok.AokError) as ex:
        aok.read_bandwidth(ctx, budget - used + (1 << 20), 1)
    assert ex.value.status == aok.AOK_E_OOM


def test_maximum_world_extent(ctx):
    """A world 131072 voxels long, the largest extent the 2^-12 fixed-point
    origin allows (|o| < 2^17): cameras near its far end looking back along it
    (rays crossing 256 chunk regions) and toward its boundary, every pixel
    against the oracle; the tile-chunk pipeline renders the same frames."""
    spec = sg.WorldSpec("long131072", seed=41, wx=131072, wy=1024, wz=1024, chunk=512, n_lods=4, octaves=6,
                        period0=4096, h_min=32, h_max=300, crust=8, n_boxes=4000, box_min=4, box_max=64,
                        box_hollow=1)
    w, sc, S = scene_for(ctx, spec)
    x, y, z = 130990.25, 500.5, 900.0
    amb = n = 0
    for fwd in [(-1.0, 0.05, -0.3), (1.0, -0.1, -0.4), (-1.0, 0.0, -0.035)]:
        cam = sg.make_camera((x, y, z), fwd, 160, 90)
        g, ref, sel = run(ctx, spec, cam, 1.0)
        amb += compare(g, ref, max_amb_frac=1.0)[1]  # the ambiguous share is bounded over the three frames
        n += cam.W * cam.H
        hit, t = aok.alloc_frame(cam.W, cam.H)
        aok.render_tiles(ctx, sc, cam, 1.0, hit, t)
        torch.cuda.synchronize()
        gt = decode(hit, t)
        assert all((gt[k] == g[k]).all() for k in ("hit", "x", "y", "z", "lod", "mat", "normal"))
    assert amb <= 1e-4 * n, (amb, n)
    assert (g["hit"] == 1).sum() > 500 and (g["x"][g["hit"] == 1] < 131072 - 16 * 512).any()


def test_checked_casting_stays_in_bounds(ctx):
    """Checked casting (every node, leaf and colour index tested against the
    pool sizes before its load): on small worlds, the 4096^3 benchmark frame
    and a colour-block scene, no index is ever out of range and the frames
    equal the unchecked ones."""
    cases = [(CASES[i][0], CASES[i][1], CASES[i][2]) for i in (0, 2, 4, 5)]
    cases.append((sg.CITY_4096, lambda w: sg.ground_camera(w, 102, 640, 360), 1.0))
    cases.append((sg.CITY_4096, lambda w: sg.ground_camera(w, 8, 320, 180, z_lo=600, z_hi=900,
                                                           pitch=(-20.0, -8.0)), 1.0 / 3.0))
    assert aok.checked_errors(ctx) == 0
    for spec, camf, tau in cases:
        w, sc, _ = scene_for(ctx, spec)
        cam = camf(w)
        ref = aok.alloc_frame(cam.W, cam.H)
        aok.render(ctx, sc, cam, tau, *ref)
        aok.set_checked(ctx, True)
        try:
            out = aok.alloc_frame(cam.W, cam.H)
            aok.render(ctx, sc, cam, tau, *out)
            torch.cuda.synchronize()
        finally:
            aok.set_checked(ctx, False)
        assert aok.checked_errors(ctx) == 0, spec.name
        assert torch.equal(ref[0], out[0]) and torch.equal(ref[1].view(torch.int32), out[1].view(torch.int32))
    # colour blocks: the block structure's bounds are checked too
    from worlds import MED64_LAYERED
    wl = sg.World(MED64_LAYERED)
    scb = aok.Scene.from_world(ctx, wl, threads=8, color_tol=0.0)
    cam = sg.ground_camera(wl, 4, 160, 90, z_lo=4, z_hi=40)
    ref = aok.alloc_frame(cam.W, cam.H)
    aok.render(ctx, scb, cam, 2.0, *ref)
    aok.set_checked(ctx, True)
    out = aok.alloc_frame(cam.W, cam.H)
    aok.render(ctx, scb, cam, 2.0, *out)
    aok.set_checked(ctx, False)
    assert aok.checked_errors(ctx) == 0
    assert torch.equal(ref[0], out[0])
    scb.destroy()
