"""Beam pass (ESVO's beam optimisation, made exact) through aok_set_beam:
every frame equals the frame without the pass bit for bit -- voxel, LOD,
material, normal, hit flag and distance -- and the oracle on every
non-ambiguous pixel; every tile's bound is at most the L-infinity distance
from the camera of every voxel hit in it; a camera matrix the pass cannot
invert turns it off (all bounds 0); on the benchmark's 4096^3 frame the pass
removes node visits."""
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

INT32_MAX = 2**31 - 1


@pytest.fixture(scope="module")
def ctx():
    c = aok.Context(0)
    aok.beam_tune(c, 8, 2, 0, 0)  # the pass on every frame size
    yield c
    aok.set_beam(c, False)
    c.close()


_scenes = {}


def scene_for(ctx, spec):
    key = (id(ctx), spec.name)
    if key not in _scenes:
        w = sg.World(spec)
        _scenes[key] = (w, aok.Scene.from_world(ctx, w, threads=16), orc.OracleScene(w))
    return _scenes[key]


def render(ctx, sc, cam, tau, beam):
    aok.set_beam(ctx, beam)
    hit, t = aok.alloc_frame(cam.W, cam.H)
    aok.render(ctx, sc, cam, tau, hit, t)
    torch.cuda.synchronize()
    return hit, t


def same(a, b):
    return torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32), b[1].view(torch.int32))


def check_bounds(ctx, cam, frame):
    """Every hit voxel's L-inf distance from the origin (2^-12 units) >= its tile's bound."""
    b, levels = aok.beam_info(ctx)
    assert b.shape == ((cam.H + 3) // 4, (cam.W + 7) // 8)
    assert all(v <= 1 << 20 for v in levels)  # no queue overflowed on these frames
    g = decode(*frame)
    O = np.round(cam.origin.astype(np.float64) * 4096).astype(np.int64)
    py, px = np.divmod(np.arange(cam.W * cam.H), cam.W)
    h = g["hit"] == 1
    lo = np.stack([g["x"], g["y"], g["z"]], 1).astype(np.int64) * 4096 - O
    hi = lo + (np.int64(4096) << g["lod"].astype(np.int64))[:, None]
    d = np.maximum(np.maximum(lo, -hi), 0).max(1)
    tb = b[py // 4, px // 8].astype(np.int64)
    assert (tb[h] <= d[h]).all(), int((tb[h] > d[h]).sum())
    # tiles whose rays all miss may hold any bound; the pass found something to skip
    return b, levels


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
def test_small_worlds_equal_and_oracle(ctx, case):
    spec, camf, tau = CASES[case]
    w, sc, S = scene_for(ctx, spec)
    cam = camf(w)
    off = render(ctx, sc, cam, tau, False)
    on = render(ctx, sc, cam, tau, True)
    assert same(off, on)
    b, _ = check_bounds(ctx, cam, on)
    compare(decode(*on), S.cast(cam, S.select(cam, tau), view_dist=spec.view_dist))


def test_entry_points_on_planes(ctx):
    """Origins on voxel and chunk planes, directions along two- and three-axis
    diagonals: restart points and chunk entries on several planes at once."""
    w, sc, S = scene_for(ctx, MULTI16)
    origins = [(16.0, 16.0, 27.0), (32.0, 32.0, 29.0), (48.0, 16.0, 26.0), (16.0, 24.5, 28.0)]
    dirs = [(1.0, 1.0, -1.0), (-1.0, -1.0, -1.0), (1.0, -1.0, -0.5), (1.0, 0.0, -1.0), (1.0, 1.0, -2.0),
            (2.0, -1.0, -1.0)]
    for o in origins:
        for f in dirs:
            for tau in (1.0, 6.0):
                cam = sg.make_camera(o, f, 33, 17)
                off = render(ctx, sc, cam, tau, False)
                on = render(ctx, sc, cam, tau, True)
                assert same(off, on), (o, f, tau)
                check_bounds(ctx, cam, on)
                compare(decode(*on), S.cast(cam, S.select(cam, tau), view_dist=MULTI16.view_dist), max_amb_frac=0.25,
                        min_pixels_checked=0)


def test_bounds_are_used(ctx):
    """On a walker view most tiles get a positive bound (geometry is not at the camera)."""
    w, sc, _ = scene_for(ctx, MED64)
    cam = sg.ground_camera(w, 9, 203, 117, z_lo=4, z_hi=40)
    render(ctx, sc, cam, 1.5, True)
    b, levels = aok.beam_info(ctx)
    assert (b > 0).mean() > 0.5
    assert levels[0] > 0 and levels[1] > 0  # the walk refined nodes below the chunk roots


def test_moving_camera_and_view_distance(ctx):
    spec = replace(MULTI32, name="multi32vd_beam", view_dist=45.0)
    w, sc, S = scene_for(ctx, spec)
    for seed in (4, 5, 6):
        cam = sg.ground_camera(w, seed, 64, 40, z_lo=4, z_hi=20)
        off = render(ctx, sc, cam, 1.0, False)
        on = render(ctx, sc, cam, 1.0, True)
        assert same(off, on)
        check_bounds(ctx, cam, on)
    orc_ref = S.cast(cam, S.select(cam, 1.0), view_dist=spec.view_dist)
    compare(decode(*on), orc_ref)
    w, sc, _ = scene_for(ctx, MED64)
    for cam in sg.path_cameras(w, 31, 6, 150, 100, n_waypoints=3, span=150.0, z_lo=4.0, z_hi=40.0):
        assert same(render(ctx, sc, cam, 1.0, False), render(ctx, sc, cam, 1.0, True))
        check_bounds(ctx, cam, render(ctx, sc, cam, 1.0, True))


def test_axis_aligned_and_degenerate_images(ctx):
    """Rays with zero direction components, 1-pixel-wide images, an origin on
    chunk planes and one next to the ground."""
    spec = MED64
    w, sc, S = scene_for(ctx, spec)
    cams = [sg.make_camera((100.25, 130.5, 120.0), fwd, 1, 1)
            for fwd in [(0.0, 0.0, -1.0), (1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (1.0, 1.0, -1.0)]]
    cams.append(sg.make_camera((100.25, 130.5, 120.0), (0.3, 0.2, -1.0), 7, 1))
    cams.append(sg.make_camera((128.0, 64.0, 100.0), (0.0, 0.0, -1.0), 9, 9))
    h = w.height(100, 130)
    cams.append(sg.make_camera((100.25, 130.5, h + 0.5), (1.0, 0.3, -0.2), 33, 17))  # just above the ground
    cams.append(sg.make_camera((100.25, 130.5, h - 2.5), (1.0, 0.3, 0.4), 16, 8))    # inside it
    for cam in cams:
        off = render(ctx, sc, cam, 1.0, False)
        on = render(ctx, sc, cam, 1.0, True)
        assert same(off, on)
        check_bounds(ctx, cam, on)


def test_camera_matrix_without_inverse(ctx):
    """Back column equal to the right column: the pass cannot project, every
    bound is 0 and nothing is skipped."""
    w, sc, _ = scene_for(ctx, MED64)
    cam = sg.ground_camera(w, 4, 48, 32, z_lo=4, z_hi=40)
    R = cam.R.copy()
    R[:, 2] = R[:, 0]
    cam = replace(cam, R=R)
    off = render(ctx, sc, cam, 1.0, False)
    on = render(ctx, sc, cam, 1.0, True)
    assert same(off, on)
    b, _ = aok.beam_info(ctx)
    assert (b == 0).all()


def test_city4096_1080p_equal_and_fewer_visits(ctx):
    """The benchmark's frame: equal output, fewer interior-node visits."""
    w, sc, _ = scene_for(ctx, sg.CITY_4096)
    cam = sg.ground_camera(w, 102, 1920, 1080)
    off = render(ctx, sc, cam, 1.0, False)
    on = render(ctx, sc, cam, 1.0, True)
    assert same(off, on)
    check_bounds(ctx, cam, on)
    visits = []
    for beam in (False, True):
        aok.set_beam(ctx, beam)
        hit, t = aok.alloc_frame(cam.W, cam.H)
        counts = torch.zeros(cam.W * cam.H * 3, dtype=torch.int32, device="cuda")
        aok.render_counted(ctx, sc, cam, 1.0, hit, t, counts)
        torch.cuda.synchronize()
        assert same(off, (hit, t))
        visits.append(int(counts.view(-1, 3)[:, 0].sum()))
    assert visits[1] < visits[0], visits
    # a far view with LOD 1-3 surfaces
    cam = sg.ground_camera(w, 8, 640, 360, z_lo=600, z_hi=900, pitch=(-20.0, -8.0))
    on = render(ctx, sc, cam, 1.0 / 3.0, True)
    assert same(render(ctx, sc, cam, 1.0 / 3.0, False), on)
    check_bounds(ctx, cam, on)


def test_streamed_open_world_path(ctx):
    """View distance + residency streaming (resident-LOD stand-ins): every pose equal."""
    from paper_2505_02017_gb300.stream import Streamer
    spec = sg.OPEN_8192
    w = sg.World(spec)
    sc = aok.Scene(ctx, spec, node_words=64 << 20, leaves=16 << 20, mat_bytes=1 << 30)
    st = Streamer(ctx, w, sc, threads=16)
    for cam in sg.path_cameras(w, 77, 5, 320, 180, n_waypoints=3, span=3000.0):
        st.update(cam, 1.0 / 3.0)
        off = render(ctx, sc, cam, 1.0 / 3.0, False)
        on = render(ctx, sc, cam, 1.0 / 3.0, True)
        assert same(off, on)
        check_bounds(ctx, cam, on)
    sc.destroy()


def test_beam_selected_then_cast(ctx):
    """aok_beam_selected + aok_cast_selected equal a render; a later selection
    or another camera makes the cast compute its own bounds."""
    w, sc, _ = scene_for(ctx, MED64)
    cam_a = sg.ground_camera(w, 4, 160, 90, z_lo=4, z_hi=40)
    cam_b = sg.ground_camera(w, 9, 160, 90, z_lo=4, z_hi=40)
    ref_a = render(ctx, sc, cam_a, 1.0, False)
    ref_b = render(ctx, sc, cam_b, 1.0, False)
    aok.set_beam(ctx, True)
    hit, t = aok.alloc_frame(cam_a.W, cam_a.H)
    aok.select_chunks(ctx, sc, cam_a, 1.0)
    aok.beam_selected(ctx, sc, cam_a)
    aok.cast_selected(ctx, sc, cam_a, hit, t)
    torch.cuda.synchronize()
    assert same(ref_a, (hit, t))
    # bounds of camera a, then a selection for camera b: recomputed
    aok.beam_selected(ctx, sc, cam_a)
    aok.select_chunks(ctx, sc, cam_b, 1.0)
    aok.cast_selected(ctx, sc, cam_b, hit, t)
    torch.cuda.synchronize()
    assert same(ref_b, (hit, t))
    # same selection, other camera: recomputed
    aok.select_chunks(ctx, sc, cam_a, 1.0)
    aok.beam_selected(ctx, sc, cam_a)
    aok.select_chunks(ctx, sc, cam_b, 1.0)
    aok.beam_selected(ctx, sc, cam_a)  # stale for cam_b
    aok.cast_selected(ctx, sc, cam_b, hit, t)
    torch.cuda.synchronize()
    assert same(ref_b, (hit, t))


def test_queue_overflow_same_output(ctx):
    """Queues far too small for the walk: parents stand in for the children
    that do not fit, the bounds stay below every hit, the frame is unchanged."""
    w, sc, _ = scene_for(ctx, MED64)
    cam = sg.ground_camera(w, 9, 203, 117, z_lo=4, z_hi=40)
    ref = render(ctx, sc, cam, 1.5, False)
    try:
        for cap in (1, 7, 40, 300):
            aok.beam_tune(ctx, 0, 2, 0, cap)  # refine everything, tiny queues
            out = render(ctx, sc, cam, 1.5, True)
            assert same(ref, out), cap
            b, _ = aok.beam_info(ctx)
            g = decode(*out)
            O = np.round(cam.origin.astype(np.float64) * 4096).astype(np.int64)
            py, px = np.divmod(np.arange(cam.W * cam.H), cam.W)
            h = g["hit"] == 1
            lo = np.stack([g["x"], g["y"], g["z"]], 1).astype(np.int64) * 4096 - O
            hi = lo + (np.int64(4096) << g["lod"].astype(np.int64))[:, None]
            d = np.maximum(np.maximum(lo, -hi), 0).max(1)
            assert (b[py // 4, px // 8].astype(np.int64)[h] <= d[h]).all(), cap
    finally:
        aok.beam_tune(ctx, 8, 2, 0, 0)


def test_checked_casting_with_the_pass(ctx):
    """Checked casting keeps the beam pass and tests the pass's node and leaf
    indices as well as the cast's: on several worlds, with ample and with
    overflowing queues, no index is out of range, the bounds stay below
    every hit and the frame equals the plain march's."""
    assert aok.checked_errors(ctx) == 0
    try:
        for spec, camf, tau in (CASES[2], CASES[4], CASES[6]):
            w, sc, _ = scene_for(ctx, spec)
            cam = camf(w)
            ref = render(ctx, sc, cam, tau, False)
            for cap in (0, 40):
                aok.beam_tune(ctx, 8, 2, 0, cap)
                aok.set_checked(ctx, True)
                try:
                    out = render(ctx, sc, cam, tau, True)
                finally:
                    aok.set_checked(ctx, False)
                assert aok.checked_errors(ctx) == 0, (spec.name, cap)
                assert same(ref, out), (spec.name, cap)
                b, _ = aok.beam_info(ctx)
                g = decode(*out)
                O = np.round(cam.origin.astype(np.float64) * 4096).astype(np.int64)
                py, px = np.divmod(np.arange(cam.W * cam.H), cam.W)
                h = g["hit"] == 1
                lo = np.stack([g["x"], g["y"], g["z"]], 1).astype(np.int64) * 4096 - O
                hi = lo + (np.int64(4096) << g["lod"].astype(np.int64))[:, None]
                d = np.maximum(np.maximum(lo, -hi), 0).max(1)
                assert (b[py // 4, px // 8].astype(np.int64)[h] <= d[h]).all(), (spec.name, cap)
                if cap == 0 and spec is MED64:
                    assert (b > 0).mean() > 0.5  # the checked pass bounds the walker view's tiles
    finally:
        aok.beam_tune(ctx, 8, 2, 0, 0)
        aok.set_beam(ctx, False)


def test_refinement_settings_same_output(ctx):
    """Any refinement setting gives the frame of the plain march."""
    w, sc, _ = scene_for(ctx, MED64)
    cam = sg.ground_camera(w, 9, 203, 117, z_lo=4, z_hi=40)
    ref = render(ctx, sc, cam, 1.5, False)
    try:
        for refine, lg in ((0, 2), (4, 2), (64, 3), (1 << 30, 9), (8, 16)):
            aok.beam_tune(ctx, refine, lg, 0, 0)
            out = render(ctx, sc, cam, 1.5, True)
            assert same(ref, out), (refine, lg)
            check_bounds(ctx, cam, out)
        # below the frame-size threshold the pass does not run: the last
        # pass's bounds stay, the frame is the plain march's
        b0, _ = aok.beam_info(ctx)
        cam2 = sg.ground_camera(w, 4, 203, 117, z_lo=4, z_hi=40)
        ref2 = render(ctx, sc, cam2, 1.5, False)
        aok.beam_tune(ctx, 8, 2, cam2.W * cam2.H + 1, 0)
        assert same(ref2, render(ctx, sc, cam2, 1.5, True))
        assert (aok.beam_info(ctx)[0] == b0).all()
    finally:
        aok.beam_tune(ctx, 8, 2, 0, 0)


def test_batch_with_beam_equals_plain(ctx):
    """Batched rendering with the beam pass (one pass for all views of a
    group): every view equals its plain single-view render; views of two
    worlds, mixed sizes, one camera without a usable inverse."""
    w1, sc1, _ = scene_for(ctx, MED64)
    w2, sc2, _ = scene_for(ctx, MULTI32)
    cams = [(sc1, sg.ground_camera(w1, s, W, H, z_lo=4, z_hi=40)) for s, W, H in
            ((4, 160, 90), (9, 203, 117), (11, 64, 48), (12, 1, 1))]
    cams += [(sc2, sg.ground_camera(w2, s, W, H, z_lo=4, z_hi=20)) for s, W, H in ((4, 64, 40), (5, 97, 33))]
    bad = sg.ground_camera(w1, 13, 48, 32, z_lo=4, z_hi=40)
    R = bad.R.copy()
    R[:, 2] = R[:, 0]
    cams.append((sc1, replace(bad, R=R)))
    refs = [render(ctx, sc, cam, 1.0, False) for sc, cam in cams]
    aok.set_beam(ctx, True)
    outs = [aok.alloc_frame(cam.W, cam.H) for _, cam in cams]
    views = [aok.make_view(sc, cam, 1.0, h, t) for (sc, cam), (h, t) in zip(cams, outs)]
    aok.render_batch(ctx, views)
    torch.cuda.synchronize()
    for i, (ref, out) in enumerate(zip(refs, outs)):
        assert same(ref, out), i


def test_served_with_beam_equals_plain(ctx):
    """The server runs the beam pass for its batches (per-request bound
    pyramids, passes on several streams one after another): every served
    frame equals the plain render."""
    w1, sc1, _ = scene_for(ctx, MED64)
    w2, sc2, _ = scene_for(ctx, MULTI32)
    reqs = [(sc1, sg.ground_camera(w1, s, 96 + 8 * (s % 5), 64 + 4 * (s % 3), z_lo=4, z_hi=40)) for s in range(20, 32)]
    reqs += [(sc2, sg.ground_camera(w2, s, 64, 40, z_lo=4, z_hi=20)) for s in range(4, 10)]
    refs = [render(ctx, sc, cam, 1.0, False) for sc, cam in reqs]
    aok.set_beam(ctx, True)
    srv = aok.Server(ctx, max_slots=16, max_batch=4, n_streams=3)
    try:
        tickets = [srv.submit(sc, cam, 1.0) for sc, cam in reqs]
        for i, tk in enumerate(tickets):
            st, f = srv.wait(tk, 60000)
            assert st == aok.AOK_OK, st
            assert same(refs[i], srv.result(tk, f)), i
            assert srv.release(tk) == aok.AOK_OK
    finally:
        srv.stop()


def test_random_cameras_equal(ctx):
    """Seeded random poses inside and outside the worlds, looking anywhere
    (axis-aligned and grazing directions included): beam on == beam off."""
    rng = sg.Rng(2024)
    for spec in (MULTI16, MED64):
        w, sc, _ = scene_for(ctx, spec)
        for k in range(24):
            o = (rng.uniform(-0.3, 1.3) * spec.wx, rng.uniform(-0.3, 1.3) * spec.wy, rng.uniform(-0.2, 1.2) * spec.wz)
            if k % 6 == 0:
                fwd = [(1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.0, 0.0, -1.0)][(k // 6) % 3]
            else:
                fwd = (rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-1, 0.3))
            cam = sg.make_camera(o, fwd, 24 + (k % 5) * 8, 16 + (k % 3) * 4, fovy_deg=30.0 + 20.0 * (k % 4))
            off = render(ctx, sc, cam, 1.0, False)
            on = render(ctx, sc, cam, 1.0, True)
            assert same(off, on), (spec.name, k)
            check_bounds(ctx, cam, on)


def test_pipelined_host_frames_with_beam(ctx):
    """aok_render_host_async: each slot's selection and beam pass run on the
    prep stream while the previous slot casts; every frame equals the plain
    render, for a sequence of poses longer than the pipeline."""
    w, sc, _ = scene_for(ctx, MED64)
    cams = sg.path_cameras(w, 31, 7, 150, 100, n_waypoints=3, span=150.0, z_lo=4.0, z_hi=40.0)
    refs = [render(ctx, sc, cam, 1.0, False) for cam in cams]
    aok.set_beam(ctx, True)
    hh = [torch.empty((c.H, c.W, 4), dtype=torch.int32, pin_memory=True) for c in cams]
    th = [torch.empty((c.H, c.W), dtype=torch.float32, pin_memory=True) for c in cams]
    tickets = [aok.render_host_async(ctx, sc, c, 1.0, h, t) for c, h, t in zip(cams, hh, th)]
    for tk in tickets:
        aok.host_frame_wait(ctx, tk)
    for i, (ref, h, t) in enumerate(zip(refs, hh, th)):
        assert torch.equal(ref[0].cpu(), h) and torch.equal(ref[1].cpu().view(torch.int32), t.view(torch.int32)), i


@pytest.mark.parametrize("spec", [MULTI16, MED64, replace(MULTI32, name="multi32vd_fused", view_dist=45.0)],
                         ids=lambda s: s.name)
def test_selection_inside_the_pass(ctx, spec):
    """The beam pass that selects the frame table as the first step of its
    walk (aok_render with the pass on, aok_select_beam) gives the frame of
    the selection kernel followed by the pass and the cast, bit for bit."""
    w, sc, _ = scene_for(ctx, spec)
    aok.set_beam(ctx, True)
    for seed in (3, 4, 9):
        cam = sg.ground_camera(w, seed, 203, 117, z_lo=3, z_hi=20)
        tau = 1.5
        ref = aok.alloc_frame(cam.W, cam.H)
        aok.select_chunks(ctx, sc, cam, tau)  # the selection kernel, then the pass, then the cast
        aok.beam_selected(ctx, sc, cam)
        aok.cast_selected(ctx, sc, cam, *ref)
        fused = aok.alloc_frame(cam.W, cam.H)
        aok.select_beam(ctx, sc, cam, tau)
        aok.cast_selected(ctx, sc, cam, *fused)
        rendered = aok.alloc_frame(cam.W, cam.H)
        aok.render(ctx, sc, cam, tau, *rendered)
        torch.cuda.synchronize()
        assert same(ref, fused) and same(ref, rendered), seed
    aok.set_beam(ctx, False)
    plain = aok.alloc_frame(cam.W, cam.H)  # without the pass: the selection kernel alone
    aok.select_beam(ctx, sc, cam, tau)
    aok.cast_selected(ctx, sc, cam, *plain)
    torch.cuda.synchronize()
    assert same(ref, plain)
