"""Pins of the oracle's first-hit caster (Sec. 3.5 ray marching + colour resolve).

The FP64 hierarchical caster is compared with a brute-force caster that tests
every voxel of the dense LOD-cut grid (no DAG, no DFS index), on every pixel of
small worlds, with cameras outside and inside the world, forced mixed LOD
selections and a view distance.  Analytic cases pin the geometry, the normal
code and the distance; the materials are checked against the generator."""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from worlds import MULTI16, MULTI32, TINY32

FIELDS = ["x", "y", "z", "lod", "mat", "normal", "hit", "amb"]


def compare(a, b):
    for k in FIELDS:
        assert (a[k] == b[k]).all(), (k, np.nonzero(a[k] != b[k])[0][:10])
    h = a["hit"] == 1
    assert np.allclose(a["dist"][h], b["dist"][h], rtol=1e-12, atol=0)


def test_ray_dir_closed_forms():
    # W = H = 1: u = v = 0 exactly, so d = -(third column of R)
    cam = sg.make_camera((1.0, 2.0, 3.0), (0.3, -0.4, 0.5), 1, 1)
    assert (orc.ray_dir(cam, 0, 0) == -cam.R[:, 2]).all()
    # W = H = 2, dyadic R and t: every operation is exact
    cam.W, cam.H = 2, 2
    cam.tan_half_fovy = np.float32(0.5)
    cam.R = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    # pixel (0, 0): u = (1/2 - 1) * 0.5 = -0.25, v = (1 - 1/2) * 0.5 = 0.25, d = (u, v, -1)
    assert orc.ray_dir(cam, 0, 0).tolist() == [-0.25, 0.25, -1.0]
    assert orc.ray_dir(cam, 1, 1).tolist() == [0.25, -0.25, -1.0]
    # aspect W/H enters u only
    cam.W, cam.H = 4, 2
    assert orc.ray_dir(cam, 3, 0).tolist() == [0.75, 0.25, -1.0]


def test_analytic_straight_down_hit():
    # no terrain (h = 0), one floating box; aim straight down at its top face
    spec = sg.WorldSpec("box", seed=21, wx=32, wy=32, wz=32, chunk=32, n_lods=1, octaves=1, period0=8,
                        h_min=0, h_max=0, crust=0, n_boxes=1, box_min=3, box_max=3, box_hollow=0)
    w = sg.World(spec)
    bx, by, bz, sx, sy, sz, _ = w.boxes()[0]
    cam = sg.make_camera((bx + 1.5, by + 1.5, bz + sz + 7.25), (0.0, 0.0, -1.0), 1, 1)
    assert orc.ray_dir(cam, 0, 0).tolist() == [0.0, 0.0, -1.0]
    S = orc.OracleScene(w)
    r = S.cast(cam, np.zeros(1, np.int8))[0]
    assert r["hit"] == 1 and r["amb"] == 0
    assert (r["x"], r["y"], r["z"]) == (bx + 1, by + 1, bz + sz - 1)
    assert r["normal"] == 5  # entered through the +z face (d_z < 0)
    assert r["dist"] == 7.25
    assert r["mat"] == w.material(bx + 1, by + 1, bz + sz - 1)
    # the same ray through a face plane (x on a voxel boundary) is ambiguous
    cam2 = sg.make_camera((bx + 1.0, by + 1.5, bz + sz + 7.25), (0.0, 0.0, -1.0), 1, 1)
    assert S.cast(cam2, np.zeros(1, np.int8))[0]["amb"] == 1
    # aimed beside the box: a miss
    cam3 = sg.make_camera((bx + 10.5, by + 1.5, bz + sz + 7.25), (0.0, 0.0, -1.0), 1, 1)
    r3 = S.cast(cam3, np.zeros(1, np.int8))[0]
    assert r3["hit"] == 0 and r3["lod"] == 255 and np.isinf(r3["dist"])


def test_entry_through_an_edge_or_corner_takes_the_lowest_axis():
    """A ray entering its voxel through an edge or a corner crosses the lower
    faces of several axes at once; the entry face (normal) is the lowest of
    those axes, the distance is the common entry distance."""
    spec = sg.WorldSpec("box", seed=21, wx=32, wy=32, wz=32, chunk=32, n_lods=1, octaves=1, period0=8,
                        h_min=0, h_max=0, crust=0, n_boxes=1, box_min=3, box_max=3, box_hollow=0)
    w = sg.World(spec)
    bx, by, bz, sx, sy, sz, _ = w.boxes()[0]
    S = orc.OracleScene(w)
    top = bz + sz
    cases = [
        # x-z edge of the top face: faces -x (normal 0) and +z (normal 5) at once
        ((bx - 5.0, by + 1.5, top + 5.0), (1.0, 0.0, -1.0), (bx, by + 1, top - 1), 0),
        # y-z edge: faces -y (normal 2) and +z
        ((bx + 1.5, by - 4.0, top + 4.0), (0.0, 1.0, -1.0), (bx + 1, by, top - 1), 2),
        # +x side and top: faces +x (normal 1) and +z
        ((bx + sx + 3.0, by + 1.5, top + 3.0), (-1.0, 0.0, -1.0), (bx + sx - 1, by + 1, top - 1), 1),
        # corner: -x, -y and +z at once
        ((bx - 6.0, by - 6.0, top + 6.0), (1.0, 1.0, -1.0), (bx, by, top - 1), 0),
    ]
    for o, f, vox, normal in cases:
        cam = sg.make_camera(o, f, 1, 1)
        d = orc.ray_dir(cam, 0, 0).astype(np.float64)
        nz = np.abs(d[d != 0])
        assert (nz == nz[0]).all()  # equal |d| components: the faces are crossed at one instant
        r = S.cast(cam, np.zeros(1, np.int8))[0]
        assert r["hit"] == 1 and r["amb"] == 0
        assert (r["x"], r["y"], r["z"]) == vox
        assert r["normal"] == normal
        t = (top - o[2]) / d[2]  # the common entry parameter, from the z face
        assert abs(r["dist"] - t * np.linalg.norm(d)) <= 1e-12 * r["dist"]
        b = orc.cast_brute(w, 32, 1, np.zeros(1, np.int8), cam)[0]
        assert b["normal"] == normal and (b["x"], b["y"], b["z"]) == vox


def test_single_chunk_matches_brute_force():
    w = sg.World(TINY32)
    S = orc.OracleScene(w)
    for seed in (5, 6, 7):
        cam = sg.orbit_camera(TINY32, seed, 40, 30)
        for lod in (0, 1):
            sel = np.array([lod], np.int8)
            compare(S.cast(cam, sel), orc.cast_brute(w, 32, 2, sel, cam))


def test_multi_chunk_mixed_lods_match_brute_force():
    w = sg.World(MULTI16)
    S = orc.OracleScene(w)
    rng = np.random.default_rng(0)
    n = int(np.prod(S.grid))
    for seed in (1, 2):
        cam = sg.orbit_camera(MULTI16, seed, 36, 28, radius=80)
        sel = rng.integers(0, 2, n).astype(np.int8)
        compare(S.cast(cam, sel), orc.cast_brute(w, 16, 2, sel, cam))
    # camera inside the world (walker pose) and Eq. 1 selection
    cam = sg.ground_camera(w, 3, 40, 24, lo_frac=0.3, hi_frac=0.7, z_lo=3, z_hi=8)
    sel = S.select(cam, 2.0)
    assert len(set(sel.tolist())) == 2  # Eq. 1 mixes LOD 0 and 1 here
    compare(S.cast(cam, sel), orc.cast_brute(w, 16, 2, sel, cam))


def test_view_distance_and_three_lods():
    w = sg.World(MULTI32)
    S = orc.OracleScene(w)
    cam = sg.ground_camera(w, 4, 32, 20, z_lo=4, z_hi=20)
    sel = S.select(cam, 1.0)
    assert len(set(sel.tolist())) == 2  # Eq. 1 mixes LOD 0 and 1 here
    for vd in (0.0, 40.0):
        compare(S.cast(cam, sel, view_dist=vd), orc.cast_brute(w, 32, 3, sel, cam, view_dist=vd))
    sel3 = np.random.default_rng(1).integers(0, 3, len(sel)).astype(np.int8)
    compare(S.cast(cam, sel3, view_dist=60.0), orc.cast_brute(w, 32, 3, sel3, cam, view_dist=60.0))
    far = S.cast(cam, sel)
    near = S.cast(cam, sel, view_dist=40.0)
    # the view distance only turns far hits into misses
    clip = (far["hit"] == 1) & (far["dist"] > 40.0)
    assert (near["hit"][clip] == 0).all()
    keep = (far["hit"] == 1) & (far["dist"] <= 40.0) & (far["amb"] == 0)
    assert (near["x"][keep] == far["x"][keep]).all()


def test_hits_are_solid_generator_voxels_with_their_material():
    w = sg.World(MULTI32)
    S = orc.OracleScene(w)
    cam = sg.orbit_camera(MULTI32, 9, 48, 32, radius=150)
    sel = np.zeros(int(np.prod(S.grid)), np.int8)
    r = S.cast(cam, sel)
    h = np.nonzero(r["hit"] == 1)[0]
    assert len(h) > 100
    for i in h:
        assert w.solid(int(r["x"][i]), int(r["y"][i]), int(r["z"][i]))
        assert r["mat"][i] == w.material(int(r["x"][i]), int(r["y"][i]), int(r["z"][i]))


def test_visit_counts_are_consistent():
    w = sg.World(MULTI32)
    S = orc.OracleScene(w)
    cam = sg.orbit_camera(MULTI32, 9, 24, 16, radius=150)
    sel = S.select(cam, 1.5)
    r = S.cast(cam, sel)
    h = r["hit"] == 1
    # a hit needs at least a root, one interior level per further depth and its leaf block
    assert (r["v_leaf"][h] >= 1).all()
    assert (r["v_int"][h] >= 1).all()
    assert (r["resolve_bytes"][h] >= 1).all() and (r["resolve_bytes"][~h] == 0).all()
