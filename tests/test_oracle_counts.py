"""Pins of the oracle's traversal counters, which define the algorithmic bytes
of the casting kernel's roofline: interior-node visits, leaf-block visits and
the material-resolve bytes (Sec. 3.2 node format, Sec. 3.3 depth-first index).

Definition (the oracle's reading): a chunk is entered iff the ray segment
[0, t_hit] (a miss: the whole ray) meets the closed box of its solid voxels;
its root is one interior visit, and every occupied cell below it whose closed
box the segment meets is one visit -- interior for a node, leaf for a 4x4x4
leaf block.  The resolve reads, per level of the hit's path, the counts of the
earlier occupied siblings (4 bytes each; 8 bytes each for leaf blocks, whose
mask is popcounted) plus the material byte.

Each scene below is a handful of voxels placed by hand in one 32^3 chunk, and
each ray points straight down, so that the expected numbers are counted by
hand from the voxel coordinates (comments give the count)."""
import numpy as np

import oracle as orc
import scenegen as sg
from worlds import HAND_CASES, hand_world


def scene(voxels, n_lods=1, size=1):
    w = hand_world(voxels, n_lods, size)
    return w, orc.OracleScene(w)


def down(S, x, y, lod=0, z=40.0):
    cam = sg.make_camera((x, y, z), (0.0, 0.0, -1.0), 1, 1)
    assert orc.ray_dir(cam, 0, 0).tolist() == [0.0, 0.0, -1.0]
    return S.cast(cam, np.array([lod], np.int8))[0]


def test_generator_places_hand_made_boxes():
    w, _ = scene([(9, 9, 9), (28, 28, 28)])
    assert w.boxes() == [(9, 9, 9, 1, 1, 1, 0), (28, 28, 28, 1, 1, 1, 0)]
    occ = w.dense(0, 0, 0, 32, 32, 32)
    assert occ.sum() == 2 and occ[9, 9, 9] == 1 and occ[28, 28, 28] == 1  # [z, y, x]


def test_hit_in_one_leaf_block():
    # a 2x2x2 cube at 9..10: every level holds one occupied cell on the path
    w, S = scene([(9, 9, 9)], size=2)
    r = down(S, 9.5, 10.5)
    assert r["hit"] == 1 and r["amb"] == 0
    assert (r["x"], r["y"], r["z"]) == (9, 10, 10) and r["dist"] == 40.0 - 11.0
    assert r["mat"] == w.material(9, 10, 10)
    # root (32^3), the 16^3 cell [0,16)^3, the 8^3 cell [8,16)^3; the leaf block [8,12)^3
    assert (r["v_int"], r["v_leaf"]) == (3, 1)
    # no earlier occupied sibling on the path: the material byte only
    assert r["resolve_bytes"] == 1


def test_chunk_aabb_met_but_no_occupied_cell():
    # cubes in root octants 0 and 7: the AABB [2,28]^3 spans both
    _, S = scene([(2, 2, 2), (26, 26, 26)], size=2)
    r = down(S, 20.5, 4.5)  # inside the AABB's footprint, through empty octants 5 and 1
    assert r["hit"] == 0 and r["amb"] == 0
    assert (r["v_int"], r["v_leaf"], r["resolve_bytes"]) == (1, 0, 0)  # the root only
    r = down(S, 30.5, 4.5)  # outside the AABB: the chunk is not entered
    assert (r["hit"], r["v_int"], r["v_leaf"], r["resolve_bytes"]) == (0, 0, 0, 0)


def test_earlier_siblings_and_cells_past_the_hit():
    vox = [(1, 1, 1), (20, 1, 1), (20, 20, 1),  # root octants 0, 1, 3
           (17, 17, 17), (28, 28, 20),          # octant 7: its sub-octants 0 and 3
           (25, 25, 25), (28, 28, 28)]          # octant 7, sub-octant 7: leaf blocks 0 and 7
    w, S = scene(vox)
    r = down(S, 28.5, 28.5)
    assert r["hit"] == 1 and r["amb"] == 0
    assert (r["x"], r["y"], r["z"]) == (28, 28, 28) and r["dist"] == 40.0 - 29.0 and r["normal"] == 5
    assert r["mat"] == w.material(28, 28, 28)
    # root, [16,32)^3, [24,32)^3 and the leaf block [28,32)^3; the cells of (28,28,20)
    # below the hit and of (25,25,25) beside the ray are not met by [0, t_hit]
    assert (r["v_int"], r["v_leaf"]) == (3, 1)
    # earlier occupied siblings: 3 at the root (4 B), 2 in [16,32)^3 (4 B), one
    # leaf block in [24,32)^3 (8 B), plus the material byte
    assert r["resolve_bytes"] == 1 + 3 * 4 + 2 * 4 + 1 * 8


def test_cells_met_before_the_hit():
    # (5,5,10) lies beside the ray (y in [5,6), the ray at y = 6.5) but its leaf
    # block [4,8)x[4,8)x[8,12) holds the ray's column
    w, S = scene([(5, 5, 10), (5, 6, 3)])
    r = down(S, 5.5, 6.5)
    assert r["hit"] == 1 and r["amb"] == 0
    assert (r["x"], r["y"], r["z"]) == (5, 6, 3) and r["dist"] == 36.0
    # root, [0,16)^3, the 8^3 cells [0,8)^2x[8,16) and [0,8)^3; both leaf blocks
    assert (r["v_int"], r["v_leaf"]) == (4, 2)
    assert r["resolve_bytes"] == 1
    assert r["mat"] == w.material(5, 6, 3)


def test_counts_at_lod1():
    # LOD 1 of a 2x2x2 cube at 8: one LOD-1 voxel; leaf blocks now cover 8^3 LOD-0 voxels
    w, S = scene([(8, 8, 8)], n_lods=2, size=2)
    r = down(S, 8.5, 9.5, lod=1)
    assert r["hit"] == 1 and r["amb"] == 0 and r["lod"] == 1
    assert (r["x"], r["y"], r["z"]) == (8, 8, 8) and r["dist"] == 40.0 - 10.0
    assert (r["v_int"], r["v_leaf"], r["resolve_bytes"]) == (2, 1, 1)  # root, [0,16)^3; leaf block [8,16)^3


def test_case_table_is_the_hand_counts():
    """The table the GPU counting test reuses holds the numbers asserted above."""
    for voxels, size, n_lods, lod, x, y, want in HAND_CASES:
        _, S = scene(voxels, n_lods, size)
        r = down(S, x, y, lod=lod)
        assert r["amb"] == 0
        assert (int(r["v_int"]), int(r["v_leaf"]), int(r["resolve_bytes"])) == want
