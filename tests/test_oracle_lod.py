"""Pins of the oracle's LOD aggregation (Sec. 3.4: density = 2, average value).

Each case is a hand-made block whose aggregate follows from the rule by
inspection, so a dropped term, a wrong threshold or a wrong reading of the
recursion fails one of them."""
import numpy as np

import oracle as orc


def grid(r, voxels):
    occ = np.zeros((r, r, r), np.uint8)
    mat = np.zeros((r, r, r), np.uint8)
    for (x, y, z, m) in voxels:
        occ[z, y, x] = 1
        mat[z, y, x] = m
    return occ, mat


def test_single_voxel_dropped():
    occ, mat = grid(2, [(1, 0, 1, 200)])
    o2, m2 = orc.lod_down(occ, mat)
    assert o2.shape == (1, 1, 1) and o2[0, 0, 0] == 0 and m2[0, 0, 0] == 0


def test_pair_kept_with_rounded_mean():
    # density = 2: two of eight children are enough; value = mean (10+13)/2 = 11.5 -> 12
    occ, mat = grid(2, [(0, 0, 0, 10), (1, 1, 1, 13)])
    o2, m2 = orc.lod_down(occ, mat)
    assert o2[0, 0, 0] == 1 and m2[0, 0, 0] == 12
    # mean of 1 and 2 is 1.5, rounds half up to 2
    occ, mat = grid(2, [(0, 1, 0, 1), (1, 0, 0, 2)])
    assert orc.lod_down(occ, mat)[1][0, 0, 0] == 2


def test_full_block_and_three_of_eight():
    occ = np.ones((2, 2, 2), np.uint8)
    mat = np.arange(8, dtype=np.uint8).reshape(2, 2, 2) * 10  # 0..70, mean 35
    o2, m2 = orc.lod_down(occ, mat)
    assert o2[0, 0, 0] == 1 and m2[0, 0, 0] == 35
    occ, mat = grid(2, [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 255)])  # mean 85
    assert orc.lod_down(occ, mat)[1][0, 0, 0] == 85


def test_only_solid_children_enter_the_mean():
    # empty children carry material 0 in the grid but must not count
    occ, mat = grid(2, [(0, 0, 0, 100), (1, 0, 0, 100)])
    mat[1, 1, 1] = 7  # garbage under an empty voxel
    assert orc.lod_down(occ, mat)[1][0, 0, 0] == 100


def test_recursive_not_direct_from_lod0():
    # eight isolated voxels, one per 2^3 block of a 4^3 region: LOD1 is empty
    # (each block has one voxel), hence LOD2 is empty although 8 >= 2 LOD-0
    # voxels lie in the LOD-2 cell.
    vox = [(2 * (o & 1), 2 * ((o >> 1) & 1), 2 * (o >> 2), 50) for o in range(8)]
    occ, mat = grid(4, vox)
    o1, m1 = orc.lod_down(occ, mat)
    assert o1.sum() == 0
    o2, _ = orc.lod_down(o1, m1)
    assert o2.sum() == 0
    # two full 2^3 blocks -> two LOD-1 voxels -> one LOD-2 voxel
    occ = np.zeros((4, 4, 4), np.uint8)
    occ[0:2, 0:2, 0:2] = 1
    occ[2:4, 2:4, 2:4] = 1
    mat = occ * 40
    o1, m1 = orc.lod_down(occ, mat)
    assert o1.sum() == 2
    o2, m2 = orc.lod_down(o1, m1)
    assert o2[0, 0, 0] == 1 and m2[0, 0, 0] == 40


def test_checkerboard_every_block_has_four():
    r = 8
    z, y, x = np.mgrid[0:r, 0:r, 0:r]
    occ = ((x + y + z) % 2 == 0).astype(np.uint8)
    mat = np.where(occ == 1, 9, 0).astype(np.uint8)
    o2, m2 = orc.lod_down(occ, mat)
    assert o2.all() and (m2 == 9).all()


def test_layout_is_x_fastest():
    # a pair in the 2^3 block at parent (x=1, y=0, z=0) must land at [0, 0, 1]
    occ, mat = grid(4, [(2, 0, 0, 5), (3, 1, 1, 5)])
    o2, _ = orc.lod_down(occ, mat)
    assert o2[0, 0, 1] == 1 and o2.sum() == 1


def test_monotone_in_occupancy():
    rng = np.random.default_rng(3)
    for _ in range(20):
        occ = (rng.random((8, 8, 8)) < 0.2).astype(np.uint8)
        more = occ | (rng.random((8, 8, 8)) < 0.1).astype(np.uint8)
        mat = np.zeros_like(occ)
        a, _ = orc.lod_down(occ, mat)
        b, _ = orc.lod_down(more, mat)
        assert (b >= a).all()
