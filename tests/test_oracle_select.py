"""Pins of the oracle's LOD selection (Sec. 3.4, Eq. 1).

LODError = ChunkSize * StreamingFactor - |ChunkCenter - Camera|: subdivide when
> 0, load when < 0; the tie (== 0) loads.  The paper's recursive octree search
is compared with the per-chunk closed form, and exact tie positions (dyadic
values, so FP64 is exact) check the sign convention."""
import math

import numpy as np
import pytest

import oracle as orc


def test_exact_tie_loads_and_just_inside_subdivides():
    M, L, sf = 512, 2, 2.0
    # level-1 block (0,0,0) spans chunks 0..1, centre (512,512,512), S = 1024, S*SF = 2048
    at = np.array([512.0 + 2048.0, 512.0, 512.0], np.float32)
    inside = np.array([512.0 + 2048.0 - 2.0 ** -8, 512.0, 512.0], np.float32)
    assert orc.lod_loads(1, (0, 0, 0), M, at, sf)
    assert not orc.lod_loads(1, (0, 0, 0), M, inside, sf)
    assert (orc.select((2, 2, 2), M, L, at, sf) == 1).all()
    assert (orc.select((2, 2, 2), M, L, inside, sf) == 0).all()


def test_far_camera_gets_coarsest_and_near_camera_finest():
    M, L = 64, 4
    grid = (8, 8, 8)
    far = np.array([1e5, 1e5, 1e5], np.float32)
    assert (orc.select(grid, M, L, far, 2.0) == L - 1).all()
    # camera at the centre of chunk (3,3,3) with a large SF: every level subdivides
    cam = np.array([3.5 * M, 3.5 * M, 3.5 * M], np.float32)
    sel = orc.select(grid, M, L, cam, 50.0).reshape(8, 8, 8)
    assert (sel == 0).all()
    # with SF small everything loads at the top level
    assert (orc.select(grid, M, L, cam, 0.01) == L - 1).all()


def test_lod_grows_with_distance_along_a_line():
    M, L = 64, 4
    grid = (16, 1, 1)
    cam = np.array([2.0, 32.0, 32.0], np.float32)
    sel = orc.select(grid, M, L, cam, 1.0)
    assert sel[0] == 0 and (np.diff(sel.astype(int)) >= 0).all() and sel[-1] == L - 1


@pytest.mark.parametrize("grid,M,L", [((8, 8, 8), 512, 4), ((6, 5, 3), 64, 3), ((16, 16, 2), 512, 4),
                                      ((3, 7, 1), 32, 2), ((9, 2, 4), 16, 1)])
def test_recursive_equals_closed_form(grid, M, L):
    rng = np.random.default_rng(sum(grid) * 7 + M + L)
    ext = np.array(grid) * M
    for _ in range(300):
        o = (rng.random(3) * 1.6 - 0.3) * ext
        o = np.floor(o * 256) / 256
        sf = float(rng.uniform(0.2, 4.0))
        a = orc.select(grid, M, L, o.astype(np.float32), sf, recursive=False)
        b = orc.select(grid, M, L, o.astype(np.float32), sf, recursive=True)
        assert (a == b).all()
        assert a.min() >= 0 and a.max() <= L - 1


def test_chunks_of_one_block_share_the_level():
    # a selected level n applies to all (2^n)^3 chunks of its octree block
    M, L = 64, 4
    rng = np.random.default_rng(5)
    grid = (8, 8, 8)
    for _ in range(100):
        o = (rng.random(3) * 8 * M).astype(np.float32)
        sel = orc.select(grid, M, L, o, float(rng.uniform(0.5, 3))).reshape(8, 8, 8)  # [z,y,x]
        for z in range(8):
            for y in range(8):
                for x in range(8):
                    n = sel[z, y, x]
                    s = 1 << n
                    blk = sel[(z // s) * s:(z // s + 1) * s, (y // s) * s:(y // s + 1) * s,
                              (x // s) * s:(x // s + 1) * s]
                    assert (blk == n).all()


def test_streaming_factor_is_the_pixel_threshold():
    t = np.float32(math.tan(math.radians(30.0)))
    sf = orc.streaming_factor(1080, float(t), 1.0, 512)
    assert abs(sf - 1.8268) < 1e-4
    # at the cut-off distance S*SF an LOD-n voxel covers exactly tau pixels
    for n in range(4):
        for tau in (0.5, 1.0, 2.0):
            s = orc.streaming_factor(1080, float(t), tau, 512)
            d = (512 << n) * s
            pixels = (2 ** n) * 1080 / (2 * float(t)) / d
            assert abs(pixels - tau) < 1e-12
