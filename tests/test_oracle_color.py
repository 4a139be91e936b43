"""Oracle colour-block compression (Sec. 3.3) and its resolve (Sec. 3.5),
pinned by what the paper's description fixes: at e_c = 0 the blocks are the
runs of equal values; a tolerance covering the whole value range gives one
block with the average of all entries; hand-worked merges (including the
average drifting away from early entries); the greedy rule's invariants on
random arrays; the resolve equals a sorted search; scenes built with a
tolerance resolve every DFS index through the blocks."""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from worlds import MULTI16, TINY32


def rounded_mean(a):
    a = np.asarray(a, np.int64)
    return int((a.sum() + len(a) // 2) // len(a))


def runs(v):
    return np.flatnonzero(np.r_[True, v[1:] != v[:-1]])


@pytest.mark.parametrize("seed", range(6))
def test_zero_tolerance_is_runs_of_equal_values(seed):
    rng = np.random.default_rng(seed)
    vals = rng.integers(0, 256, 200).astype(np.uint8)
    lens = rng.integers(1, 9, 200)
    v = np.repeat(vals, lens)
    start, color = orc.color_blocks(v, 0.0)
    assert (start == runs(v)).all()
    assert (color == v[start]).all()


@pytest.mark.parametrize("seed", range(4))
def test_full_range_tolerance_is_one_block_with_the_mean(seed):
    v = np.random.default_rng(100 + seed).integers(0, 256, 1000).astype(np.uint8)
    start, color = orc.color_blocks(v, 1.0)
    assert start.tolist() == [0]
    assert int(color[0]) == rounded_mean(v)


def test_hand_worked_merges():
    # tol 2: 10 | 11 joins (|11-10| = 1), colour (21+1)//2 = 11 | 30 opens (|30-11| = 19) |
    # 31 joins 30 -> (61+1)//2 = 31 | 31 joins -> (92+1)//3 = 31
    s, c = orc.color_blocks(np.array([10, 11, 30, 31, 31], np.uint8), 2 / 255)
    assert s.tolist() == [0, 2] and c.tolist() == [11, 31]
    # tol 4, a drifting average: 100 | 104 joins (4 <= 4) -> 102 | 108 opens (6 > 4) |
    # 112 joins 108 -> 110 | 116 opens (6 > 4)
    s, c = orc.color_blocks(np.array([100, 104, 108, 112, 116], np.uint8), 4 / 255)
    assert s.tolist() == [0, 2, 4] and c.tolist() == [102, 110, 116]
    # tol 4, compared with the average, not the block's first entry: 100 | 103 joins -> 102 |
    # 106 joins (|106-102| = 4) -> (309+1)//3 = 103
    s, c = orc.color_blocks(np.array([100, 103, 106], np.uint8), 4 / 255)
    assert s.tolist() == [0] and c.tolist() == [103]
    # tol 3, compared with the average, not the previous entry: 100 | 103 joins -> 102 |
    # 106 opens (|106-102| = 4 > 3) | 109 joins 106 -> (215+1)//2 = 108
    s, c = orc.color_blocks(np.array([100, 103, 106, 109], np.uint8), 3 / 255)
    assert s.tolist() == [0, 2] and c.tolist() == [102, 108]
    # tol 1, round half up: 1 | 2 joins -> (3+1)//2 = 2 | 0 opens (|0-2| = 2 > 1)
    s, c = orc.color_blocks(np.array([1, 2, 0], np.uint8), 1 / 255)
    assert s.tolist() == [0, 2] and c.tolist() == [2, 0]
    # single entry, empty array
    s, c = orc.color_blocks(np.array([77], np.uint8), 0.05)
    assert s.tolist() == [0] and c.tolist() == [77]
    s, c = orc.color_blocks(np.zeros(0, np.uint8), 0.05)
    assert len(s) == 0 and len(c) == 0


@pytest.mark.parametrize("e_c", [0.0, 0.01, 0.05, 0.2])
def test_greedy_invariants(e_c):
    rng = np.random.default_rng(7)
    # a smooth ramp with noise plus jumps: many merges and many splits
    v = np.clip(np.cumsum(rng.integers(-3, 4, 5000)) // 4 + 128 + 60 * (rng.random(5000) < 0.01),
                0, 255).astype(np.uint8)
    tol = e_c * 255.0
    start, color = orc.color_blocks(v, e_c)
    assert start[0] == 0 and (np.diff(start.astype(np.int64)) > 0).all() and start[-1] < len(v)
    ends = np.r_[start[1:], len(v)].astype(np.int64)
    for b, (s0, s1) in enumerate(zip(start.astype(np.int64), ends)):
        blk = v[s0:s1].astype(np.int64)
        assert int(color[b]) == rounded_mean(blk)
        # every later entry was within tol of the block's running average when it joined
        cs = np.cumsum(blk)
        k = np.arange(1, len(blk))
        run_avg = (cs[:-1] + k // 2) // k
        assert (np.abs(blk[1:] - run_avg) <= tol).all()
        # a block opens only when its first entry is farther than tol from the previous colour
        if b > 0:
            assert abs(int(v[s0]) - int(color[b - 1])) > tol
    if e_c > 0:
        assert len(start) < len(runs(v))


def test_lookup_is_the_last_block_not_after_the_index():
    rng = np.random.default_rng(3)
    v = rng.integers(0, 256, 3000).astype(np.uint8)
    v[rng.random(3000) < 0.5] = 9
    start, color = orc.color_blocks(v, 0.02)
    for idx in list(range(0, 3000, 7)) + [0, 2999]:
        j = int(np.searchsorted(start, idx, side="right")) - 1
        assert orc.color_lookup(start, color, idx) == int(color[j])


@pytest.mark.parametrize("spec", [TINY32, MULTI16], ids=lambda s: s.name)
def test_scene_colour_arrays_resolve_through_blocks(spec):
    w = sg.World(spec)
    exact = orc.OracleScene(w)
    lossless = orc.OracleScene(w, color_tol=0.0)
    lossy = orc.OracleScene(w, color_tol=0.05)
    grid = exact.grid
    n_chunks = grid[0] * grid[1] * grid[2]
    changed = 0
    for lod in range(spec.n_lods):
        sel = np.full(n_chunks, lod, np.int8)
        for S in (exact, lossless, lossy):
            S.prepare(sel)
        for c in range(n_chunks):
            g0, _ = exact.dag(c, lod)
            if g0 is None or g0.n_mats == 0:
                continue
            m0 = np.ctypeslib.as_array(g0.mats, shape=(g0.n_mats,)).copy()
            g1, _ = lossless.dag(c, lod)
            g2, _ = lossy.dag(c, lod)
            m1 = np.ctypeslib.as_array(g1.mats, shape=(g1.n_mats,))
            m2 = np.ctypeslib.as_array(g2.mats, shape=(g2.n_mats,))
            assert (m1 == m0).all()
            start, color = orc.color_blocks(m0, 0.05)
            j = np.searchsorted(start, np.arange(len(m0)), side="right") - 1
            assert (m2 == color[j]).all()
            changed += int((m2 != m0).sum())
    assert changed > 0
    # casting: geometry identical, colours from the blocks
    cam = sg.orbit_camera(spec, 5, 40, 30)
    sel = exact.select(cam, 1.0)
    r0, r1, r2 = (S.cast(cam, sel) for S in (exact, lossless, lossy))
    for k in ("hit", "x", "y", "z", "lod", "normal", "amb"):
        assert (r0[k] == r1[k]).all() and (r0[k] == r2[k]).all()
    assert (r0["mat"] == r1["mat"]).all()
