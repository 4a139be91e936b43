"""Pins of the oracle SVDAG (Sec. 3.2 geometry, Sec. 3.3 DFS colour order).

The DAG is checked against the dense grid it encodes by means independent of
its builder: decompression, distinct-block counts from numpy, a sort-based
depth-first enumeration, leaf-count sums and the node word format."""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from worlds import MULTI32, TINY32


def random_grid(r, p, seed):
    rng = np.random.default_rng(seed)
    occ = (rng.random((r, r, r)) < p).astype(np.uint8)
    mat = rng.integers(0, 256, (r, r, r), dtype=np.uint8) * occ
    return occ, mat


def clustered_grid(r, seed):
    """Repeating structure so that dedup actually merges subtrees."""
    occ, mat = random_grid(r, 0.0, 0)
    rng = np.random.default_rng(seed)
    tile = (rng.random((4, 4, 4)) < 0.5).astype(np.uint8)
    for bz in range(r // 4):
        for by in range(r // 4):
            for bx in range(r // 4):
                if rng.random() < 0.4:
                    occ[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4] = tile
    mat = (rng.integers(0, 256, occ.shape, dtype=np.uint8) * occ).astype(np.uint8)
    return occ, mat


def distinct_blocks(occ, s):
    """Number of distinct non-empty s^3 blocks (numpy; no DAG involved)."""
    r = occ.shape[0]
    n = r // s
    b = occ.reshape(n, s, n, s, n, s).transpose(0, 2, 4, 1, 3, 5).reshape(n ** 3, s ** 3)
    b = b[b.any(axis=1)]
    if len(b) == 0:
        return 0
    return len(np.unique(np.packbits(b, axis=1), axis=0))


def dfs_sorted_materials(occ, mat):
    """Materials ordered by (octree path with octant x|y<<1|z<<2, then leaf bit x+4y+16z)."""
    r = occ.shape[0]
    zs, ys, xs = np.nonzero(occ)
    key = np.zeros(len(xs), np.int64)
    lev = r.bit_length() - 1
    for b in range(lev - 1, 1, -1):  # octree digits from the top down to 4^3 blocks
        dig = ((xs >> b) & 1) | (((ys >> b) & 1) << 1) | (((zs >> b) & 1) << 2)
        key = key * 8 + dig
    key = key * 64 + ((xs & 3) + 4 * (ys & 3) + 16 * (zs & 3))
    order = np.argsort(key, kind="stable")
    return mat[zs[order], ys[order], xs[order]]


def walk(dag):
    """Yield (node word index, depth) for every distinct node reachable from the root."""
    nodes = dag.nodes()
    seen = {}
    stack = [(dag.root, 0)]
    while stack:
        n, dpt = stack.pop()
        if n in seen:
            assert seen[n] == dpt, "node reused at two depths"
            continue
        seen[n] = dpt
        mask = int(nodes[n]) & 0xFF
        if dpt < dag.n_int - 1:
            for c in range(bin(mask).count("1")):
                stack.append((int(nodes[n + 2 + c]), dpt + 1))
    return seen


CASES = [("rand8", *random_grid(8, 0.3, 1)), ("rand16", *random_grid(16, 0.05, 2)),
         ("clust32", *clustered_grid(32, 3)), ("clust64", *clustered_grid(64, 4))]


@pytest.mark.parametrize("name,occ,mat", CASES, ids=[c[0] for c in CASES])
def test_roundtrip_counts_and_order(name, occ, mat):
    d = orc.OracleDag(occ, mat)
    o2, m2 = d.decode()
    assert (o2 == occ).all()
    assert (m2 == mat * occ).all()
    # per-level unique node counts == distinct non-empty blocks of that side
    r = occ.shape[0]
    lv = d.level_nodes()
    sides = [r >> k for k in range(d.n_int)] + [4]
    for k, s in enumerate(sides):
        assert lv[k] == distinct_blocks(occ, s), (k, s)
    # materials in depth-first order == sort by (octree path, leaf bit)
    assert (d.mats() == dfs_sorted_materials(occ, mat)).all()


@pytest.mark.parametrize("name,occ,mat", CASES, ids=[c[0] for c in CASES])
def test_node_format_and_leaf_counts(name, occ, mat):
    d = orc.OracleDag(occ, mat)
    nodes, leaves = d.nodes(), d.leaves()
    seen = walk(d)
    total_words = 0
    for n, dpt in seen.items():
        hdr = int(nodes[n])
        mask = hdr & 0xFF
        assert mask != 0 and hdr >> 8 == 0  # low 8 bits = child mask, rest reserved
        k = bin(mask).count("1")
        total_words += 2 + k
        kids = [int(nodes[n + 2 + c]) for c in range(k)]
        if dpt == d.n_int - 1:
            assert all(c < len(leaves) for c in kids)
            cnt = sum(bin(int(leaves[c])).count("1") for c in kids)
        else:
            cnt = sum(int(nodes[c + 1]) for c in kids)
        assert int(nodes[n + 1]) == cnt  # leaf count = sum of children's
    assert total_words == len(nodes)  # every word belongs to a reachable node
    assert int(nodes[d.root + 1]) == int(occ.sum())
    assert len(d.mats()) == int(occ.sum())


def test_dfs_index_is_a_bijection_onto_materials():
    occ, mat = clustered_grid(32, 7)
    d = orc.OracleDag(occ, mat)
    zs, ys, xs = np.nonzero(occ)
    idx = np.array([d.dfs_index(int(x), int(y), int(z)) for x, y, z in zip(xs, ys, zs)])
    assert sorted(idx.tolist()) == list(range(len(idx)))
    assert (d.mats()[idx] == mat[zs, ys, xs]).all()
    ez, ey, ex = np.nonzero(occ == 0)
    for i in range(0, len(ex), 97):
        assert d.dfs_index(int(ex[i]), int(ey[i]), int(ez[i])) == -1


def test_empty_and_full():
    occ = np.zeros((16, 16, 16), np.uint8)
    d = orc.OracleDag(occ, occ)
    assert d.empty and len(d.mats()) == 0
    occ = np.ones((16, 16, 16), np.uint8)
    mat = np.full_like(occ, 3)
    d = orc.OracleDag(occ, mat)
    assert d.level_nodes() == [1, 1, 1]  # full subtrees merge: one node per level
    assert len(d.nodes()) == 2 * (2 + 8)
    assert (d.mats() == 3).all() and len(d.mats()) == 16 ** 3


def test_generated_chunks_roundtrip_all_lods():
    w = sg.World(MULTI32)
    for (cx, cy, cz) in [(0, 0, 0), (1, 2, 0), (2, 1, 1)]:
        for lod in range(MULTI32.n_lods):
            occ, mat = orc.chunk_dense(w, MULTI32.chunk, cx, cy, cz, lod)
            if lod == 0:
                # LOD 0 equals the generator's own voxels and materials
                M = MULTI32.chunk
                ref = w.dense(cx * M, cy * M, cz * M, M, M, M)
                assert (occ == ref).all()
                zs, ys, xs = np.nonzero(occ)
                xyz = np.stack([xs + cx * M, ys + cy * M, zs + cz * M], 1)
                assert (mat[zs, ys, xs] == w.materials(xyz)).all()
            d = orc.OracleDag(occ, mat)
            o2, m2 = d.decode()
            assert (o2 == occ).all() and (m2 == mat * occ).all()


def test_tiny_world_fig2_style_region():
    # Fig. 2: a 2x2x2 region holding 4 voxels.  The caption is all that
    # survives; the smallest chunk the node format allows is 8^3, so the
    # region is embedded at the origin of an otherwise empty 8^3 chunk.
    occ = np.zeros((8, 8, 8), np.uint8)
    mat = np.zeros_like(occ)
    for i, (x, y, z) in enumerate([(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]):
        occ[z, y, x] = 1
        mat[z, y, x] = 10 + i
    d = orc.OracleDag(occ, mat)
    nodes, leaves = d.nodes(), d.leaves()
    # root: one child (octant 0), 4 voxels, one pointer; leaf bits 0, 1, 4, 16
    assert int(nodes[d.root]) == 1 and int(nodes[d.root + 1]) == 4
    assert int(leaves[int(nodes[d.root + 2])]) == (1 | 2 | 16 | 65536)
    assert d.mats().tolist() == [10, 11, 12, 13]
    assert TINY32.chunk == 32
