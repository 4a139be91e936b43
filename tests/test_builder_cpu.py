"""CPU checks of the product side that need no GPU: the native chunk builder
against the oracle's dense LOD grids and DAG node counts, the blob validator,
and the C ABI's exported symbols."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as orc
import paper_2505_02017_gb300 as aok
import scenegen as sg
from worlds import MED64, MULTI16, MULTI32

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def blob_arrays(b):
    nodes = np.ctypeslib.as_array(ctypes.cast(b.nodes, ctypes.POINTER(ctypes.c_uint32)), (b.n_node_words,)).copy() \
        if b.n_node_words else np.zeros(0, np.uint32)
    leaves = np.ctypeslib.as_array(ctypes.cast(b.leaves, ctypes.POINTER(ctypes.c_uint64)), (b.n_leaves,)).copy() \
        if b.n_leaves else np.zeros(0, np.uint64)
    mats = np.ctypeslib.as_array(ctypes.cast(b.mats, ctypes.POINTER(ctypes.c_uint8)), (b.n_mats,)).copy() \
        if b.n_mats else np.zeros(0, np.uint8)
    return nodes, leaves, mats


def decode_blob(b, res):
    """Expand a blob to dense occupancy/materials (test-side decoder)."""
    nodes, leaves, mats = blob_arrays(b)
    occ = np.zeros((res, res, res), np.uint8)
    mat = np.zeros((res, res, res), np.uint8)
    if b.n_node_words == 0:
        return occ, mat, {}
    counter = [0]
    per_level = {}

    def rec(node, x0, y0, z0, size, depth):
        per_level.setdefault(depth, set()).add(node)
        mask = int(nodes[node]) & 0xFF
        p = node + 2
        h = size // 2
        for o in range(8):
            if not (mask >> o) & 1:
                continue
            ch = int(nodes[p])
            p += 1
            cx, cy, cz = x0 + (o & 1) * h, y0 + ((o >> 1) & 1) * h, z0 + (o >> 2) * h
            if h == 4:
                per_level.setdefault("leaf", set()).add(ch)
                m = int(leaves[ch])
                for bit in range(64):
                    if (m >> bit) & 1:
                        x, y, z = cx + (bit & 3), cy + ((bit >> 2) & 3), cz + (bit >> 4)
                        occ[z, y, x] = 1
                        mat[z, y, x] = mats[counter[0]]
                        counter[0] += 1
            else:
                rec(ch, cx, cy, cz, h, depth + 1)

    rec(b.root, 0, 0, 0, res, 0)
    assert counter[0] == b.n_mats
    return occ, mat, {k: len(v) for k, v in per_level.items()}


@pytest.mark.parametrize("spec", [MULTI16, MULTI32, MED64], ids=lambda s: s.name)
def test_builder_matches_oracle_dense_and_node_counts(spec):
    w = sg.World(spec)
    bw = aok.BuiltWorld(w, threads=4)
    gx, gy, gz = spec.grid
    assert len(bw) == gx * gy * gz
    rng = np.random.default_rng(1)
    picks = rng.choice(len(bw), size=min(6, len(bw)), replace=False)
    nonempty = 0
    for i in picks:
        for lod in range(spec.n_lods):
            c, b = bw.blob(int(i), lod)
            cx, cy, cz = c % gx, (c // gx) % gy, c // (gx * gy)
            res = spec.chunk >> lod
            occ, mat = orc.chunk_dense(w, spec.chunk, cx, cy, cz, lod)
            docc, dmat, levels = decode_blob(b, res)
            assert (docc == occ).all(), (c, lod)
            assert (dmat == mat * occ).all(), (c, lod)
            if occ.any():
                nonempty += 1
                assert aok.validate_chunk(b, spec.chunk, lod) == aok.AOK_OK
                # same dedup as the oracle: unique nodes per level and unique leaves
                od = orc.OracleDag(occ, mat)
                lv = od.level_nodes()
                assert [levels[d] for d in range(od.n_int)] == lv[:-1]
                assert levels["leaf"] == lv[-1] == b.n_leaves
                # AABB of the solid voxels, chunk-local LOD-0 units
                zs, ys, xs = np.nonzero(occ)
                assert list(b.aabb_lo) == [int(xs.min()) << lod, int(ys.min()) << lod, int(zs.min()) << lod]
                assert list(b.aabb_hi) == [(int(xs.max()) + 1) << lod, (int(ys.max()) + 1) << lod,
                                           (int(zs.max()) + 1) << lod]
                # breadth-first layout: the root is the first node
                assert b.root == 0
            else:
                assert b.n_node_words == 0 and b.n_mats == 0
    assert nonempty > 0


def corrupt_variants(b, spec_chunk, lod):
    nodes, leaves, mats = blob_arrays(b)
    out = []

    def mk(n, l, m, root=b.root, lo=None, hi=None):
        c = aok.ChunkBlob()
        n = np.ascontiguousarray(n, np.uint32)
        l = np.ascontiguousarray(l, np.uint64)
        m = np.ascontiguousarray(m, np.uint8)
        c.nodes, c.n_node_words = n.ctypes.data, len(n)
        c.leaves, c.n_leaves = l.ctypes.data, len(l)
        c.mats, c.n_mats = m.ctypes.data, len(m)
        c.root = root
        for a in range(3):
            c.aabb_lo[a] = (lo or list(b.aabb_lo))[a]
            c.aabb_hi[a] = (hi or list(b.aabb_hi))[a]
        out.append((c, (n, l, m)))

    k = bin(int(nodes[b.root]) & 0xFF).count("1")
    n1 = nodes.copy(); n1[b.root + 2] = len(nodes) + 5; mk(n1, leaves, mats)           # pointer out of range
    n2 = nodes.copy(); n2[b.root] |= 0x100; mk(n2, leaves, mats)                        # reserved header bit
    n3 = nodes.copy(); n3[b.root + 1] += 1; mk(n3, leaves, mats)                        # wrong leaf count
    mk(nodes, leaves, mats[:-1])                                                         # material array too short
    mk(nodes, leaves, mats, root=len(nodes) + 1)                                        # root out of range
    mk(nodes, leaves, mats, hi=[spec_chunk + 1, 1, 1])                                  # AABB outside the chunk
    n4 = nodes.copy(); n4[b.root] = 0; mk(n4, leaves, mats)                             # empty mask
    return out, k


def test_validator_rejects_corrupt_blobs():
    spec = MULTI32
    w = sg.World(spec)
    bw = aok.BuiltWorld(w, threads=4)
    tested = 0
    for i in range(len(bw)):
        _, b = bw.blob(i, 0)
        if b.n_node_words == 0:
            continue
        assert aok.validate_chunk(b, spec.chunk, 0) == aok.AOK_OK
        variants, _ = corrupt_variants(b, spec.chunk, 0)
        for c, keep in variants:
            assert aok.validate_chunk(c, spec.chunk, 0) == aok.AOK_E_CORRUPT
        tested += 1
        if tested == 3:
            break
    assert tested == 3
    # wrong LOD for the blob's depth: node levels no longer line up
    _, b1 = bw.blob(0, 1)
    if b1.n_node_words:
        assert aok.validate_chunk(b1, spec.chunk, 0) != aok.AOK_OK
    # bad arguments
    assert aok.validate_chunk(b, 48, 0) == aok.AOK_E_INVALID


def test_abi_exports_every_declared_symbol():
    with open(os.path.join(ROOT, "include", "aok.h")) as f:
        text = f.read()
    names = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(aok_\w+)\s*\(", text, re.M))
    assert len(names) >= 20
    L = aok.lib()
    for n in sorted(names):
        assert hasattr(L, n), n


def test_chunk_source_blob_cache():
    """The procedural chunk source's blob cache: a (chunk, LOD) asked again is
    served without a build, a build also caches the coarser LODs, every blob
    equals the uncached build, the budget is kept by evicting the least
    recently used, and a blob still held outlives its eviction."""
    B = aok.blib()
    vp = ctypes.c_void_p
    B.aokb_source_build.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32,
                                    ctypes.POINTER(aok.ChunkBlob), ctypes.POINTER(vp)]
    B.aokb_source_release.argtypes = [vp, vp]
    spec = MED64
    w = sg.World(spec)
    plain = B.aokb_source_create(w.handle, spec.chunk, spec.n_lods)
    cached = B.aokb_source_create(w.handle, spec.chunk, spec.n_lods)
    B.aokb_source_set_cache(cached, 64 << 20)

    def stats(s):
        a = (ctypes.c_uint64 * 4)()
        B.aokb_source_stats(s, ctypes.byref(a))
        return list(a)

    def get(s, c, lod):
        b, h = aok.ChunkBlob(), vp()
        assert B.aokb_source_build(s, *c, lod, ctypes.byref(b), ctypes.byref(h)) == 0
        return b, h

    def same(a, b):
        return all(np.array_equal(x, y) for x, y in zip(blob_arrays(a), blob_arrays(b))) and a.root == b.root \
            and list(a.aabb_lo) == list(b.aabb_lo) and list(a.aabb_hi) == list(b.aabb_hi)

    gx, gy, gz = spec.grid
    c = (gx // 2, gy // 2, 0)
    refs = [get(plain, c, lod) for lod in range(spec.n_lods)]
    assert refs[0][0].n_node_words > 0
    b1, h1 = get(cached, c, 1)
    assert stats(cached)[:2] == [0, 1] and stats(cached)[3] == spec.n_lods - 1
    assert same(b1, refs[1][0])
    for lod in range(1, spec.n_lods):  # served from the cache, equal to the plain builds
        b, h = get(cached, c, lod)
        assert same(b, refs[lod][0])
        B.aokb_source_release(cached, h)
    assert stats(cached)[:2] == [spec.n_lods - 1, 1]
    b0, h0 = get(cached, c, 0)  # a finer LOD: a build
    assert same(b0, refs[0][0]) and stats(cached)[1] == 2
    # a budget below the region's LOD-0 blob: evicted, while the handle keeps it alive
    B.aokb_source_set_cache(cached, 1)
    st = stats(cached)
    assert st[2] == 0 and st[3] == 0
    assert same(b0, refs[0][0]) and same(b1, refs[1][0])
    for b, h in refs:
        B.aokb_source_release(plain, h)
    B.aokb_source_release(cached, h0)
    B.aokb_source_release(cached, h1)
    B.aokb_source_destroy(plain)
    B.aokb_source_destroy(cached)


def test_chunk_source_cache_under_concurrent_loaders():
    """Eight threads asking the cached source for overlapping (chunk, LOD)s at
    once, as the streamer's loaders do, with a budget small enough to evict
    while blobs are held: every blob equals the uncached build."""
    import threading
    B = aok.blib()
    vp = ctypes.c_void_p
    B.aokb_source_build.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32,
                                    ctypes.POINTER(aok.ChunkBlob), ctypes.POINTER(vp)]
    B.aokb_source_release.argtypes = [vp, vp]
    spec = MED64
    w = sg.World(spec)
    gx, gy, gz = spec.grid
    keys = [((x, y, z), lod) for x in range(gx) for y in range(gy) for z in range(gz) for lod in range(spec.n_lods)]
    plain = B.aokb_source_create(w.handle, spec.chunk, spec.n_lods)
    ref = {}
    for c, lod in keys:
        b, h = aok.ChunkBlob(), vp()
        assert B.aokb_source_build(plain, *c, lod, ctypes.byref(b), ctypes.byref(h)) == 0
        ref[(c, lod)] = (blob_arrays(b), b.root, tuple(b.aabb_lo), tuple(b.aabb_hi))
        B.aokb_source_release(plain, h)
    B.aokb_source_destroy(plain)
    cached = B.aokb_source_create(w.handle, spec.chunk, spec.n_lods)
    B.aokb_source_set_cache(cached, 256 << 10)  # a few blobs: evictions while others are held
    errors = []

    def loader(seed):
        rng = np.random.default_rng(seed)
        held = []
        for _ in range(60):
            c, lod = keys[int(rng.integers(len(keys)))]
            b, h = aok.ChunkBlob(), vp()
            if B.aokb_source_build(cached, *c, lod, ctypes.byref(b), ctypes.byref(h)) != 0:
                errors.append(("build", c, lod))
                continue
            held.append((c, lod, b, h))
            if len(held) > 3:  # keep a few blobs alive across later calls
                c0, l0, b0, h0 = held.pop(0)
                r = ref[(c0, l0)]
                got = (blob_arrays(b0), b0.root, tuple(b0.aabb_lo), tuple(b0.aabb_hi))
                if not (all(np.array_equal(x, y) for x, y in zip(got[0], r[0])) and got[1:] == r[1:]):
                    errors.append(("mismatch", c0, l0))
                B.aokb_source_release(cached, h0)
        for c0, l0, b0, h0 in held:
            B.aokb_source_release(cached, h0)

    th = [threading.Thread(target=loader, args=(s,)) for s in range(8)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    a = (ctypes.c_uint64 * 4)()
    B.aokb_source_stats(cached, ctypes.byref(a))
    B.aokb_source_destroy(cached)
    assert not errors, errors[:5]
    assert a[0] > 0 and a[1] > 0 and a[2] <= 256 << 10  # hits, builds, the budget kept
