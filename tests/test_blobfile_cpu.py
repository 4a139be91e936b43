"""Chunk-blob files (host only, no GPU): every stored (chunk, LOD) reads back
byte for byte; an absent entry reads as empty through the streaming source;
damage to the header, the index or an entry is detected by its checksum."""
import ctypes
import os

import numpy as np
import pytest

import scenegen as sg
from worlds import MULTI16, MULTI32

aok = pytest.importorskip("paper_2505_02017_gb300")


def built(spec):
    w = sg.World(spec)
    return w, aok.BuiltWorld(w, threads=4)


def blob_arrays(b):
    def arr(ptr, n, dt):
        return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(dt)), (n,)).copy() if n else np.zeros(0)
    return (arr(b.nodes, b.n_node_words, ctypes.c_uint32), arr(b.leaves, b.n_leaves, ctypes.c_uint64),
            arr(b.mats, b.n_mats, ctypes.c_uint8), int(b.root), (tuple(b.aabb_lo), tuple(b.aabb_hi)))


@pytest.mark.parametrize("spec", [MULTI16, MULTI32], ids=lambda s: s.name)
def test_round_trip(tmp_path, spec):
    w, bw = built(spec)
    path = str(tmp_path / "w.aokb")
    grid = (spec.wx // spec.chunk, spec.wy // spec.chunk, spec.wz // spec.chunk)
    n = aok.BlobFile.write(path, bw, grid, spec.chunk, spec.n_lods)
    f = aok.BlobFile(path)
    info = f.info()
    assert info == {"chunk_res": spec.chunk, "n_lods": spec.n_lods, "grid": grid, "entries": n}
    stored = 0
    for i in range(len(bw)):
        for lod in range(spec.n_lods):
            c, b = bw.blob(i, lod)
            nodes, leaves, mats, root, aabb = blob_arrays(b)
            if not b.n_node_words:
                with pytest.raises(aok.AokError) as ex:
                    f.read(c, lod)
                assert ex.value.status == aok.AOK_E_NOT_RESIDENT
                continue
            r = f.read(c, lod)
            assert (r["nodes"] == nodes).all() and (r["leaves"] == leaves).all() and (r["mats"] == mats).all()
            assert r["root"] == root and r["aabb"] == aabb
            stored += 1
    assert stored == n > 0
    # the streaming source: an absent entry is an empty chunk
    L = aok.lib()
    b = aok.ChunkBlob()
    h = ctypes.c_void_p()
    gx, gy, _ = grid
    for i in range(len(bw)):
        c, b0 = bw.blob(i, 0)
        assert L.aok_blobfile_source(f.h, c % gx, (c // gx) % gy, c // (gx * gy), 0, ctypes.byref(b),
                                     ctypes.byref(h)) == 0
        assert b.n_node_words == b0.n_node_words and b.n_mats == b0.n_mats
        L.aok_blobfile_release(None, h)
    assert L.aok_blobfile_source(f.h, gx, 0, 0, 0, ctypes.byref(b), ctypes.byref(h)) != 0  # out of the grid
    f.close()


def _corrupt(path, offset, size_from_end=False):
    data = bytearray(open(path, "rb").read())
    i = len(data) - offset if size_from_end else offset
    data[i] ^= 0x40
    open(path, "wb").write(bytes(data))


def test_damage_is_detected(tmp_path):
    spec = MULTI16
    w, bw = built(spec)
    grid = (spec.wx // spec.chunk, spec.wy // spec.chunk, spec.wz // spec.chunk)
    good = str(tmp_path / "good.aokb")
    aok.BlobFile.write(good, bw, grid, spec.chunk, spec.n_lods)
    raw = open(good, "rb").read()
    cases = {"magic": 0, "header": 20, "index": -8}
    for name, off in cases.items():
        p = str(tmp_path / f"{name}.aokb")
        open(p, "wb").write(raw)
        _corrupt(p, -off if off < 0 else off, size_from_end=off < 0)
        with pytest.raises(aok.AokError) as ex:
            aok.BlobFile(p)
        assert ex.value.status == aok.AOK_E_CORRUPT, name
    # truncated file
    p = str(tmp_path / "short.aokb")
    open(p, "wb").write(raw[:-5])
    with pytest.raises(aok.AokError) as ex:
        aok.BlobFile(p)
    assert ex.value.status == aok.AOK_E_CORRUPT
    # a damaged entry: the file opens, that entry's read fails, the others read
    p = str(tmp_path / "entry.aokb")
    open(p, "wb").write(raw)
    _corrupt(p, 64 + 60)  # inside the first entry's body
    f = aok.BlobFile(p)
    bad = ok = 0
    for i in range(len(bw)):
        for lod in range(spec.n_lods):
            c, b = bw.blob(i, lod)
            if not b.n_node_words:
                continue
            try:
                f.read(c, lod)
                ok += 1
            except aok.AokError as err:
                assert err.status == aok.AOK_E_CORRUPT
                bad += 1
    assert bad == 1 and ok > 0
    f.close()
    # writer rules
    h = ctypes.c_void_p()
    g3 = (ctypes.c_int32 * 3)(*grid)
    L = aok.lib()
    assert L.aok_blobfile_create(str(tmp_path / "w2.aokb").encode(), spec.chunk, spec.n_lods, g3,
                                 ctypes.byref(h)) == aok.AOK_OK
    c, b = next((c, b) for c, b in (bw.blob(i, 0) for i in range(len(bw))) if b.n_node_words)
    assert L.aok_blobfile_add(h, c, 0, ctypes.byref(b)) == aok.AOK_OK
    assert L.aok_blobfile_add(h, c, 0, ctypes.byref(b)) == aok.AOK_E_INVALID  # duplicate
    assert L.aok_blobfile_add(h, grid[0] * grid[1] * grid[2], 0, ctypes.byref(b)) == aok.AOK_E_INVALID
    assert L.aok_blobfile_finish(h) == aok.AOK_OK
    assert aok.BlobFile(str(tmp_path / "w2.aokb")).info()["entries"] == 1
    assert not os.path.exists(str(tmp_path / "missing.aokb"))
    with pytest.raises(aok.AokError):
        aok.BlobFile(str(tmp_path / "missing.aokb"))
