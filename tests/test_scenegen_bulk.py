"""The generator's bulk calls that the chunk builder uses return the same
voxels as its point and full-region calls: block materials equal the
per-voxel material, the z-bounded bit fill equals the counting bit fill and
reports the exact z range of the solid voxels, and rectangle heights equal
point heights over spans of several lattice rows."""
import numpy as np
import pytest

import scenegen as sg
from worlds import MED64, MULTI16


@pytest.mark.parametrize("spec", [MED64, sg.CITY_4096, sg.OPEN_65536], ids=lambda s: s.name)
def test_block_materials_equal_point_materials(spec):
    w = sg.World(spec)
    rng = np.random.default_rng(11)
    for _ in range(40):
        x0, y0, z0 = (int(v) * 4 for v in rng.integers(0, [spec.wx // 4, spec.wy // 4, spec.wz // 4]))
        mask = int(rng.integers(0, 2**63, dtype=np.uint64)) | (int(rng.integers(0, 2)) << 63)
        out = np.full(64, 0xA5, np.uint8)
        w.materials_block4(x0, y0, z0, mask, out)
        for b in range(64):
            if (mask >> b) & 1:
                assert out[b] == w.material(x0 + (b & 3), y0 + ((b >> 2) & 3), z0 + (b >> 4))
            else:
                assert out[b] == 0xA5  # untouched


def region_cases(spec, rng, n):
    M = spec.chunk
    for _ in range(n):
        cx, cy, cz = (int(v) for v in rng.integers(0, spec.grid))
        yield cx * M, cy * M, cz * M, M
    # regions reaching past the world on each side
    yield -64, -64, -64, 128
    yield spec.wx - 64, spec.wy - 64, spec.wz - 64, 128


@pytest.mark.parametrize("spec", [MULTI16, MED64, sg.CITY_4096], ids=lambda s: s.name)
def test_bounded_bit_fill_equals_bit_fill(spec):
    w = sg.World(spec)
    rng = np.random.default_rng(12)
    for x0, y0, z0, M in region_cases(spec, rng, 6):
        n = max(64, M)
        cnt, ref = w.fill_bits(x0, y0, z0, n, M, M)
        bits = np.zeros_like(ref)
        anyv, (zlo, zhi) = w.fill_bits_z(x0, y0, z0, n, M, M, bits)
        assert (bits == ref).all()
        assert anyv == (cnt > 0)
        # the bit layouts against the byte fill (one voxel at a time)
        dense = w.dense(x0, y0, z0, n, M, M)
        packed = np.packbits(dense.reshape(-1, 64), axis=1, bitorder="little").view(np.uint64).ravel()
        assert (ref == packed).all()
        rows = ref.reshape(M, M, n // 64)
        zs = np.nonzero(rows.any(axis=(1, 2)))[0]
        if cnt:
            assert (zlo, zhi) == (int(zs[0]), int(zs[-1]) + 1)
        else:
            assert (zlo, zhi) == (0, 0)


def test_bounded_bit_fill_adds_to_the_buffer_and_rejects_ragged_rows():
    w = sg.World(sg.CITY_4096)
    z0 = w.height(32, 32) - 32  # a region through the terrain surface
    cnt, ref = w.fill_bits(0, 0, z0, 64, 64, 64)
    assert cnt > 0
    i = int(np.nonzero(ref == 0)[0][0])
    pre = np.zeros_like(ref)
    pre[i] = 1 << 7  # a bit the caller left in an empty row: kept (the call clears nothing)
    anyv, _ = w.fill_bits_z(0, 0, z0, 64, 64, 64, pre)
    expect = ref.copy()
    expect[i] = 1 << 7
    assert anyv == 1 and (pre == expect).all()
    buf = np.zeros(64, np.uint64)
    assert w.fill_bits_z(0, 0, 0, 48, 8, 8, buf) == (-1, (0, 0))
    assert not buf.any()


def test_rectangle_heights_over_many_lattice_rows():
    rng = np.random.default_rng(13)
    for spec in (sg.CITY_4096, sg.OPEN_65536):
        w = sg.World(spec)
        for _ in range(3):
            x0, y0 = (int(v) for v in rng.integers(-500, spec.wx, 2))
            h = w.heights(x0, y0, 3, 700)  # > 5 lattice rows of the finest octaves
            ref = np.array([[w.height(x0 + x, y0 + y) for x in range(3)] for y in range(700)], np.int32)
            assert (h == ref).all()
