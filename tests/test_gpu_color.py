"""Colour-block compression (Sec. 3.3) with the binary-search colour resolve
(Sec. 3.5) on the GPU: lossless blocks (e_c = 0) render exactly the frame of
raw colour arrays; lossy blocks (e_c = 0.05) render the oracle's colours for
the same tolerance on every non-ambiguous pixel, with unchanged geometry;
the tile-chunk pipeline resolves the same colours; the block storage is
smaller than the raw arrays on coherent colours."""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from gpu_util import compare, decode
from worlds import MED64, MED64_LAYERED, MULTI32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2505_02017_gb300 as aok  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = aok.Context(0)
    yield c
    c.close()


def render(ctx, sc, cam, tau, tiles=False):
    hit, t = aok.alloc_frame(cam.W, cam.H)
    (aok.render_tiles if tiles else aok.render)(ctx, sc, cam, tau, hit, t)
    torch.cuda.synchronize()
    return hit, t


def same(a, b):
    return torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32), b[1].view(torch.int32))


CAMS = [lambda w: sg.ground_camera(w, 4, 160, 90, z_lo=4, z_hi=40),
        lambda w: sg.ground_camera(w, 9, 203, 117, z_lo=4, z_hi=40),
        lambda w: sg.orbit_camera(w.spec, 3, 128, 96, radius=300)]


@pytest.mark.parametrize("spec", [MED64, MED64_LAYERED, MULTI32], ids=lambda s: s.name)
def test_lossless_blocks_equal_raw_arrays(ctx, spec):
    w = sg.World(spec)
    bw = aok.BuiltWorld(w, threads=8)
    raw = aok.Scene.from_world(ctx, w, built=bw)
    blk = aok.Scene.from_world(ctx, w, built=bw, color_tol=0.0)
    for camf in CAMS:
        cam = camf(w)
        ref = render(ctx, raw, cam, 2.0)
        assert same(ref, render(ctx, blk, cam, 2.0))
        assert same(ref, render(ctx, blk, cam, 2.0, tiles=True))
    u_raw, u_blk = raw.usage(), blk.usage()
    assert u_blk["color_bytes"] <= u_raw["color_bytes"]
    if spec.mat_mode == 1:  # coherent colours compress
        assert u_blk["color_bytes"] < 0.5 * u_raw["color_bytes"]
    raw.destroy()
    blk.destroy()


@pytest.mark.parametrize("spec", [MED64_LAYERED, MED64], ids=lambda s: s.name)
def test_lossy_blocks_match_oracle(ctx, spec):
    w = sg.World(spec)
    bw = aok.BuiltWorld(w, threads=8)
    raw = aok.Scene.from_world(ctx, w, built=bw)
    lossy = aok.Scene.from_world(ctx, w, built=bw, color_tol=0.05)
    S = orc.OracleScene(w, color_tol=0.05)
    changed = amb = n = 0
    for camf in CAMS:
        cam = camf(w)
        g = decode(*render(ctx, lossy, cam, 2.0))
        ref = S.cast(cam, S.select(cam, 2.0))
        amb += compare(g, ref, max_amb_frac=1.0)[1]  # the ambiguous share is bounded over the three frames
        n += cam.W * cam.H
        g_raw = decode(*render(ctx, raw, cam, 2.0))
        for k in ("hit", "x", "y", "z", "lod", "normal", "dist"):
            assert (g[k] == g_raw[k]).all(), k
        changed += int((g["mat"] != g_raw["mat"]).sum())
        assert same(render(ctx, lossy, cam, 2.0), render(ctx, lossy, cam, 2.0, tiles=True))
    assert amb <= 1e-4 * n, (amb, n)
    if spec.mat_mode == 1:
        assert changed > 0
    assert lossy.usage()["color_bytes"] <= raw.usage()["color_bytes"]
    raw.destroy()
    lossy.destroy()


def test_color_block_arguments(ctx):
    w = sg.World(MULTI32)
    sc = aok.Scene.from_world(ctx, w, threads=4)
    for bad in (1.5, float("nan")):
        with pytest.raises(aok.AokError) as ex:
            sc.set_color_blocks(bad)
        assert ex.value.status == aok.AOK_E_INVALID
    sc.set_color_blocks(-1.0)  # back to raw arrays
    u = sc.usage()
    assert u["resident"] > 0 and u["node_bytes"] > 0 and u["leaf_bytes"] > 0 and u["color_bytes"] > 0
    sc.destroy()


def test_city4096_layered_1080p(ctx):
    """The benchmark frame on layered colours: lossless blocks render the raw
    frame exactly with a fraction of the colour bytes."""
    w = sg.World(sg.CITY_4096_LAYERED)
    bw = aok.BuiltWorld(w, threads=16)
    raw = aok.Scene.from_world(ctx, w, built=bw)
    blk = aok.Scene.from_world(ctx, w, built=bw, color_tol=0.0)
    cam = sg.ground_camera(w, 102, 1920, 1080)
    assert same(render(ctx, raw, cam, 1.0), render(ctx, blk, cam, 1.0))
    assert blk.usage()["color_bytes"] < 0.5 * raw.usage()["color_bytes"]
    raw.destroy()
    blk.destroy()
