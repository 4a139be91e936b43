"""aok_render_noalloc: rendering for callers that cannot allocate device
memory at render time (for example an engine frame loop that reserved its
device memory up front).  Its per-frame chunk table lives in a static device
array instead of scene-owned memory; its frames must equal aok_render's.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.  It builds its own context and
scene, so it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import scenegen as sg
from gpu_util import DIST_RTOL, decode
from worlds import MED64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2505_02017_gb300 as aok  # noqa: E402


def test_noalloc_matches_render_on_two_calls_in_a_row():
    ctx = aok.Context(0)
    world = sg.World(MED64)
    scene = aok.Scene.from_world(ctx, world, threads=8)
    L = aok.lib()
    stream = torch.cuda.current_stream().cuda_stream
    cams = [sg.ground_camera(world, 4, 160, 90, z_lo=4, z_hi=40),
            sg.orbit_camera(MED64, 3, 131, 77, radius=300)]
    for cam, tau in zip(cams, (4.0, 1.5)):
        ref_hit, ref_t = aok.alloc_frame(cam.W, cam.H)
        aok.render(ctx, scene, cam, tau, ref_hit, ref_t)
        hit, t = aok.alloc_frame(cam.W, cam.H)
        hit.fill_(-1)
        t.fill_(-1.0)
        c = aok.to_camera(cam)
        f = aok.frame_of(hit, t)
        rc = L.aok_render_noalloc(ctx.h, scene.id, ctypes.byref(c), tau, ctypes.byref(f), stream)
        assert rc == aok.AOK_OK, rc
        torch.cuda.synchronize()
        a, b = decode(hit, t), decode(ref_hit, ref_t)
        for k in ("hit", "x", "y", "z", "lod", "mat", "normal"):
            assert (a[k] == b[k]).all(), k
        h = b["hit"] == 1
        assert h.sum() > 0
        rel = np.abs(a["dist"][h] - b["dist"][h]) / b["dist"][h]
        assert (rel <= DIST_RTOL).all()
        assert np.isinf(a["dist"][~h]).all()

    # with checked casting on it takes the checked kernel: the same frame and no
    # pool index out of range (its error word is context memory: still no allocation)
    cam = cams[0]
    ref_hit, ref_t = aok.alloc_frame(cam.W, cam.H)
    aok.render(ctx, scene, cam, 4.0, ref_hit, ref_t)
    aok.set_checked(ctx, True)
    hit, t = aok.alloc_frame(cam.W, cam.H)
    c = aok.to_camera(cam)
    f = aok.frame_of(hit, t)
    assert L.aok_render_noalloc(ctx.h, scene.id, ctypes.byref(c), 4.0, ctypes.byref(f), stream) == aok.AOK_OK
    torch.cuda.synchronize()
    assert aok.checked_errors(ctx) == 0
    aok.set_checked(ctx, False)
    assert torch.equal(hit, ref_hit) and torch.equal(t.view(torch.int32), ref_t.view(torch.int32))

    # a camera whose casting grid could not launch (more than 65535 rows of
    # 8-pixel blocks) and one of 2^31 pixels are refused before any launch
    for W, H in ((1, 600000), (4096, 524288)):
        c = aok.to_camera(sg.make_camera((10.0, 10.0, 10.0), (1.0, 0.5, -0.2), W, H))
        f = aok.frame_of(hit, t)
        assert L.aok_render_noalloc(ctx.h, scene.id, ctypes.byref(c), 1.0, ctypes.byref(f), stream) == \
            aok.AOK_E_INVALID
    scene.destroy()

    # a grid larger than the static table is refused before any work is enqueued
    d = aok.SceneDesc()
    d.grid[0], d.grid[1], d.grid[2] = 256, 256, 2  # 131072 chunk regions
    d.chunk_res, d.n_lods = 8, 1
    d.node_words, d.leaf_count, d.mat_bytes = 64, 64, 64
    sid = ctypes.c_uint32()
    assert L.aok_scene_create(ctx.h, ctypes.byref(d), ctypes.byref(sid)) == aok.AOK_OK
    assert d.grid[0] * d.grid[1] * d.grid[2] > 65536
    cam = sg.make_camera((10.0, 10.0, 10.0), (1.0, 0.5, -0.2), 8, 8)
    hit, t = aok.alloc_frame(8, 8)
    c = aok.to_camera(cam)
    f = aok.frame_of(hit, t)
    assert L.aok_render_noalloc(ctx.h, sid.value, ctypes.byref(c), 1.0, ctypes.byref(f), stream) == aok.AOK_E_INVALID
    L.aok_scene_destroy(ctx.h, sid.value)
    ctx.close()
