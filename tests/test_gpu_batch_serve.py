"""Batched multi-view rendering and continuous-batching serving, through the
C ABI.  Every batched or served frame must equal the solo aok_render of the
same view (same kernels, same decisions): bit-exact coordinates, LOD, material,
normal and hit flag, identical distances."""
import threading
import time
from dataclasses import replace

import numpy as np
import pytest

import scenegen as sg
from gpu_util import decode
from worlds import MED64, MULTI32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2505_02017_gb300 as aok  # noqa: E402


@pytest.fixture(scope="module")
def env():
    ctx = aok.Context(0)
    worlds = {s.name: sg.World(s) for s in (MED64, MULTI32)}
    scenes = {k: aok.Scene.from_world(ctx, w, threads=8) for k, w in worlds.items()}
    yield ctx, worlds, scenes
    ctx.close()


def poses(worlds, n, seed):
    rng = sg.Rng(seed)
    sizes = [(64, 36), (97, 55), (160, 90), (33, 17), (128, 128), (200, 113)]
    out = []
    names = list(worlds)
    for i in range(n):
        name = names[rng.randint(0, len(names) - 1)]
        W, H = sizes[rng.randint(0, len(sizes) - 1)]
        cam = sg.ground_camera(worlds[name], rng.next(), W, H, z_lo=4, z_hi=30)
        tau = [0.5, 1.0, 2.0, 4.0][rng.randint(0, 3)]
        out.append((name, cam, tau))
    return out


def solo(ctx, scene, cam, tau):
    hit, t = aok.alloc_frame(cam.W, cam.H)
    aok.render(ctx, scene, cam, tau, hit, t)
    return hit, t


def same(a, b):
    ha, ta = a
    hb, tb = b
    return torch.equal(ha, hb) and torch.equal(ta.view(torch.int32), tb.view(torch.int32))


def test_batch_equals_solo_and_graph_replay(env):
    ctx, worlds, scenes = env
    ps1 = poses(worlds, 12, 101)
    # same list shape (scenes, sizes) with moved cameras: the second call replays the graph
    ps2 = [(n, replace(c, origin=c.origin + np.float32(0.5)), tau) for (n, c, tau) in ps1]
    for ps in (ps1, ps2, ps1):
        refs = [solo(ctx, scenes[n], c, tau) for (n, c, tau) in ps]
        outs = [aok.alloc_frame(c.W, c.H) for (_, c, _) in ps]
        views = [aok.make_view(scenes[n], c, tau, h, t) for (n, c, tau), (h, t) in zip(ps, outs)]
        aok.render_batch(ctx, views)
        torch.cuda.synchronize()
        for r, o in zip(refs, outs):
            assert same(r, o)


def test_batch_graph_with_beam_passes(env):
    """With the beam pass on for every view (its minimum frame size lowered),
    a batch's selection, beam pass and cast replay as one CUDA graph: the
    first call builds it, the second (same list shape, moved cameras) updates
    its nodes in place; frames equal the eager launches and the solo renders."""
    ctx, worlds, scenes = env
    aok.beam_tune(ctx, min_pixels=1)
    try:
        ps1 = poses(worlds, 9, 303)
        ps2 = [(n, replace(c, origin=c.origin + np.float32(0.25)), tau) for (n, c, tau) in ps1]
        for ps in (ps1, ps2):
            refs = [solo(ctx, scenes[n], c, tau) for (n, c, tau) in ps]
            res = {}
            for graph in (False, True):
                aok.set_batch_graph(ctx, graph)
                outs = [aok.alloc_frame(c.W, c.H) for (_, c, _) in ps]
                views = [aok.make_view(scenes[n], c, tau, h, t) for (n, c, tau), (h, t) in zip(ps, outs)]
                aok.render_batch(ctx, views)
                torch.cuda.synchronize()
                res[graph] = outs
            for r, a, b in zip(refs, res[False], res[True]):
                assert same(r, a) and same(r, b)
    finally:
        aok.set_batch_graph(ctx, True)
        aok.beam_tune(ctx)


def test_batch_over_128_views_and_every_tile_shape(env):
    ctx, worlds, scenes = env
    ps = poses(worlds, 133, 7)
    refs = [solo(ctx, scenes[n], c, tau) for (n, c, tau) in ps]
    for persistent in (False, True):
        aok.set_batch_kernel(ctx, persistent)
        for tile in (4, 8, 16, 32):
            aok.set_tile(ctx, tile)
            outs = [aok.alloc_frame(c.W, c.H) for (_, c, _) in ps]
            views = [aok.make_view(scenes[n], c, tau, h, t) for (n, c, tau), (h, t) in zip(ps, outs)]
            aok.render_batch(ctx, views)
            torch.cuda.synchronize()
            assert all(same(r, o) for r, o in zip(refs, outs)), (persistent, tile)
    aok.set_batch_kernel(ctx, False)
    aok.set_tile(ctx, 8)


def test_single_view_persistent_kernel_and_launch_shapes(env):
    ctx, worlds, scenes = env
    ps = poses(worlds, 4, 11)
    refs = [solo(ctx, scenes[n], c, tau) for (n, c, tau) in ps]
    aok.set_single_view_kernel(ctx, True)
    try:
        for persistent, ctas, threads, packet in [(False, 0, 0, 0), (True, 1, 128, 32), (True, 2, 256, 64),
                                                  (True, 0, 0, 128)]:
            aok.set_batch_kernel(ctx, persistent)
            aok.set_launch(ctx, ctas, threads, packet)
            for (n, c, tau), r in zip(ps, refs):
                assert same(r, solo(ctx, scenes[n], c, tau))
                # split select / cast with the persistent cast
                hit, t = aok.alloc_frame(c.W, c.H)
                aok.select_chunks(ctx, scenes[n], c, tau)
                aok.cast_selected(ctx, scenes[n], c, hit, t)
                assert same(r, (hit, t))
    finally:
        aok.set_single_view_kernel(ctx, False)
        aok.set_batch_kernel(ctx, False)


def test_autotune_keeps_results(env):
    ctx, worlds, scenes = env
    ps = poses(worlds, 6, 13)
    refs = [solo(ctx, scenes[n], c, tau) for (n, c, tau) in ps]
    outs = [aok.alloc_frame(c.W, c.H) for (_, c, _) in ps]
    views = [aok.make_view(scenes[n], c, tau, h, t) for (n, c, tau), (h, t) in zip(ps, outs)]
    ms = aok.autotune(ctx, views)
    assert ms > 0
    ctas, threads, packet = aok.get_launch(ctx)
    assert ctas >= 0 and threads in (128, 256) and packet in (32, 64, 128)
    aok.render_batch(ctx, views)
    torch.cuda.synchronize()
    assert all(same(r, o) for r, o in zip(refs, outs))


def test_serving_results_equal_solo_in_the_mix(env):
    ctx, worlds, scenes = env
    ps = poses(worlds, 40, 17)
    refs = [solo(ctx, scenes[n], c, tau) for (n, c, tau) in ps]
    torch.cuda.synchronize()
    srv = aok.Server(ctx, max_slots=16, max_batch=8, n_streams=3)
    try:
        tickets = [None] * len(ps)

        def submitter():  # arrivals while earlier requests are on the GPU
            for i, (n, c, tau) in enumerate(ps):
                tickets[i] = srv.submit(scenes[n], c, tau)
                time.sleep(0.0005 * (i % 3))

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        for i, tk in enumerate(tickets):
            st, f = srv.wait(tk, 60000)
            assert st == aok.AOK_OK, st
            hit, t = srv.result(tk, f)
            assert same(refs[i], (hit, t)), i
            s, d = srv.times(tk)
            assert d >= s > 0
            assert srv.release(tk) == aok.AOK_OK
    finally:
        srv.stop()


def test_serving_admission_by_budget_and_cancel(env):
    _, worlds, _ = env
    # a context whose budget holds the scene plus only ~2 request frames
    w = worlds[MULTI32.name]
    probe = aok.Context(0)
    bw = aok.BuiltWorld(w, threads=4)
    sc = aok.Scene.from_world(probe, w, built=bw)
    used, _ = probe.memory()
    cam = sg.ground_camera(w, 4, 256, 256, z_lo=4, z_hi=20)
    frame_bytes = 256 * 256 * 20 + 4096
    sc.destroy()
    probe.close()
    ctx = aok.Context(0, budget_bytes=used + int(2.5 * frame_bytes))
    sc = aok.Scene.from_world(ctx, w, built=bw)
    ref = solo(ctx, sc, cam, 1.0)
    srv = aok.Server(ctx, max_slots=8, max_batch=4, n_streams=2)
    try:
        tks = [srv.submit(sc, cam, 1.0) for _ in range(5)]
        time.sleep(0.5)
        states = [srv.poll(tk)[0] for tk in tks]
        # slow consumer: nothing released yet, so at most 2 frames fit
        assert states.count(aok.AOK_OK) == 2 and states.count(aok.AOK_PENDING) == 3
        # cancel one waiting request, release the finished ones: the rest proceed
        waiting = [tk for tk, s in zip(tks, states) if s == aok.AOK_PENDING]
        assert srv.release(waiting[0]) == aok.AOK_OK
        for tk, s in zip(tks, states):
            if s == aok.AOK_OK:
                st, f = srv.wait(tk)
                assert same(ref, srv.result(tk, f))
                srv.release(tk)
        for tk in waiting[1:]:
            st, f = srv.wait(tk, 30000)
            assert st == aok.AOK_OK
            assert same(ref, srv.result(tk, f))
            srv.release(tk)
        # a frame larger than the whole budget is refused at submission
        big = replace(cam, W=4096, H=4096)
        with pytest.raises(aok.AokError) as ex:
            srv.submit(sc, big, 1.0)
        assert ex.value.status == aok.AOK_E_OOM
    finally:
        srv.stop()
        sc.destroy()
        ctx.close()


def test_pipelined_host_frames_equal_device_frames(env):
    """aok_render_host_async: frames in flight overlap; each host frame equals
    the device render of its camera."""
    ctx, worlds, scenes = env
    ps = poses(worlds, 7, 23)
    refs = [solo(ctx, scenes[n], c, tau) for (n, c, tau) in ps]
    torch.cuda.synchronize()  # the pipeline renders on its own stream
    bufs = [(torch.empty((c.H, c.W, 4), dtype=torch.int32, pin_memory=True),
             torch.empty((c.H, c.W), dtype=torch.float32, pin_memory=True)) for (_, c, _) in ps]
    tickets = [aok.render_host_async(ctx, scenes[n], c, tau, *b) for (n, c, tau), b in zip(ps, bufs)]
    assert tickets == sorted(tickets) and len(set(tickets)) == len(tickets)
    for tk in tickets:
        aok.host_frame_wait(ctx, tk)
    for (hr, tr), (hh, th) in zip(refs, bufs):
        assert torch.equal(hr.cpu(), hh) and torch.equal(tr.cpu().view(torch.int32), th.view(torch.int32))
    with pytest.raises(aok.AokError) as ex:
        aok.host_frame_wait(ctx, tickets[-1] + 100)
    assert ex.value.status == aok.AOK_E_INVALID
