"""Residency streaming (Sec. 3.4): only the (chunk, LOD) pairs a camera needs
within the view distance are resident; moving along a path evicts and builds
chunks between frames, and every frame still equals the oracle on every
non-ambiguous pixel."""
import time

import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from gpu_util import compare, decode, stratified

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2505_02017_gb300 as aok  # noqa: E402
from paper_2505_02017_gb300.stream import Streamer  # noqa: E402


def test_streaming_path_matches_oracle():
    spec = sg.OPEN_8192
    w = sg.World(spec)
    ctx = aok.Context(0)
    sc = aok.Scene(ctx, spec, node_words=64 << 20, leaves=16 << 20, mat_bytes=1 << 30)
    st = Streamer(ctx, w, sc, threads=16)
    S = orc.OracleScene(w)
    cams = sg.path_cameras(w, 77, 5, 128, 72, n_waypoints=3, span=3000.0)
    tau = 1.0 / 3.0
    stats = []
    for i, cam in enumerate(cams):
        stats.append(st.update(cam, tau))
        plan = st.plan(cam, tau)
        hit, t = aok.alloc_frame(cam.W, cam.H)
        aok.render(ctx, sc, cam, tau, hit, t)
        torch.cuda.synchronize()
        if i in (0, 2, 4):
            sel = np.where(plan == 0xFF, -1, plan.astype(np.int32)).astype(np.int8)
            # the plan's LODs are Eq. 1's LODs (bit-identical host and oracle arithmetic)
            full = S.select(cam, tau)
            assert ((sel < 0) | (sel == full)).all()
            ref = S.cast(cam, sel, view_dist=spec.view_dist)
            compare(decode(hit, t), ref)
    assert all(s["resident"] < sc.grid[0] * sc.grid[1] * sc.grid[2] for s in stats)
    assert stats[0]["built"] > 0 and any(s["evicted"] > 0 or s["built"] > 0 for s in stats[1:])
    sc.destroy()
    ctx.close()


def within_view(spec, cam):
    """Chunk regions whose cell lies within the view distance (+2 voxels) of the
    camera: the regions a residency plan keeps (FP64)."""
    M = spec.chunk
    gx, gy, gz = spec.grid
    cz, cy, cx = np.meshgrid(np.arange(gz), np.arange(gy), np.arange(gx), indexing="ij")
    lo = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], 1).astype(np.float64) * M
    o = cam.origin.astype(np.float64)
    q = np.maximum(np.maximum(lo - o, o - (lo + M)), 0.0)
    return (q * q).sum(1) <= (spec.view_dist + 2.0) ** 2


def test_open65536_path_poses_sampled():
    """The benchmark's open world (65536x65536x1024, view distance 16384) at
    2560x1440 for three poses of its path, on stratified pixels: the streamed
    residency plan is Eq. 1's selection within the view distance, and the
    oracle traces the same selection on its own."""
    spec = sg.OPEN_65536
    w = sg.World(spec)
    ctx = aok.Context(0)
    sc = aok.Scene(ctx, spec, node_words=512 << 20, leaves=256 << 20, mat_bytes=16 << 30)
    st = Streamer(ctx, w, sc, threads=16)
    S = orc.OracleScene(w)
    tau = 1.0
    path = sg.path_cameras(w, 103, 300, 2560, 1440)
    checked = amb = hits = 0
    for k, pose in enumerate((0, 150, 299)):
        cam = path[pose]
        st.update(cam, tau)
        hit, t = aok.alloc_frame(cam.W, cam.H)
        aok.render(ctx, sc, cam, tau, hit, t)
        torch.cuda.synchronize()
        sel = S.select(cam, tau)
        plan = st.plan(cam, tau)
        inside = within_view(spec, cam)
        assert (plan[inside] == sel[inside]).all() and (plan[~inside] == 0xFF).all()
        idx = stratified(cam.W, cam.H, 7000, seed=pose)
        ref = S.cast(cam, sel, pixels=np.stack([idx % cam.W, idx // cam.W], 1), view_dist=spec.view_dist)
        c, a = compare(decode(hit, t), ref, idx=idx, max_amb_frac=1.0, min_pixels_checked=0)
        checked += c
        amb += a
        hits += int((ref["hit"] == 1).sum())
    assert checked + amb >= 20000
    assert amb <= 1e-4 * (checked + amb), (amb, checked)
    assert hits > 0.3 * (checked + amb)
    sc.destroy()
    ctx.close()


def test_async_streaming_frames_match_oracle_and_settle():
    """Asynchronous residency (Sec. 3.4): frames render while loads run in the
    background; every frame equals the oracle for the LODs it actually used
    (the selected one where installed, else the stand-in the selection chose);
    once the loads finish, the frame equals the synchronous streamer's."""
    from paper_2505_02017_gb300.stream import AsyncStreamer
    spec = sg.OPEN_8192
    w = sg.World(spec)
    ctx = aok.Context(0)
    sc_a = aok.Scene(ctx, spec, node_words=64 << 20, leaves=16 << 20, mat_bytes=1 << 30)
    sc_s = aok.Scene(ctx, spec, node_words=64 << 20, leaves=16 << 20, mat_bytes=1 << 30)
    ast = AsyncStreamer(ctx, w, sc_a, threads=8)
    sst = Streamer(ctx, w, sc_s, threads=8)
    S = orc.OracleScene(w)
    cams = sg.path_cameras(w, 77, 6, 160, 90, n_waypoints=3, span=3000.0)
    tau = 1.0 / 3.0
    n = sc_a.grid[0] * sc_a.grid[1] * sc_a.grid[2]
    partial = 0
    for i, cam in enumerate(cams):
        ast.update(cam, tau)
        if i == 2:
            ast.wait()  # one frame in the middle with every load of the previous plan finished
        lod = torch.empty(n, dtype=torch.int8, device="cuda")
        hit, t = aok.alloc_frame(cam.W, cam.H)
        aok.select_chunks(ctx, sc_a, cam, tau, lod_out=lod)
        aok.cast_selected(ctx, sc_a, cam, hit, t)
        torch.cuda.synchronize()
        used = lod.cpu().numpy().astype(np.int64)
        res = ast.resident().astype(np.int64)
        sel = np.where((res >> used) & 1, used, -1).astype(np.int8)
        partial += int(ast.stats()["missing"] > 0)
        ref = S.cast(cam, sel, view_dist=spec.view_dist)
        compare(decode(hit, t), ref)
    assert partial > 0  # some frames rendered before their loads finished
    # settle on the last pose and compare with the synchronous streamer
    assert ast.wait(120000) == aok.AOK_OK
    ast.update(cams[-1], tau)
    st = ast.stats()
    assert st["missing"] == 0 and st["failed_total"] == 0 and st["installed_total"] > 0
    assert st["max_resident"] >= st["resident"] > 0
    sst.update(cams[-1], tau)
    fa, fs = aok.alloc_frame(160, 90), aok.alloc_frame(160, 90)
    aok.render(ctx, sc_a, cams[-1], tau, *fa)
    aok.render(ctx, sc_s, cams[-1], tau, *fs)
    torch.cuda.synchronize()
    assert torch.equal(fa[0], fs[0]) and torch.equal(fa[1].view(torch.int32), fs[1].view(torch.int32))
    ast.close()
    sc_a.destroy()
    sc_s.destroy()
    ctx.close()


def test_async_streaming_under_pool_pressure():
    """Pools too small for a whole plan: loads that do not fit are deferred and
    retried after evictions free space; nothing fails, and every frame still
    equals the oracle for the LODs it used."""
    from paper_2505_02017_gb300.stream import AsyncStreamer
    spec = sg.OPEN_8192
    w = sg.World(spec)
    ctx = aok.Context(0)
    sc = aok.Scene(ctx, spec, node_words=512 << 10, leaves=128 << 10, mat_bytes=6 << 20)
    ast = AsyncStreamer(ctx, w, sc, threads=8)
    S = orc.OracleScene(w)
    cams = sg.path_cameras(w, 91, 8, 96, 54, n_waypoints=4, span=6000.0)
    tau = 1.0 / 30.0  # fine LODs far out: a plan larger than the pools
    n = sc.grid[0] * sc.grid[1] * sc.grid[2]
    for i, cam in enumerate(cams):
        ast.update(cam, tau)
        ast.wait(60000)
        ast.update(cam, tau)  # install what finished
        lod = torch.empty(n, dtype=torch.int8, device="cuda")
        hit, t = aok.alloc_frame(cam.W, cam.H)
        aok.select_chunks(ctx, sc, cam, tau, lod_out=lod)
        aok.cast_selected(ctx, sc, cam, hit, t)
        torch.cuda.synchronize()
        used = lod.cpu().numpy().astype(np.int64)
        res = ast.resident().astype(np.int64)
        sel = np.where((res >> used) & 1, used, -1).astype(np.int8)
        if i % 3 == 0:
            compare(decode(hit, t), S.cast(cam, sel, view_dist=spec.view_dist))
    st = ast.stats()
    assert st["deferred_total"] > 0 and st["failed_total"] == 0 and st["evicted_total"] > 0
    u = sc.usage()
    assert u["node_bytes"] <= 2 * 4 * (512 << 10) and u["color_bytes"] <= 6 << 20
    ast.close()
    sc.destroy()
    ctx.close()


def test_async_streaming_from_blob_file(tmp_path):
    """The paper's disk-resident chunks: the (chunk, LOD)s a path needs are
    written to a chunk-blob file; the asynchronous loader reads them from it;
    once settled, every pose renders exactly as with the synchronous,
    procedurally built residency."""
    from paper_2505_02017_gb300.stream import AsyncStreamer
    spec = sg.OPEN_8192
    w = sg.World(spec)
    ctx = aok.Context(0)
    sc_f = aok.Scene(ctx, spec, node_words=64 << 20, leaves=16 << 20, mat_bytes=1 << 30)
    sc_s = aok.Scene(ctx, spec, node_words=64 << 20, leaves=16 << 20, mat_bytes=1 << 30)
    sst = Streamer(ctx, w, sc_s, threads=8)
    cams = sg.path_cameras(w, 77, 5, 160, 90, n_waypoints=3, span=3000.0)
    tau = 1.0 / 3.0
    masks = {}
    for cam in cams:
        plan = sst.plan(cam, tau)
        for c in np.nonzero(plan != 0xFF)[0]:
            masks[int(c)] = masks.get(int(c), 0) | (1 << int(plan[c]))
    chunks = np.array(sorted(masks), np.int64)
    bw = aok.BuiltWorld(w, threads=8, chunks=chunks, lod_masks=np.array([masks[c] for c in chunks], np.uint32))
    path = str(tmp_path / "open8192_path.aokb")
    n = aok.BlobFile.write(path, bw, sc_f.grid, spec.chunk, spec.n_lods)
    bw.close()
    assert n > 0
    blobs = aok.BlobFile(path)
    ast = AsyncStreamer(ctx, None, sc_f, threads=8, blobs=blobs)
    for cam in cams:
        ast.update(cam, tau)
        assert ast.wait(60000) == aok.AOK_OK
        ast.update(cam, tau)
        assert ast.stats()["missing"] == 0
        sst.update(cam, tau)
        fa, fs = aok.alloc_frame(cam.W, cam.H), aok.alloc_frame(cam.W, cam.H)
        aok.render(ctx, sc_f, cam, tau, *fa)
        aok.render(ctx, sc_s, cam, tau, *fs)
        torch.cuda.synchronize()
        assert torch.equal(fa[0], fs[0]) and torch.equal(fa[1].view(torch.int32), fs[1].view(torch.int32))
    st = ast.stats()
    assert st["failed_total"] == 0 and st["installed_total"] > 0
    ast.close()
    blobs.close()
    sc_f.destroy()
    sc_s.destroy()
    ctx.close()


def test_async_prefetch_along_motion():
    """Prefetch along the camera's motion (aok_stream_set_prefetch): with
    every load finished between poses, the streamer that plans the camera
    extrapolated ahead already holds nearly every LOD the next pose plans when
    that pose's update runs, where the one without prefetch holds none of the
    new ones; frames equal the oracle for the LODs they used; once settled,
    frames equal the synchronous streamer's; bad arguments are refused."""
    from paper_2505_02017_gb300.stream import AsyncStreamer
    spec = sg.OPEN_8192
    w = sg.World(spec)
    ctx = aok.Context(0)
    scs = [aok.Scene(ctx, spec, node_words=64 << 20, leaves=16 << 20, mat_bytes=1 << 30) for _ in range(3)]
    pre = AsyncStreamer(ctx, w, scs[0], threads=8)
    plain = AsyncStreamer(ctx, w, scs[1], threads=8)
    try:
        sst = Streamer(ctx, w, scs[2], threads=8)
        for bad in ((-1, 2), (1001, 2), (4, 0), (4, 17)):
            with pytest.raises(aok.AokError):
                pre.set_prefetch(*bad)
        pre.set_prefetch(3, 3)
        S = orc.OracleScene(w)
        # one straight leg: poses equally spaced along it (the ground clamp aside)
        W, H = 320, 180
        cams = sg.path_cameras(w, 77, 12, W, H, n_waypoints=2, span=3000.0)
        tau = 1.0 / 3.0
        n = scs[0].grid[0] * scs[0].grid[1] * scs[0].grid[2]
        miss_pre = miss_plain = new_pairs = checked = amb = 0
        prev_plan = None
        for i, cam in enumerate(cams):
            pre.update(cam, tau)
            plain.update(cam, tau)
            plan = sst.plan(cam, tau)
            if i >= 2:  # the first update has no motion, the second extrapolates from one step
                new_pairs += int(((plan != 0xFF) & (plan != prev_plan)).sum())
                miss_pre += pre.stats()["missing"]
                miss_plain += plain.stats()["missing"]
            prev_plan = plan
            if i % 4 == 3:
                lod = torch.empty(n, dtype=torch.int8, device="cuda")
                hit, t = aok.alloc_frame(W, H)
                aok.select_chunks(ctx, scs[0], cam, tau, lod_out=lod)
                aok.cast_selected(ctx, scs[0], cam, hit, t)
                torch.cuda.synchronize()
                used = lod.cpu().numpy().astype(np.int64)
                res = pre.resident().astype(np.int64)
                sel = np.where((res >> used) & 1, used, -1).astype(np.int8)
                c, a = compare(decode(hit, t), S.cast(cam, sel, view_dist=spec.view_dist), max_amb_frac=1.0,
                               min_pixels_checked=0)
                checked += c
                amb += a
            assert pre.wait(120000) == aok.AOK_OK and plain.wait(120000) == aok.AOK_OK
        assert amb <= 1e-4 * (checked + amb), (amb, checked)
        st = pre.stats()
        assert new_pairs > 0 and miss_plain >= new_pairs // 2
        assert miss_pre <= 0.1 * miss_plain, (miss_pre, miss_plain, new_pairs)
        assert st["ahead_installed_total"] > 0 and st["failed_total"] == 0
        # settled on the last pose: the frame equals the synchronous streamer's
        pre.update(cams[-1], tau)
        assert pre.stats()["missing"] == 0
        sst.update(cams[-1], tau)
        fa, fs = aok.alloc_frame(W, H), aok.alloc_frame(W, H)
        aok.render(ctx, scs[0], cams[-1], tau, *fa)
        aok.render(ctx, scs[2], cams[-1], tau, *fs)
        torch.cuda.synchronize()
        assert torch.equal(fa[0], fs[0]) and torch.equal(fa[1].view(torch.int32), fs[1].view(torch.int32))
        pre.set_prefetch(0, 0)  # off again
    finally:
        pre.close()
        plain.close()
        for sc in scs:
            sc.destroy()
        ctx.close()


def test_async_load_installed_and_evicted_in_one_update():
    """A load that lands after its region has settled on another resident
    LOD is installed and evicted by the same update (its space goes to
    quarantine): the region's descriptor must end evicted, so that no frame
    selects that LOD while its space can be reused.  Checked on every region
    two path poses plan at different LODs, with selection at the pose that
    asked for the load and a checked render there."""
    from paper_2505_02017_gb300.stream import AsyncStreamer
    spec = sg.OPEN_8192
    w = sg.World(spec)
    ctx = aok.Context(0)
    sc = aok.Scene(ctx, spec, node_words=64 << 20, leaves=16 << 20, mat_bytes=1 << 30)
    planner_scene = aok.Scene(ctx, spec, node_words=1 << 16, leaves=1 << 16, mat_bytes=1 << 16)
    ast = AsyncStreamer(ctx, w, sc, threads=8)
    try:
        tau = 1.0 / 3.0
        # at 320 x 180 and tau = 1/3 the path's poses plan LODs 0-3 (Eq. 1 depends on the image height)
        cams = sg.path_cameras(w, 77, 6, 320, 180, n_waypoints=3, span=3000.0)
        planner = Streamer(ctx, w, planner_scene, threads=1)
        plans = [planner.plan(c, tau) for c in cams]
        best = None
        for i in range(len(cams)):
            for j in range(len(cams)):
                both = (plans[i] != 0xFF) & (plans[j] != 0xFF) & (plans[i] != plans[j])
                if i != j and (best is None or both.sum() > best[2]):
                    best = (i, j, int(both.sum()))
        ia, ib, n_diff = best
        assert n_diff > 0
        A, B = cams[ia], cams[ib]
        ast.update(A, tau)
        assert ast.wait(120000) == aok.AOK_OK
        ast.update(A, tau)  # A's plan installed
        assert ast.stats()["missing"] == 0
        ast.update(B, tau)  # B's LODs load; the regions both plan keep A's LOD meanwhile
        assert ast.wait(120000) == aok.AOK_OK
        ast.update(A, tau)  # B's loads land: installed, and evicted at once where A's LOD is resident
        torch.cuda.synchronize()
        res = ast.resident().astype(np.int64)
        n = sc.grid[0] * sc.grid[1] * sc.grid[2]
        both = (plans[ia] != 0xFF) & (plans[ib] != 0xFF) & (plans[ia] != plans[ib])
        assert not ((res[both] >> plans[ib][both].astype(np.int64)) & 1).any()  # evicted on the host
        lod = torch.empty(n, dtype=torch.int8, device="cuda")
        vis = torch.empty(n, dtype=torch.uint8, device="cuda")
        aok.select_chunks(ctx, sc, B, tau, lod_out=lod, vis_out=vis)
        torch.cuda.synchronize()
        used = lod.cpu().numpy().astype(np.int64)
        shown = vis.cpu().numpy() == 1
        assert shown.any()
        assert ((res[shown] >> used[shown]) & 1).all()  # every LOD a frame uses is resident
        assert aok.checked_errors(ctx) == 0
        aok.set_checked(ctx, True)
        try:
            hit, t = aok.alloc_frame(B.W, B.H)
            aok.render(ctx, sc, B, tau, hit, t)
            torch.cuda.synchronize()
        finally:
            aok.set_checked(ctx, False)
        assert aok.checked_errors(ctx) == 0
    finally:
        ast.close()
        sc.destroy()
        planner_scene.destroy()
        ctx.close()


def test_scene_destroyed_under_a_running_streamer():
    """Destroying a scene (or its context) while its streamer still loads
    stops the streamer first: its workers are joined, later calls are
    refused with AOK_E_NOT_RESIDENT, and closing it afterwards is safe."""
    from paper_2505_02017_gb300.stream import AsyncStreamer
    spec = sg.OPEN_8192
    w = sg.World(spec)
    ctx = aok.Context(0)
    sc = aok.Scene(ctx, spec, node_words=64 << 20, leaves=16 << 20, mat_bytes=1 << 30)
    st = AsyncStreamer(ctx, w, sc, threads=4)
    cam = sg.path_cameras(w, 77, 2, 160, 90, n_waypoints=2, span=3000.0)[0]
    st.update(cam, 1.0 / 3.0)  # loads start in the background
    sc.destroy()
    with pytest.raises(aok.AokError) as e:
        st.update(cam, 1.0 / 3.0)
    assert e.value.status == aok.AOK_E_NOT_RESIDENT
    assert st.wait(0) == aok.AOK_E_NOT_RESIDENT
    st.stats()
    st.close()
    # a wait under way when the scene goes returns (AOK_E_NOT_RESIDENT, or AOK_OK
    # if the loads finished first) instead of waiting for loads that never come
    import threading
    sc3 = aok.Scene(ctx, spec, node_words=64 << 20, leaves=16 << 20, mat_bytes=1 << 30)
    st3 = AsyncStreamer(ctx, w, sc3, threads=2)
    st3.update(cam, 1.0 / 3.0)
    res = []
    th = threading.Thread(target=lambda: res.append(st3.wait(60000)))
    th.start()
    time.sleep(0.05)
    sc3.destroy()
    th.join(90)
    assert not th.is_alive() and res and res[0] in (aok.AOK_OK, aok.AOK_E_NOT_RESIDENT), res
    st3.close()
    # the same through the context: its scenes go, and with them the streamer's
    sc2 = aok.Scene(ctx, spec, node_words=64 << 20, leaves=16 << 20, mat_bytes=1 << 30)
    st2 = AsyncStreamer(ctx, w, sc2, threads=4)
    st2.update(cam, 1.0 / 3.0)
    ctx.close()
    assert st2.wait(0) == aok.AOK_E_NOT_RESIDENT
    st2.close()
