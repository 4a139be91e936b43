#!/usr/bin/env python3
"""Benchmark: primary rays/s of the single-view 1920x1080 render of the
4096^3 city world (8^3 chunks of 512^3, 4 LODs, LOD threshold 1 px), one
step = Eq. 1 selection + visibility + per-pixel first-hit cast of one frame
(with the beam pass on, the selection is the first step of the pass's walk,
one launch; then the casting launch).

Prints one JSON line.  `value` is device time (CUDA events on the launch
stream, L2 flushed between steps, scene resident in HBM); `e2e` is the same
metric through aok_render_host (camera in, frame copied to pinned host memory
every step); `roofline` divides the cast kernel's algorithmic bytes (visit
counts from the counting kernel, whose counts equal the oracle's) by its
event time and by the measured HBM copy bandwidth; `cpu_baseline` is the CPU
oracle timed on a bounded pixel sample on this host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank renders its own replica (no collective in the path).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import scenegen as sg  # noqa: E402

METRIC = "primary rays/s + % memory roofline; batched/served vs plain aggregate, p50/p99"
UNIT = "rays/s"
TAU = 1.0
CAM_SEED = 102
BEAM_DEFAULT = True  # the beam pass runs before casting in the timed step
W, H = 1920, 1080
WORKLOAD = "city4096: 4096^3 world, 8x8x8 chunks of 512^3, 4 LODs, crust terrain + 4000 hollow blocks; " \
           "one 1920x1080 view, LOD threshold 1 px, camera seed 102"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


PROFILE = os.path.join(ROOT, "profiles", "cast_kernel_city4096_1080p.md")
KERNEL_SRCS = [os.path.join(ROOT, "paper_2505_02017_gb300", "csrc", f)
               for f in ("aok_kernels.cu", "aok_trace.cuh", "aok_internal.h")]


def kernel_sources_hash():
    """sha256 (16 hex digits) of the sources cast_kernel is compiled from."""
    import hashlib
    h = hashlib.sha256()
    for p in KERNEL_SRCS:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes (read + write) of one cast_kernel launch on this workload from
    the committed ncu summary, if it was taken on the current kernel sources;
    else None (the counters no longer describe the kernel)."""
    import re
    try:
        h = kernel_sources_hash()
        with open(PROFILE) as f:
            m = re.search(r"^traffic: (\d+) bytes per launch, kernel sources sha256 ([0-9a-f]{16})", f.read(), re.M)
    except OSError:
        return None
    return int(m.group(1)) if m and m.group(2) == h else None


class Clocks:
    """nvidia-smi sampler (clocks + throttle reasons) around the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (the job takes as long as its slowest rank)."""
    if dist is None:
        return x
    import torch
    tt = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(units_per_rank: float, world_size: int, seconds: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world_size * units_per_rank / seconds


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def cpu_oracle_sample(world, cam, budget_s=20.0, max_pixels=400_000, gpu_frame=None):
    """Oracle rays/s on a stratified pixel sample of the same frame (all host
    cores).  With the GPU's frame (hit int32 [H, W, 4], t float32 [H, W] on
    the host), also the parity of that sample: pixels the oracle flags
    ambiguous, and non-ambiguous pixels whose voxel, LOD, material, normal or
    hit flag differ or whose distance is off by more than 1e-5 relative."""
    import oracle as orc
    S = orc.OracleScene(world)
    sel = S.select(cam, TAU)
    t0 = time.perf_counter()
    S.prepare(sel)
    prep = time.perf_counter() - t0
    n = W * H
    # calibrate on a small sample, then size the timed one to ~budget_s
    step = 97
    idx = np.arange(0, n, step)
    pix = np.stack([idx % W, idx // W], 1)
    t0 = time.perf_counter()
    S.cast(cam, sel, pix)
    rate = len(idx) / max(time.perf_counter() - t0, 1e-6)
    m = int(min(max_pixels, max(20_000, rate * budget_s)))
    step = max(1, n // m)
    idx = np.arange(0, n, step)
    pix = np.stack([idx % W, idx // W], 1)
    t0 = time.perf_counter()
    ref = S.cast(cam, sel, pix)
    dt = time.perf_counter() - t0
    cores = orc.default_threads()
    out = {"value": len(idx) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"every {step}th pixel of the frame ({len(idx)} rays), FP64 oracle on {cores} threads; "
                     f"oracle DAG build for the frame's LOD selection took {prep:.1f} s and is not timed"}
    if gpu_frame is not None:
        h = np.asarray(gpu_frame[0]).reshape(-1, 4).view(np.uint32)[idx]
        t = np.asarray(gpu_frame[1]).reshape(-1).astype(np.float64)[idx]
        meta = h[:, 3]
        ok = ref["amb"] == 0
        bad = ((((meta >> 19) & 1).astype(np.int32) != ref["hit"]) |
               (h[:, 0].view(np.int32) != ref["x"]) | (h[:, 1].view(np.int32) != ref["y"]) |
               (h[:, 2].view(np.int32) != ref["z"]) | ((meta & 0xFF).astype(np.int32) != ref["lod"]) |
               (((meta >> 8) & 0xFF).astype(np.int32) != ref["mat"]) |
               (((meta >> 16) & 7).astype(np.int32) != ref["normal"]))
        hit = ref["hit"] == 1
        far = np.zeros(len(idx), bool)
        far[hit] = np.abs(t[hit] - ref["dist"][hit]) > 1e-5 * np.maximum(ref["dist"][hit], 1e-30)
        out["parity"] = {"pixels": int(len(idx)), "ambiguous": int((~ok).sum()),
                         "mismatched_non_ambiguous": int(((bad | far) & ok).sum())}
    return out


def time_events(fn, reps, flush, stream):
    """Median and best ms of fn() over reps, L2 flushed before each rep."""
    import torch
    ms = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms), min(ms)


def bench_batched(aok, ctx, scene, world, flush, reps=5):
    """64 walker views of the city world at resolutions drawn from five sizes:
    one aok_render_batch (the autotuner's launch kind; with the grid launch,
    selection, one beam pass for the large views and the cast replayed as one
    CUDA graph) vs 64 separate aok_render launches on one stream, and the same
    batch with its launches issued one by one.  Outputs must be identical."""
    import torch
    cams = sg.batch_cameras(world, 104, 64)
    rays = sum(c.W * c.H for c in cams)
    stream = torch.cuda.current_stream()
    plain = [aok.alloc_frame(c.W, c.H) for c in cams]
    batch = [aok.alloc_frame(c.W, c.H) for c in cams]
    views = [aok.make_view(scene, c, TAU, h, t) for c, (h, t) in zip(cams, batch)]

    def run_plain():
        for c, (h, t) in zip(cams, plain):
            aok.render(ctx, scene, c, TAU, h, t)

    def run_batch():
        aok.render_batch(ctx, views)

    run_plain()
    t0 = time.perf_counter()
    tune_ms = aok.autotune(ctx, views)
    tune_s = time.perf_counter() - t0
    run_batch()
    torch.cuda.synchronize()
    equal = all(torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32), b[1].view(torch.int32))
                for a, b in zip(plain, batch))
    p_med, p_best = time_events(run_plain, reps, flush, stream)
    b_med, b_best = time_events(run_batch, reps, flush, stream)
    aok.set_batch_graph(ctx, False)
    e_med, e_best = time_events(run_batch, reps, flush, stream)
    eager = [aok.alloc_frame(c.W, c.H) for c in cams]
    aok.render_batch(ctx, [aok.make_view(scene, c, TAU, h, t) for c, (h, t) in zip(cams, eager)])
    aok.set_batch_graph(ctx, True)
    torch.cuda.synchronize()
    equal = equal and all(torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32), b[1].view(torch.int32))
                          for a, b in zip(plain, eager))
    ctas, threads, packet = aok.get_launch(ctx)
    # the beam pass runs for views of at least 1.5 M pixels: one launch per
    # such plain render, one for the batch (grid launch)
    big = sum(1 for c in cams if c.W * c.H >= 1_500_000) if BEAM_DEFAULT else 0
    return {"workload": "city4096, 64 views (seed 104), resolutions uniform over "
                        "{320x180, 640x360, 1280x720, 1920x1080, 2560x1440}, tau = 1 px",
            "rays": rays, "plain_rays_per_s": rays / (p_med / 1e3), "batched_rays_per_s": rays / (b_med / 1e3),
            "plain_ms": p_med, "batched_ms": b_med, "plain_best_ms": p_best, "batched_best_ms": b_best,
            "speedup": p_med / b_med, "identical_outputs": bool(equal),
            "graph": True, "eager_batched_ms": e_med, "graph_vs_eager": e_med / b_med, "plain_launches": 128 + big,
            "batched_launches": 2 + (1 if big and ctas == 0 else 0), "views_with_beam_pass": big,
            "autotuned": {"ctas_per_sm": ctas, "threads": threads, "packet_rays": packet,
                          "best_ms": tune_ms, "tune_s": round(tune_s, 2)}}


def bench_walk(aok, ctx, scene, world, flush, n_poses=120):
    """The benchmark frame's metric along a moving camera: a path of poses at
    walker height through the city (1920x1080, tau = 1 px).  Device time: per
    pose the beam pass that selects first (aok_select_beam) and the cast on
    one stream, L2 flushed before each pose.  End to end: the same poses through aok_render_host_async, every
    frame copied to pinned host memory."""
    import torch
    cams = sg.path_cameras(world, 106, n_poses, W, H, n_waypoints=6, span=2500.0, z_lo=64.0, z_hi=400.0,
                           pitch=(-30.0, 5.0))
    stream = torch.cuda.current_stream()
    hit, t = aok.alloc_frame(W, H)
    for cam in cams[:3]:
        aok.render(ctx, scene, cam, TAU, hit, t)
    torch.cuda.synchronize()
    ms = []
    for cam in cams:
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        aok.select_beam(ctx, scene, cam, TAU, stream=stream)
        aok.cast_selected(ctx, scene, cam, hit, t, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    nbuf = 3
    hh = [torch.empty((H, W, 4), dtype=torch.int32, pin_memory=True) for _ in range(nbuf)]
    th = [torch.empty((H, W), dtype=torch.float32, pin_memory=True) for _ in range(nbuf)]
    t0 = time.perf_counter()
    tickets = []
    for k, cam in enumerate(cams):
        if len(tickets) >= nbuf:
            aok.host_frame_wait(ctx, tickets[-nbuf])
        tickets.append(aok.render_host_async(ctx, scene, cam, TAU, hh[k % nbuf], th[k % nbuf]))
    for tk in tickets[-nbuf:]:
        aok.host_frame_wait(ctx, tk)
    e2e_s = time.perf_counter() - t0
    srt = sorted(ms)
    return {"workload": f"city4096, {n_poses}-pose walker path (seed 106, 6 waypoints over 2500 voxels, "
                        "64-400 voxels above the terrain at the waypoints), 1920x1080, tau = 1 px",
            "rays_per_s": W * H * len(ms) / (sum(ms) / 1e3), "frame_ms_median": srt[len(srt) // 2],
            "frame_ms_p99": srt[int(len(srt) * 0.99) - 1], "e2e_rays_per_s": W * H * len(cams) / e2e_s,
            "e2e_api": "aok_render_host_async (3 frames in flight)"}


def bench_served(aok, ctx, base_scene, threads, rates=(200, 500, 1000, 2000, 4000), n_req=1000, n_warm=100):
    """Poisson arrivals over 4 resident worlds (two 4096^3 cities, two 2048^3),
    each request a random walker pose, a resolution from the five sizes and a
    threshold U[0.5, 2] px: continuous-batching server vs serial FIFO renders."""
    import threading
    import torch
    worlds = [sg.World(s) for s in sg.SERVE_WORLDS]
    scenes = [base_scene] + [aok.Scene.from_world(ctx, w, threads) for w in worlds[1:]]
    rng = sg.Rng(105)
    pools = []
    for wi, w in enumerate(worlds):
        pools.append([sg.ground_camera(w, rng.next(), 64, 64) for _ in range(96)])
    out = {"workload": "4 resident worlds (city4096 seeds 2, 5; city2048 seeds 6, 7), Poisson arrivals, "
                       "poses by the walker rule, resolutions from the five sizes, tau ~ U[0.5, 2] px",
           "requests_per_rate": n_req, "warmup_per_rate": n_warm, "rates": []}
    stream = torch.cuda.current_stream()
    for rate in rates:
        reqs = []
        t = 0.0
        for i in range(n_req + n_warm):
            t += -math.log(1.0 - (rng.next() >> 11) * (1.0 / 9007199254740992.0)) / rate
            wi = rng.randint(0, 3)
            W, H = sg.RESOLUTIONS[rng.randint(0, len(sg.RESOLUTIONS) - 1)]
            cam = pools[wi][rng.randint(0, len(pools[wi]) - 1)]
            cam = sg.Camera(cam.origin, cam.R, cam.tan_half_fovy, W, H)
            tau = 0.5 + 1.5 * ((rng.next() >> 11) * (1.0 / 9007199254740992.0))
            reqs.append((t, wi, cam, tau))
        rays = sum(r[2].W * r[2].H for r in reqs[n_warm:])
        # --- served ---
        srv = aok.Server(ctx, max_slots=64, max_batch=16, n_streams=3)
        tickets = [None] * len(reqs)
        lat = [None] * len(reqs)
        done_ns = [0] * len(reqs)

        def submitter(t0):
            for i, (ta, wi, cam, tau) in enumerate(reqs):
                d = t0 + ta - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets[i] = srv.submit(scenes[wi], cam, tau)

        def releaser():
            for i in range(len(reqs)):
                while tickets[i] is None:
                    time.sleep(0.0001)
                st, f = srv.wait(tickets[i], 120000)
                s_ns, d_ns = srv.times(tickets[i])
                lat[i] = (d_ns - s_ns) / 1e6
                done_ns[i] = d_ns
                srv.release(tickets[i])

        t0 = time.perf_counter()
        th1 = threading.Thread(target=submitter, args=(t0,))
        th2 = threading.Thread(target=releaser)
        th1.start(); th2.start(); th1.join(); th2.join()
        srv.stop()
        span = (max(done_ns[n_warm:]) - min(done_ns[n_warm:])) / 1e9
        ls = sorted(lat[n_warm:])
        served = {"p50_ms": ls[len(ls) // 2], "p99_ms": ls[int(len(ls) * 0.99)],
                  "req_per_s": (n_req - 1) / max(span, 1e-9), "rays_per_s": rays / max(span, 1e-9)}
        # --- serial FIFO plain renders of the same trace ---
        frames = {}
        lat2 = []
        t0 = time.perf_counter()
        t_first = t_last = None
        for i, (ta, wi, cam, tau) in enumerate(reqs):
            d = t0 + ta - time.perf_counter()
            if d > 0:
                time.sleep(d)
            key = (cam.W, cam.H)
            if key not in frames:
                frames[key] = aok.alloc_frame(cam.W, cam.H)
            h, tt = frames[key]
            aok.render(ctx, scenes[wi], cam, tau, h, tt)
            stream.synchronize()
            now = time.perf_counter()
            if i >= n_warm:
                lat2.append((now - (t0 + ta)) * 1e3)
                t_first = now if t_first is None else t_first
                t_last = now
        ls2 = sorted(lat2)
        span2 = t_last - t_first
        serial = {"p50_ms": ls2[len(ls2) // 2], "p99_ms": ls2[int(len(ls2) * 0.99)],
                  "req_per_s": (n_req - 1) / max(span2, 1e-9), "rays_per_s": rays / max(span2, 1e-9)}
        out["rates"].append({"arrival_req_per_s": rate, "served": served, "serial_plain": serial})
    for sc in scenes[1:]:
        sc.destroy()
    return out


def bench_tiles(aok, ctx, scene, world, flush, reps=20):
    """The paper's tile-chunk pipeline (aok_render_tiles) against the per-ray
    march (aok_render) on the benchmark frame: first frame (no Hi-Z history)
    and steady state (the previous frame's Hi-Z), same outputs required."""
    import torch
    cam = sg.ground_camera(world, CAM_SEED, W, H)
    hit, t = aok.alloc_frame(W, H)
    hit2, t2 = aok.alloc_frame(W, H)
    stream = torch.cuda.current_stream()

    def first():
        aok.tiles_forget(ctx)
        aok.render_tiles(ctx, scene, cam, TAU, hit2, t2)

    out = {"workload": WORKLOAD}
    for name, fn in (("march", lambda: aok.render(ctx, scene, cam, TAU, hit, t)), ("tiles_first_frame", first),
                     ("tiles_steady", lambda: aok.render_tiles(ctx, scene, cam, TAU, hit2, t2))):
        for _ in range(3):
            fn()
        out[name + "_ms_median"], out[name + "_ms_best"] = time_events(fn, reps, flush, stream)
        if name != "march":
            out[name + "_stats"] = aok.tiles_stats(ctx)
    out["identical_outputs"] = bool(torch.equal(hit, hit2) and torch.equal(t.view(torch.int32), t2.view(torch.int32)))
    return out


def bench_beam(aok, ctx, scene, world, flush, reps=20):
    """The beam pass (aok_set_beam) on and off for the benchmark frame and four
    more walker views of the same world, 1920x1080: render time (selection,
    beam pass, cast) and interior-node visits per ray; outputs must match."""
    import torch
    stream = torch.cuda.current_stream()
    out = {"workload": "city4096 walker views, 1920x1080, tau = 1 px"}
    for seed in (CAM_SEED, 5, 7, 11, 23):
        cam = sg.ground_camera(world, seed, W, H)
        row = {}
        frames = []
        for on in (False, True):
            aok.set_beam(ctx, on)
            hit, t = aok.alloc_frame(W, H)
            fn = lambda: aok.render(ctx, scene, cam, TAU, hit, t)  # noqa: E731
            for _ in range(3):
                fn()
            med, _ = time_events(fn, reps, flush, stream)
            counts = torch.zeros(W * H * 3, dtype=torch.int32, device="cuda")
            hc, tc = aok.alloc_frame(W, H)
            aok.render_counted(ctx, scene, cam, TAU, hc, tc, counts)
            torch.cuda.synchronize()
            key = "on" if on else "off"
            row[key + "_ms_median"] = med
            row[key + "_interior_visits_per_ray"] = round(float(counts.view(-1, 3)[:, 0].double().mean()), 2)
            frames.append((hit, t))
        row["identical_outputs"] = bool(torch.equal(frames[0][0], frames[1][0]) and
                                        torch.equal(frames[0][1].view(torch.int32), frames[1][1].view(torch.int32)))
        out[f"camera_seed_{seed}"] = row
    aok.set_beam(ctx, BEAM_DEFAULT)
    return out


def bench_color(aok, ctx, threads, flush, reps=20):
    """Colour-block compression (Sec. 3.3) on the city world with layered
    (coherent) colours: colour bytes resident and the benchmark frame's time
    with raw arrays, lossless blocks (e_c = 0) and the paper's e_c = 0.05."""
    import torch
    world = sg.World(sg.CITY_4096_LAYERED)
    bw = aok.BuiltWorld(world, threads)
    cam = sg.ground_camera(world, CAM_SEED, W, H)
    stream = torch.cuda.current_stream()
    out = {"workload": "city4096 with layered colours (8-voxel strata x 64-voxel column cells, 1/64 hashed), "
                       "1920x1080, camera seed 102, tau = 1 px"}
    frames = {}
    for name, tol in (("raw", None), ("lossless_e0", 0.0), ("lossy_e0.05", 0.05)):
        sc = aok.Scene.from_world(ctx, world, built=bw, color_tol=tol)
        hit, t = aok.alloc_frame(W, H)
        for _ in range(3):
            aok.render(ctx, sc, cam, TAU, hit, t)
        med, best = time_events(lambda: aok.render(ctx, sc, cam, TAU, hit, t), reps, flush, stream)
        out[name] = {"color_bytes": sc.usage()["color_bytes"], "frame_ms_median": med, "frame_ms_best": best}
        frames[name] = (hit, t)
        sc.destroy()
    r, l0, l5 = frames["raw"], frames["lossless_e0"], frames["lossy_e0.05"]
    out["lossless_identical"] = bool(torch.equal(r[0], l0[0]) and torch.equal(r[1], l0[1]))
    meta_r, meta_5 = r[0].view(-1, 4)[:, 3], l5[0].view(-1, 4)[:, 3]
    out["lossy_pixels_with_other_colour"] = float(((meta_r >> 8) & 0xFF).ne((meta_5 >> 8) & 0xFF).float().mean())
    return out


def bench_open(aok, ctx, threads, n_poses=300):
    """Open world 65536x65536x1024 (128x128x2 chunks of 512^3, 4 LODs), view
    distance 16384: along a 300-pose path at 2560x1440, only the (chunk, LOD)
    pairs within the view distance are resident (streamed between frames);
    per frame the render (selection a1+a2 and cast a4-a7 in one call) is
    timed, and the selection alone once more after it."""
    import torch
    from paper_2505_02017_gb300.stream import Streamer
    spec = sg.OPEN_65536
    world = sg.World(spec)
    cams = sg.path_cameras(world, 103, n_poses, 2560, 1440)
    scene = aok.Scene(ctx, spec, node_words=512 << 20, leaves=256 << 20, mat_bytes=16 << 30)
    st = Streamer(ctx, world, scene, threads)
    hit, t = aok.alloc_frame(2560, 1440)
    hit2, t2 = aok.alloc_frame(2560, 1440)
    hit3, t3 = aok.alloc_frame(2560, 1440)
    stream = torch.cuda.current_stream()
    sel_ms, cast_ms, tiles_ms, other_ms, host = [], [], [], [], []
    tiles_same = other_same = True
    aok.tiles_forget(ctx)
    # each timed region starts behind a short spin kernel, so that the host's
    # launch latency after a synchronisation is not counted as frame time
    gate = 200_000  # cycles, ~0.1 ms
    frame = []
    for i, cam in enumerate(cams):
        host.append(st.update(cam, TAU))
        e = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        torch.cuda._sleep(gate)
        e[0].record(stream)
        aok.render(ctx, scene, cam, TAU, hit, t, stream=stream)  # selection + cast, one call
        e[1].record(stream)
        # the same frame with the beam pass the other way round
        aok.set_beam(ctx, not BEAM_DEFAULT)
        torch.cuda._sleep(gate)
        e[5].record(stream)
        aok.render(ctx, scene, cam, TAU, hit3, t3, stream=stream)
        e[6].record(stream)
        aok.set_beam(ctx, BEAM_DEFAULT)
        # the paper's tile-chunk pipeline on the same frame (Hi-Z history: the previous pose)
        aok.render_tiles(ctx, scene, cam, TAU, hit2, t2, stream=stream)
        e[2].record(stream)
        torch.cuda._sleep(gate)
        e[3].record(stream)
        aok.select_chunks(ctx, scene, cam, TAU, stream=stream)  # the selection alone
        e[4].record(stream)
        e[4].synchronize()
        frame.append(e[0].elapsed_time(e[1]))
        tiles_ms.append(e[6].elapsed_time(e[2]))
        other_ms.append(e[5].elapsed_time(e[6]))
        other_same &= torch.equal(hit, hit3) and torch.equal(t.view(torch.int32), t3.view(torch.int32))
        sel_ms.append(e[3].elapsed_time(e[4]))
        tiles_same &= torch.equal(hit, hit2) and torch.equal(t.view(torch.int32), t2.view(torch.int32))
    cast_ms = [f - s_ for f, s_ in zip(frame, sel_ms)]
    rays = 2560 * 1440
    srt = sorted(frame)
    out = {"workload": "open65536: 65536x65536x1024, 128x128x2 chunks of 512^3, 4 LODs, view distance 16384; "
                       f"{n_poses}-pose path (seed 103), 2560x1440, tau = 1 px",
           "rays_per_s": rays * len(frame) / (sum(frame) / 1e3),
           "frame_ms_median": srt[len(srt) // 2], "frame_ms_p99": srt[int(len(srt) * 0.99) - 1],
           "select_ms_mean": sum(sel_ms) / len(sel_ms), "cast_ms_mean": sum(cast_ms) / len(cast_ms),
           "max_resident_chunks": st.max_resident, "max_resident_mb": round(st.max_bytes / 1e6, 1),
           "first_frame_built": host[0]["built"], "first_frame_build_s": round(host[0]["build_s"], 2),
           "later_frames_built_total": sum(h["built"] for h in host[1:]),
           "later_frames_evicted_total": sum(h["evicted"] for h in host[1:]),
           "streaming_host_s_total": round(sum(h["plan_s"] + h["build_s"] + h["upload_s"] for h in host), 2),
           "tile_pipeline": {"frame_ms_median": sorted(tiles_ms)[len(tiles_ms) // 2],
                             "march_frame_ms_median": srt[len(srt) // 2],
                             "identical_outputs_all_poses": bool(tiles_same)},
           ("march_without_beam" if BEAM_DEFAULT else "march_with_beam"): {
               "frame_ms_median": sorted(other_ms)[len(other_ms) // 2],
               "identical_outputs_all_poses": bool(other_same)}}
    scene.destroy()
    return out


def _chunks_met(spec, cam, pix, tmax):
    """Chunk regions whose cell meets the segment [0, tmax[i]] of each sampled ray."""
    import oracle as orc
    M = spec.chunk
    gx, gy, gz = spec.grid
    cz, cy, cx = np.meshgrid(np.arange(gz), np.arange(gy), np.arange(gx), indexing="ij")
    lo = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], 1).astype(np.float64) * M
    hi = lo + M
    o = cam.origin.astype(np.float64)
    keep = np.zeros(len(lo), bool)
    for i, (px, py) in enumerate(pix):
        d = orc.ray_dir(cam, int(px), int(py)).astype(np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            t1, t2 = (lo - o) / d, (hi - o) / d
        tn = np.nanmax(np.where(d == 0, np.where((o >= lo) & (o <= hi), -np.inf, np.inf), np.minimum(t1, t2)), 1)
        tf = np.nanmin(np.where(d == 0, np.where((o >= lo) & (o <= hi), np.inf, -np.inf), np.maximum(t1, t2)), 1)
        keep |= (tn <= tf) & (tf >= 0) & (tn <= tmax[i])
    return keep


def cpu_scaling(threads):
    """Oracle rays/s at 1 thread and at all host threads for a single128 frame
    (256x256, camera seed 101), the city4096 1080p frame and one open65536
    2560x1440 frame (pose 150 of the path; the oracle is given the chunks the
    sampled rays meet up to the GPU's hit distance).  DAG builds are not timed."""
    import torch
    import oracle as orc
    import paper_2505_02017_gb300 as aok
    from paper_2505_02017_gb300.stream import Streamer
    res = {}

    def rate(S, cam, sel, pix, nthr, view_dist=0.0):
        S.cast(cam, sel, pix[: max(1, len(pix) // 20)], view_dist=view_dist, threads=nthr)  # warm
        t0 = time.perf_counter()
        S.cast(cam, sel, pix, view_dist=view_dist, threads=nthr)
        return len(pix) / (time.perf_counter() - t0)

    def stride_pix(cam, n):
        step = max(1, cam.W * cam.H // n)
        idx = np.arange(0, cam.W * cam.H, step)
        return np.stack([idx % cam.W, idx // cam.W], 1)

    for name, spec, cam_fn, n1 in (("single128_256x256", sg.SINGLE_128, lambda w: sg.orbit_camera(w.spec, 101, 256, 256), 20000),
                                   ("city4096_1080p", sg.CITY_4096, lambda w: sg.ground_camera(w, CAM_SEED, W, H), 4000)):
        w = sg.World(spec)
        cam = cam_fn(w)
        S = orc.OracleScene(w)
        sel = S.select(cam, TAU)
        S.prepare(sel)
        res[name] = {"threads_1": rate(S, cam, sel, stride_pix(cam, n1), 1),
                     f"threads_{threads}": rate(S, cam, sel, stride_pix(cam, n1 * threads), threads)}
    spec = sg.OPEN_65536
    w = sg.World(spec)
    ctx = aok.Context(0)
    sc = aok.Scene(ctx, spec, node_words=512 << 20, leaves=256 << 20, mat_bytes=16 << 30)
    st = Streamer(ctx, w, sc, threads)
    cam = sg.path_cameras(w, 103, 300, 2560, 1440)[150]
    st.update(cam, TAU)
    hit, t = aok.alloc_frame(cam.W, cam.H)
    aok.render(ctx, sc, cam, TAU, hit, t)
    torch.cuda.synchronize()
    pix = stride_pix(cam, 400)
    idx = pix[:, 1] * cam.W + pix[:, 0]
    meta = hit.view(-1, 4)[:, 3].cpu().numpy()[idx]
    dist = np.where((meta >> 19) & 1, t.view(-1).cpu().numpy()[idx], spec.view_dist)
    dn = np.array([np.linalg.norm(orc.ray_dir(cam, int(x), int(y)).astype(np.float64)) for x, y in pix])
    plan = st.plan(cam, TAU)
    sel = np.where(_chunks_met(spec, cam, pix, dist / dn + 2.0) & (plan != 0xFF), plan.astype(np.int32), -1)
    sel = sel.astype(np.int8)
    S = orc.OracleScene(w)
    S.prepare(sel)
    res["open65536_1440p_pose150"] = {"threads_1": rate(S, cam, sel, pix, 1, spec.view_dist),
                                      f"threads_{threads}": rate(S, cam, sel, pix, threads, spec.view_dist)}
    sc.destroy()
    ctx.close()
    print(json.dumps({"oracle_rays_per_s": res, "host_threads": threads}), flush=True)


def scene_grid(spec):
    return (spec.wx // spec.chunk, spec.wy // spec.chunk, spec.wz // spec.chunk)


def bench_open_async(aok, ctx, threads, n_poses=300, fps=60.0, from_file=False, prefetch=(8, 2),
                     build_cache_mb=4096):
    """The open-world path with asynchronous residency (aok_stream): frames
    are paced at `fps`; each frame installs what the background workers
    loaded since the previous one (coarser LODs first, then nearest), renders
    with stand-in LODs where a load is still missing, and never waits for a
    load.  The first pose is loaded completely before the path starts.  The
    loaders build chunks from the procedural world, or (from_file) read them
    from a chunk-blob file holding every (chunk, LOD) the path plans, as the
    paper streams preprocessed chunks from disk.  prefetch = (frames,
    samples) also loads the plans of the camera extrapolated up to `frames`
    frames ahead along its last displacement (aok_stream_set_prefetch);
    None plans the current camera only, as the paper does.  The procedural
    source keeps up to build_cache_mb of built blobs in host memory
    (aokb_source_set_cache; 0: none)."""
    import torch
    from paper_2505_02017_gb300.stream import AsyncStreamer, Streamer
    spec = sg.OPEN_65536
    world = sg.World(spec)
    cams = sg.path_cameras(world, 103, n_poses, 2560, 1440)
    file_info = {}
    blobs = None
    path = None
    if from_file:
        t0 = time.perf_counter()
        plan_scene = aok.Scene(ctx, spec, node_words=1 << 16, leaves=1 << 16, mat_bytes=1 << 16)
        planner = Streamer(ctx, world, plan_scene, threads)
        masks = {}
        for cam in cams:
            plan = planner.plan(cam, TAU)
            for c in np.nonzero(plan != 0xFF)[0]:
                masks[int(c)] = masks.get(int(c), 0) | (1 << int(plan[c]))
        plan_scene.destroy()
        chunks = np.array(sorted(masks), np.int64)
        built = aok.BuiltWorld(world, threads, chunks=chunks,
                               lod_masks=np.array([masks[int(c)] for c in chunks], np.uint32))
        t1 = time.perf_counter()
        path = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"aok_open65536_path_{os.getpid()}.aokb")
        n = aok.BlobFile.write(path, built, scene_grid(spec), spec.chunk, spec.n_lods)
        built.close()
        t2 = time.perf_counter()
        file_info = {"file_entries": n, "file_mb": round(os.path.getsize(path) / 1e6, 1),
                     "file_build_s": round(t1 - t0, 2), "file_write_s": round(t2 - t1, 2)}
        blobs = aok.BlobFile(path)
    scene = aok.Scene(ctx, spec, node_words=512 << 20, leaves=256 << 20, mat_bytes=16 << 30)
    st = AsyncStreamer(ctx, world, scene, threads, blobs=blobs, build_cache_mb=0 if from_file else build_cache_mb)
    if prefetch:
        st.set_prefetch(*prefetch)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    st.update(cams[0], TAU, stream=stream)
    st.wait()
    st.update(cams[0], TAU, stream=stream)
    warm_s = time.perf_counter() - t0
    hit, t = aok.alloc_frame(2560, 1440)
    render_ms, update_ms, missing, shown = [], [], [], []
    period = 1.0 / fps
    for cam in cams:
        f0 = time.perf_counter()
        st.update(cam, TAU, stream=stream)
        update_ms.append(1e3 * (time.perf_counter() - f0))
        sst = st.stats()
        missing.append(sst["missing"])
        shown.append(1.0 - sst["missing"] / max(1, sst["planned"]))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(200_000)  # the timed region starts after the launch below is queued
        e0.record(stream)
        aok.render(ctx, scene, cam, TAU, hit, t, stream=stream)
        e1.record(stream)
        e1.synchronize()
        render_ms.append(e0.elapsed_time(e1))
        rest = period - (time.perf_counter() - f0)
        if rest > 0:
            time.sleep(rest)
    s = st.stats()
    cache = st.source_stats()
    st.close()
    scene.destroy()
    if blobs is not None:
        blobs.close()
        os.remove(path)
    rs, us = sorted(render_ms), sorted(update_ms)
    return {"workload": f"open65536 path (seed 103), {n_poses} poses at 2560x1440 paced at {fps:g} frames/s, "
                        f"tau = 1 px; {threads} loader threads "
                        + ("reading a chunk-blob file" if from_file else "building chunks procedurally")
                        + (f"; prefetch {prefetch[0]} frames ahead ({prefetch[1]} extrapolated plans)" if prefetch
                           else "; no prefetch")
                        + (f"; {build_cache_mb} MB host blob cache" if build_cache_mb and not from_file else ""),
            **file_info,
            "first_pose_load_s": round(warm_s, 2),
            "render_ms_median": rs[len(rs) // 2], "render_ms_p99": rs[int(len(rs) * 0.99) - 1],
            "update_ms_median": us[len(us) // 2], "update_ms_p99": us[int(len(us) * 0.99) - 1],
            "frames_with_every_planned_lod": sum(m == 0 for m in missing) / len(missing),
            "planned_lods_installed_frac_median": sorted(shown)[len(shown) // 2],
            "planned_lods_installed_frac_min": min(shown),
            "regions_missing_median": sorted(missing)[len(missing) // 2], "max_regions_missing": max(missing), "max_resident_chunks": s["max_resident"],
            "max_resident_mb": round(s["max_resident_bytes"] / 1e6, 1), "installed_total": s["installed_total"],
            "evicted_total": s["evicted_total"], "cancelled_total": s["cancelled_total"],
            "failed_total": s["failed_total"], "deferred_total": s["deferred_total"],
            "ahead_installed_total": s["ahead_installed_total"],
            **({"builder_cache": cache} if cache else {})}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, same workload/metric, bounded sample per step."""
    rank, world_size, _ = dist_env()
    if rank != 0:
        return
    import oracle as orc
    world = sg.World(sg.CITY_4096)
    cam = sg.ground_camera(world, CAM_SEED, W, H)
    S = orc.OracleScene(world)
    sel = S.select(cam, TAU)
    S.prepare(sel)
    n = W * H
    per_step = 4096
    rng = np.random.default_rng(0)
    for _ in range(args.warmup):
        idx = rng.integers(0, n, per_step)
        S.cast(cam, sel, np.stack([idx % W, idx // W], 1))
    t0 = time.perf_counter()
    rays = 0
    for _ in range(args.steps):
        idx = rng.integers(0, n, per_step)
        S.cast(cam, sel, np.stack([idx % W, idx // W], 1))
        rays += per_step
    dt = time.perf_counter() - t0
    v = rays / dt
    cores = orc.default_threads()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": f"{per_step} random pixels of the frame per step"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} random pixels per step, {args.steps} steps"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-open", action="store_true")
    ap.add_argument("--no-tiles", action="store_true")
    ap.add_argument("--no-color", action="store_true")
    ap.add_argument("--no-beam-ab", action="store_true")
    ap.add_argument("--no-walk", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--cpu-scaling", action="store_true",
                    help="print the oracle's 1-thread / all-thread rays/s for three workloads and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.cpu_scaling:
        return cpu_scaling(args.threads or os.cpu_count() or 1)

    import torch
    import paper_2505_02017_gb300 as aok

    rank, world_size, local_rank = dist_env()
    dist = None
    if world_size > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = local_rank if world_size > 1 else 0
    torch.cuda.set_device(dev)
    threads = args.threads or os.cpu_count() or 1

    # ---- scene: build every chunk x LOD on the host, upload (untimed) ----
    t0 = time.perf_counter()
    world = sg.World(sg.CITY_4096)
    built = aok.BuiltWorld(world, threads)
    t_build = time.perf_counter() - t0
    ctx = aok.Context(dev)
    aok.set_beam(ctx, BEAM_DEFAULT)
    t0 = time.perf_counter()
    scene = aok.Scene.from_world(ctx, world, built=built)
    t_upload = time.perf_counter() - t0
    cam = sg.ground_camera(world, CAM_SEED, W, H)
    stream = torch.cuda.current_stream()
    hit, t = aok.alloc_frame(W, H, device=f"cuda:{dev}")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=f"cuda:{dev}")  # > 129 MB L2

    # ---- algorithmic bytes of this frame (counting kernel, untimed) ----
    # The method's traversal (no beam restart) visits what the oracle counts;
    # its bytes are the roofline's numerator.  With the restart the casting
    # kernel reads fewer: reported beside it.
    counts = torch.zeros((H, W, 3), dtype=torch.int32, device=f"cuda:{dev}")

    def frame_bytes(beam):
        aok.set_beam(ctx, beam)
        aok.render_counted(ctx, scene, cam, TAU, hit, t, counts)
        torch.cuda.synchronize()
        c = counts.view(-1, 3).to(torch.int64).sum(0).tolist()
        return 8 * c[0] + 8 * c[1] + c[2] + 20 * W * H, c  # node visits, leaf visits, resolve, output

    algo_bytes, algo_counts = frame_bytes(False)
    restart_bytes, restart_counts = frame_bytes(True)
    aok.set_beam(ctx, BEAM_DEFAULT)
    del counts
    n_visible = aok.select_chunks(ctx, scene, cam, TAU, count=True)
    meta = hit.view(-1, 4)[:, 3]
    is_hit = ((meta >> 19) & 1) == 1
    hit_frac = float(is_hit.float().mean().item())
    lod_hist = torch.bincount((meta[is_hit] & 0xFF).long(), minlength=4).tolist()

    # ---- warmup ----
    for _ in range(args.warmup):
        aok.render(ctx, scene, cam, TAU, hit, t)
    torch.cuda.synchronize()

    # ---- timed: K steps, L2 flushed between steps; a step is the beam pass that
    # selects the frame table as its first step (aok_select_beam; the selection
    # kernel alone when the pass is off), then the cast, events around each ----
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = Clocks(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        aok.select_beam(ctx, scene, cam, TAU, stream=stream)
        ev[k][1].record(stream)
        aok.cast_selected(ctx, scene, cam, hit, t, stream=stream)
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    time.sleep(0.3)
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[2]) for e in ev]
    beam_ms = [e[0].elapsed_time(e[1]) for e in ev]  # selection inside the pass
    cast_ms = [e[1].elapsed_time(e[2]) for e in ev]
    # the same frame with the selection kernel before the pass (untimed for the value)
    split = []
    for _ in range(20):
        flush.zero_()
        es = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        es[0].record(stream)
        aok.select_chunks(ctx, scene, cam, TAU, stream=stream)
        es[1].record(stream)
        aok.beam_selected(ctx, scene, cam, stream=stream)
        es[2].record(stream)
        split.append(es)
    torch.cuda.synchronize()
    split_select_ms = statistics.median([e[0].elapsed_time(e[1]) for e in split])
    split_pass_ms = statistics.median([e[1].elapsed_time(e[2]) for e in split])
    total_ms = sum(step_ms)
    if dist:
        total_ms = max_over_ranks(total_ms, dist, f"cuda:{dev}")
    rays = W * H
    value = job_rate(rays * args.steps, world_size, total_ms / 1000.0)
    cast_avg = sum(cast_ms) / len(cast_ms)
    hbm, peak_kind = peaks()
    achieved = algo_bytes / (cast_avg / 1000.0) / 1e9
    # the library's own read microbenchmark: L2-resident (64 MB) and HBM (4 GB) buffers
    l2_gbs = aok.read_bandwidth(ctx, 64 << 20, 200)
    hbm_read_gbs = aok.read_bandwidth(ctx, 4 << 30, 5)

    # ---- e2e: public API with host buffers (camera in, frame copied out every step) ----
    # pipelined (aok_render_host_async: a frame's render overlaps the previous
    # frame's copy; every frame lands in its own pinned host buffer) and
    # synchronous (aok_render_host: render, copy, wait)
    nbuf = 3
    hh = [torch.empty((H, W, 4), dtype=torch.int32, pin_memory=True) for _ in range(nbuf)]
    th = [torch.empty((H, W), dtype=torch.float32, pin_memory=True) for _ in range(nbuf)]
    e2e_steps = max(3, min(args.steps, 50))
    for k in range(3):
        aok.host_frame_wait(ctx, aok.render_host_async(ctx, scene, cam, TAU, hh[k], th[k]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = []
    for k in range(e2e_steps):
        if len(tickets) >= nbuf:  # the buffer about to be reused must hold a finished frame
            aok.host_frame_wait(ctx, tickets[-nbuf])
        tickets.append(aok.render_host_async(ctx, scene, cam, TAU, hh[k % nbuf], th[k % nbuf]))
    for tk in tickets[-nbuf:]:
        aok.host_frame_wait(ctx, tk)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = job_rate(rays, world_size, max_over_ranks(e2e_s, dist, f"cuda:{dev}"))
    for _ in range(3):
        aok.render_host(ctx, scene, cam, TAU, hh[0], th[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        aok.render_host(ctx, scene, cam, TAU, hh[0], th[0])
    e2e_sync_s = (time.perf_counter() - t0) / e2e_steps
    e2e_sync = job_rate(rays, world_size, max_over_ranks(e2e_sync_s, dist, f"cuda:{dev}"))

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world_size, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i64/f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rays_per_step": rays, "parallelism": f"replicas x{world_size}",
                   "l2": "flushed between steps (512 MB write)", "scene_build_s": round(t_build, 2),
                   "scene_upload_s": round(t_upload, 2), "hit_frac": hit_frac, "hit_lod_hist": lod_hist, "visible_chunks": n_visible,
                   "scene_bytes": {"nodes": built.node_words * 4, "leaves": built.leaves * 8,
                                   "mats": built.mat_bytes}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": profiled_traffic(), "kernel": "cast_kernel", "peak_kind": f"{peak_kind} hbm_gbs",
                     "algo_bytes_per_launch": algo_bytes, "algo_bytes_per_ray": algo_bytes / rays,
                     "algo_bytes_def": "oracle traversal visits (no beam restart): 8 B per interior and per leaf "
                                       "visit, 4 B per earlier-sibling count (8 B for leaf masks) + 1 B per hit, "
                                       "20 B output; counting kernel equal to the oracle per pixel",
                     "visits_per_ray": [algo_counts[0] / rays, algo_counts[1] / rays],
                     "bytes_read_with_beam_restart": restart_bytes,
                     "frac_on_restart_bytes": restart_bytes / (cast_avg / 1000.0) / 1e9 / hbm,
                     "cast_ms": cast_avg, "cast_ms_median": statistics.median(cast_ms),
                     "cast_ms_best": min(cast_ms),
                     "l2_read_gbs": l2_gbs, "frac_of_l2_read": achieved / l2_gbs,
                     "hbm_read_gbs": hbm_read_gbs},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 52, "d2h_bytes_per_step": rays * 20,
                "api": "aok_render_host_async (3 frames in flight) + aok_host_frame_wait",
                "ms_per_step": 1e3 * e2e_s, "synchronous_value": e2e_sync,
                "synchronous_api": "aok_render_host"},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
        "wall_s_timed": wall,
        "beam_pass": {"on": BEAM_DEFAULT, "select_and_pass_ms_median": statistics.median(beam_ms),
                      "split": {"select_ms_median": split_select_ms, "pass_ms_median": split_pass_ms}},
    }
    # The records after the headline: one that fails is reported as
    # {"error": ...} in its place and the line is still printed.
    def record(key, fn, *a, **kw):
        try:
            out[key] = fn(*a, **kw)
        except Exception as ex:  # noqa: BLE001
            out[key] = {"error": f"{type(ex).__name__}: {ex}"}
        return out[key]

    if not args.no_beam_ab:
        out["beam_pass"]["on_off"] = record("beam_on_off", bench_beam, aok, ctx, scene, world, flush)
        del out["beam_on_off"]
    if not args.no_walk:
        record("walk", bench_walk, aok, ctx, scene, world, flush)
    if not args.no_tiles:
        record("tile_pipeline", bench_tiles, aok, ctx, scene, world, flush)
    if not args.no_color:
        record("color_blocks", bench_color, aok, ctx, threads, flush)
    if not args.no_batch:
        record("batched", bench_batched, aok, ctx, scene, world, flush)
    if not args.no_serve:
        record("served", bench_served, aok, ctx, scene, threads)
    if not args.no_open:
        record("open_world", bench_open, aok, ctx, threads)
        record("open_world_async", bench_open_async, aok, ctx, threads)
        plain = record("open_world_async_plain", bench_open_async, aok, ctx, threads, prefetch=None,
                       build_cache_mb=0)
        del out["open_world_async_plain"]
        if "error" not in out["open_world_async"]:
            out["open_world_async"]["without_prefetch_or_cache"] = plain if "error" in plain else {
                k: plain[k] for k in ("frames_with_every_planned_lod", "planned_lods_installed_frac_median",
                                      "planned_lods_installed_frac_min", "regions_missing_median",
                                      "installed_total", "max_resident_mb")}
        record("open_world_async_file", bench_open_async, aok, ctx, threads, from_file=True)
    if rank == 0 and world_size == 1 and not args.no_cpu_baseline:
        try:
            aok.render(ctx, scene, cam, TAU, hit, t)
            torch.cuda.synchronize()
            gpu_frame = (hit.cpu().numpy(), t.cpu().numpy())
        except Exception:  # noqa: BLE001 -- the oracle is still timed, without the parity check
            gpu_frame = None
        record("cpu_baseline", cpu_oracle_sample, world, cam, gpu_frame=gpu_frame)
    # the records a reader of the line's tail needs, last
    summ = {"device_rays_per_s": out["value"], "e2e_rays_per_s": out["e2e"]["value"],
            "cast_ms": out["roofline"]["cast_ms"], "roofline_frac": out["roofline"]["frac"]}
    if "walk" in out and "error" not in out["walk"]:
        summ["walk_rays_per_s"] = out["walk"]["rays_per_s"]
        summ["walk_e2e_rays_per_s"] = out["walk"]["e2e_rays_per_s"]
    if "batched" in out and "error" not in out["batched"]:
        b = out["batched"]
        summ["batched"] = {"rays_per_s": b["batched_rays_per_s"], "plain_rays_per_s": b["plain_rays_per_s"],
                           "speedup": b["speedup"], "graph": b["graph"], "identical": b["identical_outputs"]}
    if "served" in out and "error" not in out["served"]:
        summ["served"] = {str(r["arrival_req_per_s"]): {"req_per_s": round(r["served"]["req_per_s"], 1),
                                                        "p50_ms": round(r["served"]["p50_ms"], 3),
                                                        "p99_ms": round(r["served"]["p99_ms"], 3),
                                                        "serial_p99_ms": round(r["serial_plain"]["p99_ms"], 3)}
                          for r in out["served"]["rates"]}
    if "open_world" in out and "error" not in out["open_world"]:
        summ["open_world_frame_ms_median"] = out["open_world"]["frame_ms_median"]
    for k in ("open_world_async", "open_world_async_file"):
        if k in out and "error" not in out[k]:
            summ[k] = {"installed_median": out[k]["planned_lods_installed_frac_median"],
                       "frames_with_every_planned_lod": out[k]["frames_with_every_planned_lod"]}
    errors = [k for k, v in out.items() if isinstance(v, dict) and "error" in v]
    if isinstance(out["beam_pass"].get("on_off"), dict) and "error" in out["beam_pass"]["on_off"]:
        errors.append("beam_pass.on_off")
    if errors:
        summ["records_failed"] = errors
    if "cpu_baseline" in out and "value" in out["cpu_baseline"]:
        summ["cpu_oracle_rays_per_s"] = out["cpu_baseline"]["value"]
    out["summary"] = summ
    if rank == 0:
        print(json.dumps(out), flush=True)
    try:
        scene.destroy()
        ctx.close()
    except Exception:  # noqa: BLE001 -- after a failed record the context may be unusable
        if not errors:
            raise
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
