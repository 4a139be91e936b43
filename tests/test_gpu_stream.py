"""Residency streaming (Sec. 3.4): only the (chunk, LOD) pairs a camera needs
within the view distance are resident; moving along a path evicts and builds
chunks between frames, and every frame still equals the oracle on every
non-ambiguous pixel."""
import numpy as np
import pytest

import oracle as orc
import scenegen as sg
from gpu_util import compare, decode

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
            compare(decode(hit, t), ref, max_amb_frac=1e-3)
    assert all(s["resident"] < sc.grid[0] * sc.grid[1] * sc.grid[2] for s in stats)
    assert stats[0]["built"] > 0 and any(s["evicted"] > 0 or s["built"] > 0 for s in stats[1:])
    sc.destroy()
    ctx.close()
