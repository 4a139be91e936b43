"""Helpers of the GPU parity tests: decode the library's frame and compare it
with oracle results.

Tolerances (the path's accuracy contract): on every pixel the oracle does not
flag as ambiguous, the hit flag, voxel coordinate, LOD, material and normal
are bit-exact and the hit distance agrees within 1e-5 relative error; the
ambiguous fraction is reported and bounded by the caller."""
import numpy as np

DIST_RTOL = 1e-5


def decode(hit, t):
    """hit int32[H, W, 4] / t float32[H, W] (torch or numpy) -> dict of flat arrays."""
    h = hit.cpu().numpy() if hasattr(hit, "cpu") else np.asarray(hit)
    tt = t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)
    h = h.reshape(-1, 4).view(np.uint32)
    meta = h[:, 3]
    return {"x": h[:, 0].view(np.int32), "y": h[:, 1].view(np.int32), "z": h[:, 2].view(np.int32),
            "lod": (meta & 0xFF).astype(np.int32), "mat": ((meta >> 8) & 0xFF).astype(np.int32),
            "normal": ((meta >> 16) & 7).astype(np.int32), "hit": ((meta >> 19) & 1).astype(np.int32),
            "dist": tt.reshape(-1).astype(np.float64)}


def compare(gpu, ref, idx=None, max_amb_frac=1e-4, min_pixels_checked=1):
    """gpu: decode() output (full frame); ref: oracle records for pixel indices idx
    (row-major, default all).  Returns (checked, ambiguous)."""
    if idx is None:
        idx = np.arange(len(ref))
    g = {k: v[idx] for k, v in gpu.items()}
    ok = ref["amb"] == 0
    n_amb = int((~ok).sum())
    assert n_amb <= max(1, max_amb_frac * len(ref)), f"ambiguous {n_amb} of {len(ref)}"
    for k in ("hit", "x", "y", "z", "lod", "mat", "normal"):
        bad = np.nonzero((g[k] != ref[k]) & ok)[0]
        assert len(bad) == 0, (k, len(bad), [(int(idx[i]), int(g[k][i]), int(ref[k][i])) for i in bad[:8]])
    h = ok & (ref["hit"] == 1)
    rel = np.abs(g["dist"][h] - ref["dist"][h]) / np.maximum(ref["dist"][h], 1e-30)
    assert (rel <= DIST_RTOL).all(), float(rel.max())
    miss = ok & (ref["hit"] == 0)
    assert np.isinf(g["dist"][miss]).all()
    assert int(ok.sum()) >= min_pixels_checked
    return int(ok.sum()), n_amb


def stratified(W, H, n, seed):
    """Row-major pixel indices: one seeded pixel in each cell of a grid of at
    least n cells over the W x H image."""
    s = max(1, int((W * H / n) ** 0.5))
    while ((W + s - 1) // s) * ((H + s - 1) // s) < n and s > 1:
        s -= 1
    rng = np.random.default_rng(seed)
    ys, xs = np.mgrid[0:H:s, 0:W:s]
    xs = np.minimum(xs + rng.integers(0, s, xs.shape), W - 1)
    ys = np.minimum(ys + rng.integers(0, s, ys.shape), H - 1)
    return np.unique((ys * W + xs).ravel())
