"""Chunk residency for large worlds (the streaming side of Sec. 3.4).

For each camera, aok_plan_residency gives the LOD Eq. 1 selects for every
chunk region within the view distance (bit-identical to the GPU selection);
regions whose resident LOD differs are evicted, missing (chunk, LOD) pairs are
built by the native builder (only the needed LOD of each region) and uploaded.
Every step runs in the native libraries; this module only moves lists.
"""
from __future__ import annotations

import ctypes
import os
import time

import numpy as np

from . import BuiltWorld, Scene, check, lib, to_camera


class Streamer:
    """Keeps exactly the (chunk, LOD) pairs a camera needs resident in `scene`."""

    def __init__(self, ctx, world, scene: Scene, threads: int | None = None):
        self.ctx, self.world, self.scene = ctx, world, scene
        self.threads = threads or os.cpu_count() or 1
        gx, gy, gz = scene.grid
        self.n = gx * gy * gz
        self.resident = np.full(self.n, 0xFF, np.uint8)  # resident LOD per region (0xFF = none)
        self.bytes = np.zeros(self.n, np.int64)  # blob bytes per resident region
        self.max_resident = 0
        self.max_bytes = 0

    def plan(self, cam, tau: float) -> np.ndarray:
        out = np.empty(self.n, np.uint8)
        kept = ctypes.c_uint32()
        c = to_camera(cam)
        check(lib().aok_plan_residency(self.ctx.h, self.scene.id, ctypes.byref(c), float(tau), out.ctypes.data,
                                       ctypes.byref(kept)), "aok_plan_residency")
        return out

    def update(self, cam, tau: float) -> dict:
        """Make the camera's plan resident; returns counts and host times."""
        t0 = time.perf_counter()
        want = self.plan(cam, tau)
        gx, gy, _ = self.scene.grid
        stale = np.nonzero((self.resident != 0xFF) & (self.resident != want))[0]
        for c in stale:
            self.scene.evict(int(c % gx), int((c // gx) % gy), int(c // (gx * gy)), int(self.resident[c]))
            self.resident[c] = 0xFF
            self.bytes[c] = 0
        missing = np.nonzero((want != 0xFF) & (self.resident != want))[0]
        t1 = time.perf_counter()
        built = None
        if len(missing):
            built = BuiltWorld(self.world, self.threads, chunks=missing.astype(np.int64),
                               lod_masks=(1 << want[missing].astype(np.uint32)))
        t2 = time.perf_counter()
        for i in range(len(missing)):
            c = int(missing[i])
            lod = int(want[c])
            cc, blob = built.blob(i, lod)
            self.scene.upload(c % gx, (c // gx) % gy, c // (gx * gy), lod, blob)
            self.resident[c] = lod
            self.bytes[c] = 4 * blob.n_node_words + 8 * blob.n_leaves + blob.n_mats
        if built is not None:
            built.close()
        t3 = time.perf_counter()
        nres = int((self.resident != 0xFF).sum())
        nbytes = int(self.bytes.sum())
        self.max_resident = max(self.max_resident, nres)
        self.max_bytes = max(self.max_bytes, nbytes)
        return {"evicted": int(len(stale)), "built": int(len(missing)), "resident": nres, "resident_bytes": nbytes,
                "plan_s": t1 - t0, "build_s": t2 - t1, "upload_s": t3 - t2}
