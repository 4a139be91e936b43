"""Chunk residency for large worlds (the streaming side of Sec. 3.4).

Streamer (synchronous): for each camera, aok_plan_residency gives the LOD
Eq. 1 selects for every chunk region within the view distance (bit-identical
to the GPU selection); regions whose resident LOD differs are evicted, missing
(chunk, LOD) pairs are built by the native builder (only the needed LOD of
each region) and uploaded before the frame renders.

AsyncStreamer: the native background loader of aok_stream_* -- worker threads
build and upload in the paper's load order (coarser LODs first, then nearest)
while frames render; changes are installed between frames.  The builder's C
functions are handed to it directly as the chunk source.

Every step runs in the native libraries; this module only moves lists.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import time
import weakref

import numpy as np

from . import BuiltWorld, Scene, _stream_handle, blib, check, lib, to_camera

# streamers still open: their worker threads are joined before the interpreter
# (and the CUDA runtime) shuts down
_open_streamers: "weakref.WeakSet[AsyncStreamer]" = weakref.WeakSet()


@atexit.register
def _close_open_streamers():
    for st in list(_open_streamers):
        try:
            st.close()
        except Exception:
            pass


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


STREAM_STATS = ("resident", "resident_bytes", "max_resident", "max_resident_bytes", "queued", "running",
                "loaded_not_installed", "installed_total", "evicted_total", "cancelled_total", "failed_total",
                "deferred_total", "missing", "planned", "ahead_installed_total")


class AsyncStreamer:
    """Background residency for `scene` (aok_stream_*), loading from the
    native builder over `world`, or from a chunk-blob file (`blobs`, an open
    BlobFile) -- the paper's disk-resident chunks.  build_cache_mb > 0 gives
    the native builder a host-memory blob cache of that size
    (aokb_source_set_cache)."""

    def __init__(self, ctx, world, scene: Scene, threads: int | None = None, blobs=None, build_cache_mb: int = 0):
        self.ctx, self.world, self.scene = ctx, world, scene
        self._src = None
        self._blobs = blobs
        if blobs is not None:
            build = ctypes.cast(lib().aok_blobfile_source, ctypes.c_void_p)
            release = ctypes.cast(lib().aok_blobfile_release, ctypes.c_void_p)
            user = blobs.h
        else:
            spec = world.spec
            self._src = blib().aokb_source_create(world.handle, spec.chunk, spec.n_lods)
            if not self._src:
                raise ValueError("bad chunking for the builder")
            blib().aokb_source_set_cache(self._src, int(build_cache_mb) << 20)
            build = ctypes.cast(blib().aokb_source_build, ctypes.c_void_p)
            release = ctypes.cast(blib().aokb_source_release, ctypes.c_void_p)
            user = self._src
        h = ctypes.c_void_p()
        check(lib().aok_stream_create(ctx.h, scene.id, build, release, user, int(threads or os.cpu_count() or 1),
                                      ctypes.byref(h)), "aok_stream_create")
        self.h = h
        _open_streamers.add(self)
        gx, gy, gz = scene.grid
        self.n = gx * gy * gz

    def update(self, cam, tau: float, stream=None):
        c = to_camera(cam)
        return check(lib().aok_stream_update(self.h, ctypes.byref(c), float(tau), _stream_handle(stream)),
                     "aok_stream_update")

    def set_prefetch(self, frames: int, samples: int = 2):
        """Load the plans of the camera extrapolated `frames` updates ahead
        (aok_stream_set_prefetch); 0 turns it off."""
        return check(lib().aok_stream_set_prefetch(self.h, int(frames), int(samples)), "aok_stream_set_prefetch")

    def wait(self, timeout_ms: int = -1) -> int:
        return int(lib().aok_stream_wait(self.h, int(timeout_ms)))

    def stats(self) -> dict:
        a = (ctypes.c_uint64 * len(STREAM_STATS))()
        check(lib().aok_stream_stats(self.h, a), "aok_stream_stats")
        return dict(zip(STREAM_STATS, (int(v) for v in a)))

    def source_stats(self) -> dict:
        """The native builder's blob cache: hits, builds, cached bytes and blobs."""
        if not self._src:
            return {}
        a = (ctypes.c_uint64 * 4)()
        blib().aokb_source_stats(self._src, ctypes.byref(a))
        return dict(zip(("cache_hits", "builds", "cached_bytes", "cached_blobs"), (int(v) for v in a)))

    def resident(self) -> np.ndarray:
        out = np.zeros(self.n, np.uint8)
        check(lib().aok_stream_resident(self.h, out.ctypes.data), "aok_stream_resident")
        return out

    def close(self):
        if self.h:
            lib().aok_stream_destroy(self.h)
            self.h = None
        if self._src:
            blib().aokb_source_destroy(self._src)
            self._src = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
