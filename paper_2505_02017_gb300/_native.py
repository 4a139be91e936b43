"""Builds and loads the native libraries of the package (in-tree, sm_103a).

libaok.so      : the C ABI of include/aok.h (host runtime + CUDA kernels).
libaokbuild.so : offline chunk preparation (LOD aggregation + SVDAG build)
                 over scenegen worlds.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_BUILD = os.path.join(_PKG, "_build")
LIBAOK = os.path.join(_BUILD, "libaok.so")
LIBBUILD = os.path.join(_BUILD, "libaokbuild.so")
GENCODE = "arch=compute_103a,code=sm_103a"
_lock = threading.Lock()


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libaok")


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    subprocess.check_call(cmd)


def build(force: bool = False, verbose: bool = False) -> None:
    """Compile libaok.so (nvcc, -gencode arch=compute_103a,code=sm_103a) and
    libaokbuild.so (g++/gcc).  Translation units compile in parallel."""
    hdrs = [os.path.join(_ROOT, "include", "aok.h"), os.path.join(_CSRC, "aok_internal.h"),
            os.path.join(_CSRC, "aok_runtime.h"), os.path.join(_CSRC, "aok_trace.cuh"),
            os.path.join(_CSRC, "aok_select.cuh")]
    srcs_cu = [os.path.join(_CSRC, f) for f in ("aok_kernels.cu", "aok_tiles.cu", "aok_beam.cu")]
    srcs_cpp = [os.path.join(_CSRC, f) for f in ("aok_runtime.cpp", "aok_serve.cpp", "aok_stream.cpp", "aok_file.cpp")]
    bsrc = os.path.join(_CSRC, "aok_build.cpp")
    sg = os.path.join(_ROOT, "scenegen", "scenegen.c")
    sgh = os.path.join(_ROOT, "scenegen", "scenegen.h")
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        nvcc = _nvcc()
        jobs = []
        objs = []
        for s in srcs_cu + srcs_cpp:
            o = os.path.join(_BUILD, os.path.basename(s) + ".o")
            objs.append(o)
            if force or _newer(o, [s] + hdrs):
                # host code: no floating-point contraction (Eq. 1 must round exactly as on the GPU)
                flags = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-lineinfo",
                         "-I", os.path.join(_ROOT, "include")]
                if s.endswith(".cu"):
                    flags += ["-gencode", GENCODE, "--fmad=false", "-Xptxas", "-v"] if verbose else \
                             ["-gencode", GENCODE, "--fmad=false"]
                jobs.append([nvcc, *flags, "-c", s, "-o", o])
        bo = os.path.join(_BUILD, "aok_build.o")
        so = os.path.join(_BUILD, "scenegen.o")
        if force or _newer(bo, [bsrc, sgh, hdrs[0]]):
            jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-c", bsrc, "-o", bo])
        if force or _newer(so, [sg, sgh]):
            jobs.append(["gcc", "-O2", "-std=c11", "-fPIC", "-c", sg, "-o", so])
        if jobs:
            with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
                list(ex.map(_run, jobs))
        if force or _newer(LIBAOK, objs):
            tmp = LIBAOK + f".tmp{os.getpid()}"
            _run([nvcc, "-shared", "-gencode", GENCODE, *objs, "-o", tmp])
            os.replace(tmp, LIBAOK)
        if force or _newer(LIBBUILD, [bo, so]):
            tmp = LIBBUILD + f".tmp{os.getpid()}"
            _run(["g++", "-shared", "-pthread", bo, so, "-o", tmp])
            os.replace(tmp, LIBBUILD)
