"""In-tree build of the CUDA library for sm_103a (nvcc, no cmake).

``build()`` compiles ``csrc/hpmc_dep.cu`` into ``_lib/libhpmc_dep.so``, the
same source with bounds and invariant checks into ``_lib/libhpmc_dep_checked.so``
and ``csrc/pipe_peaks.cu`` (the ALU-pipe microbenchmarks used for the roofline
denominators) into ``_lib/libhpmc_peaks.so``, in parallel.  FP64 decision
paths must not be contracted into FMAs, hence ``-fmad=false`` (device) and
``-ffp-contract=off`` (host: the Poisson table).
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-shared",
                 "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "-I", INCLUDE,
                 "-diag-suppress", "1444"]

_HEADERS = ["hpmc_common.cuh", "hpmc_cells.cuh", "hpmc_misc.cuh", "hpmc_sphere_fp64.cuh",
            "hpmc_sphere_fp32.cuh", "hpmc_shapes.cuh", "hpmc_aniso_fp64.cuh",
            "hpmc_shapes32.cuh", "hpmc_aniso_fp32.cuh", "hpmc_probe.cuh", "hpmc_gibbs.cuh"]
# name: (sources, headers, extra flags).  The checked build bounds-checks the
# FP32 sphere path's indices and the checkerboard invariant (HPMC_CHECKED).
TARGETS = {
    "libhpmc_dep.so": (["hpmc_dep.cu"], _HEADERS, []),
    "libhpmc_dep_checked.so": (["hpmc_dep.cu"], _HEADERS, ["-DHPMC_CHECKED"]),
    "libhpmc_peaks.so": (["pipe_peaks.cu"], [], []),
}


def _stale(out: str, srcs: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = srcs + [os.path.join(INCLUDE, "hpmc_dep.h"), __file__]
    return any(os.path.exists(d) and os.path.getmtime(d) > t for d in deps)


def _nvcc(name: str, force: bool) -> str:
    srcs, hdrs, extra = TARGETS[name]
    src_paths = [os.path.join(CSRC, s) for s in srcs]
    out = os.path.join(LIBDIR, name)
    if not force and not _stale(out, src_paths + [os.path.join(CSRC, h) for h in hdrs]):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["nvcc"] + COMMON + extra + ["-o", tmp] + src_paths
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (name, " ".join(cmd), r.stderr))
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> list[str]:
    os.makedirs(LIBDIR, exist_ok=True)
    names = [n for n in TARGETS if all(os.path.exists(os.path.join(CSRC, s))
                                       for s in TARGETS[n][0])]
    with ThreadPoolExecutor(max_workers=len(names)) as ex:
        return list(ex.map(lambda n: _nvcc(n, force), names))


if __name__ == "__main__":
    for p in build(force=True):
        print(p)
