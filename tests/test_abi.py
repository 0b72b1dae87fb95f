"""CPU-side checks of the C-ABI boundary: the library builds for sm_103a,
loads, and exports every entry point include/hpmc_dep.h declares; argument
validation that needs no GPU; and the oracle/product independence rules."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hpmc_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def built():
    from paper_1508_07077_gb300 import build
    return build.build()


@pytest.mark.parametrize("which", ["LIB_PATH", "CHECKED_LIB_PATH"])
def test_library_exports_every_declared_entry_point(built, which):
    from paper_1508_07077_gb300 import hpmc
    path = getattr(hpmc, which)
    lib = ctypes.CDLL(path)
    declared = _declared("hpmc_dep.h")
    assert "hpmc_sweep" in declared and "hpmc_cell_list" in declared
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(hpmc_[a-z0-9_]+)\b", out))
    assert set(declared) <= exported
    assert set(hpmc.EXPORTS) == set(declared)




def test_host_side_validation_without_gpu(built):
    from paper_1508_07077_gb300 import hpmc
    lib = hpmc.load()
    assert hpmc.strerror(0) == "ok"
    assert "overlap" in hpmc.strerror(-2)
    ctx = ctypes.c_void_p()
    # n = 0 and a NULL pointer are rejected before any CUDA call
    assert lib.hpmc_init(ctypes.byref(ctx), 0, 5.0, None, None, 0, 1, 0, 0, 0) == -1
    assert lib.hpmc_init(None, 4, 5.0, None, None, 0, 1, 0, 0, 0) == -1
    assert lib.hpmc_set_depletant(None, 0.1, 1.0, 0) == -1
    assert lib.hpmc_set_v0(None, 1) == -1
    assert lib.hpmc_cell_list(4, 5.0, 3, None, 1, 0, 0, None, None, None) == -1


def test_every_entry_point_rejects_bad_arguments_before_the_device(built):
    """Every entry point that takes a context rejects a null one, and the
    context-free ones their invalid arguments, with HPMC_ERR_ARG (or
    HPMC_ERR_CAP for the allocation-free cell list's limits) before any CUDA
    call: this runs without a GPU.  The binding refuses buffers it cannot
    pass (not contiguous float64, not an array) before calling the library."""
    from paper_1508_07077_gb300 import hpmc
    lib = hpmc.load()
    ARG, CAP = -1, -6           # HPMC_ERR_ARG, HPMC_ERR_CAP (include/hpmc_dep.h)
    i = ctypes.c_int()
    u = ctypes.c_uint64()
    d = ctypes.c_double()
    cnt = hpmc.hpmc_counters()
    one = (ctypes.c_int * 1)(1)
    calls = {
        "hpmc_set_shape": lambda: lib.hpmc_set_shape(None, 0, (ctypes.c_double * 1)(1.0), 1),
        "hpmc_set_depletant": lambda: lib.hpmc_set_depletant(None, 0.1, 1.0, 0),
        "hpmc_set_moves": lambda: lib.hpmc_set_moves(None, 0.1, 0.0, 1.0),
        "hpmc_set_replica_moves": lambda: lib.hpmc_set_replica_moves(None, 0, 0.1, 0.0, 1.0),
        "hpmc_set_cells": lambda: lib.hpmc_set_cells(None, 4),
        "hpmc_set_launch": lambda: lib.hpmc_set_launch(None, 1, 0),
        "hpmc_set_phase_waves": lambda: lib.hpmc_set_phase_waves(None, -1),
        "hpmc_set_wait_limit": lambda: lib.hpmc_set_wait_limit(None, 1.0),
        "hpmc_debug_withhold_cell": lambda: lib.hpmc_debug_withhold_cell(None, -1),
        "hpmc_autotune": lambda: lib.hpmc_autotune(None, one, 1, one, 1, 1, None, None, None),
        "hpmc_sweep": lambda: lib.hpmc_sweep(None, 1, None),
        "hpmc_set_fp32_margin": lambda: lib.hpmc_set_fp32_margin(None, 0.0),
        "hpmc_set_v0": lambda: lib.hpmc_set_v0(None, 0),
        "hpmc_set_soft": lambda: lib.hpmc_set_soft(None, 0.0),
        "hpmc_set_timing": lambda: lib.hpmc_set_timing(None, 1),
        "hpmc_get_timing": lambda: lib.hpmc_get_timing(None, ctypes.byref(d), ctypes.byref(u), 1),
        "hpmc_get_state": lambda: lib.hpmc_get_state(None, None, None, hpmc.HPMC_HOST,
                                                     ctypes.byref(u), ctypes.byref(cnt), None),
        "hpmc_get_replica": lambda: lib.hpmc_get_replica(None, 0, None, None, ctypes.byref(cnt)),
        "hpmc_set_state": lambda: lib.hpmc_set_state(None, None, None, hpmc.HPMC_HOST, 0, None),
        "hpmc_get_size": lambda: lib.hpmc_get_size(None, ctypes.byref(i), ctypes.byref(i)),
        "hpmc_reset_counters": lambda: lib.hpmc_reset_counters(None),
        "hpmc_sync": lambda: lib.hpmc_sync(None),
        "hpmc_set_live": lambda: lib.hpmc_set_live(None, 0, 1),
        "hpmc_get_live": lambda: lib.hpmc_get_live(None, ctypes.byref(i)),
        "hpmc_gibbs_exchange": lambda: lib.hpmc_gibbs_exchange(None, 1, None),
        "hpmc_get_gibbs": lambda: lib.hpmc_get_gibbs(None, 0, ctypes.byref(u), ctypes.byref(u)),
        "hpmc_free_volume": lambda: lib.hpmc_free_volume(None, 0, 0.1, 1, 0, 10, ctypes.byref(u)),
        # context-free entry points: invalid arguments
        "hpmc_init_batch": lambda: lib.hpmc_init_batch(None, 1, None, 0, None, 0, 1, 1, 0),
        "hpmc_philox": lambda: lib.hpmc_philox(4, None, None, None, 2, None),
        "hpmc_kernel_arch": lambda: lib.hpmc_kernel_arch(None, None),
        "hpmc_cell_list_noalloc": lambda: lib.hpmc_cell_list_noalloc(4, 5.0, 3, None, 1, 0, 0,
                                                                     None, None, None),
    }
    for name, call in calls.items():
        assert call() == ARG, name
    # every exported entry point that takes a context or validates arguments is covered
    covered = set(calls) | {"hpmc_init", "hpmc_cell_list", "hpmc_strerror", "hpmc_destroy"}
    assert set(hpmc.EXPORTS) <= covered, sorted(set(hpmc.EXPORTS) - covered)
    lib.hpmc_destroy(None)                       # a null context is a no-op
    assert lib.hpmc_philox(0, None, None, None, 0, None) == hpmc.HPMC_OK   # nothing to draw
    # the allocation-free list's own limits (never dereferences its buffers)
    fake = ctypes.c_void_p(4096)
    assert lib.hpmc_cell_list_noalloc(4, 50.0, 42, fake, 1, 0, 0, fake, fake, None) == CAP
    assert lib.hpmc_cell_list_noalloc(4, 50.0, 1026, fake, 1, 0, 0, fake, fake, None) == ARG
    # the binding's own checks, before any library call
    with pytest.raises(ValueError):
        hpmc.hpmc_init(4, 5.0, np.zeros((4, 3), dtype=np.float32))
    with pytest.raises(ValueError):
        hpmc.hpmc_init(4, 5.0, np.zeros((3, 4))[:, :3])     # not contiguous
    with pytest.raises(TypeError):
        hpmc.hpmc_init(4, 5.0, [[0.0, 0.0, 0.0]] * 4)


def test_oracle_and_product_are_independent():
    pkg = os.path.join(ROOT, "paper_1508_07077_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt).lower() or f == "workloads.py", f
    src = open(os.path.join(ROOT, "oracle", "hpmc_oracle.c")).read()
    assert "#include \"" not in src            # no project headers
    assert "hpmc_dep.h" not in src
