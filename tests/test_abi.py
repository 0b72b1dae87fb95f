"""CPU-side checks of the C-ABI boundary: the library builds for sm_103a,
loads, and exports every entry point include/hpmc_dep.h declares; argument
validation that needs no GPU; and the oracle/product independence rules."""
import ctypes
import os
import re
import subprocess

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
