"""The allocation-free cell list (hpmc_cell_list_noalloc) against the regular
one (hpmc_cell_list), through the C ABI.

It exists for callers that cannot allocate device memory when they need a
cell list (a fixed memory budget after start-up, an allocator owned by another
component); its scratch is a static device array shared by every call.  Cell
lists are integer data, so the two entry points must agree exactly, on two
calls in a row (the second call must not see the first one's leftovers).
The property the entry point exists for is checked too: the device's
stream-ordered memory pool sees no allocation during its calls, while the
allocating entry point raises the pool's high-water mark (the control).
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1508_07077_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07077_gb300 import build, hpmc
    build.build()
    hpmc.load()
    return hpmc


def _lists(lib, fn, s, nc, sweep):
    pos = torch.tensor(s.pos, device="cuda")
    start = torch.full((nc ** 3 + 1,), -7, dtype=torch.int32, device="cuda")
    idx = torch.full((s.n,), -7, dtype=torch.int32, device="cuda")
    fn(s.n, s.L, nc, pos, 1, 0, sweep, start, idx)
    torch.cuda.synchronize()
    return start.cpu().numpy(), idx.cpu().numpy()


def test_noalloc_matches_allocating_cell_list_twice(lib):
    big = W.spheres_16384(0.2)
    small = W.spheres_256()
    cases = [(big, 26, 11), (small, 6, 3)]   # large first, so leftovers would show
    for s, nc, sweep in cases:
        ref = _lists(lib, lib.hpmc_cell_list, s, nc, sweep)
        got = _lists(lib, lib.hpmc_cell_list_noalloc, s, nc, sweep)
        assert np.array_equal(ref[0], got[0])
        assert np.array_equal(ref[1], got[1])
        assert got[0][-1] == s.n


class _Pool:
    """The current memory pool of device 0 through the driver API: its bytes
    in use and their high-water mark (which can be reset to the current use)."""
    USED_CURRENT, USED_HIGH = 7, 8   # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_HIGH, ctypes.byref(z)) == 0


def test_noalloc_takes_nothing_from_the_memory_pool(lib):
    s = W.spheres_16384(0.3)
    pos = torch.tensor(s.pos, device="cuda")
    start = torch.empty(26 ** 3 + 1, dtype=torch.int32, device="cuda")
    idx = torch.empty(s.n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    pool = _Pool()
    # warm-up call: the one-time symbol lookup happens here
    lib.hpmc_cell_list_noalloc(s.n, s.L, 26, pos, 1, 0, 4, start, idx)
    torch.cuda.synchronize()
    base = pool.get(pool.USED_CURRENT)
    pool.reset_high()
    for sweep in (5, 6):
        lib.hpmc_cell_list_noalloc(s.n, s.L, 26, pos, 1, 0, sweep, start, idx)
    torch.cuda.synchronize()
    assert pool.get(pool.USED_HIGH) == base
    assert pool.get(pool.USED_CURRENT) == base
    # control: the allocating entry point's scratch does show in the pool
    pool.reset_high()
    lib.hpmc_cell_list(s.n, s.L, 26, pos, 1, 0, 7, start, idx)
    torch.cuda.synchronize()
    assert pool.get(pool.USED_HIGH) > base


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    s = W.spheres_256()
    pos = torch.tensor(s.pos, device="cuda")
    start = torch.empty(42 ** 3 + 1, dtype=torch.int32, device="cuda")
    idx = torch.empty(s.n, dtype=torch.int32, device="cuda")
    with pytest.raises(lib.HPMCError) as e:
        lib.hpmc_cell_list_noalloc(s.n, 100.0, 42, pos, 1, 0, 0, start, idx)
    assert e.value.code == -6
    # beyond what the allocating entry point accepts: an invalid argument on
    # both, as the header states
    for fn in (lib.hpmc_cell_list, lib.hpmc_cell_list_noalloc):
        with pytest.raises(lib.HPMCError) as e:
            fn(s.n, 100.0, 1026, pos, 1, 0, 0, start, idx)
        assert e.value.code == -1
