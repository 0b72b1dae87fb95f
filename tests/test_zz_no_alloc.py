"""The allocation-free cell list (hpmc_cell_list_noalloc) against the regular
one (hpmc_cell_list), through the C ABI.

It exists for callers that cannot allocate device memory when they need a
cell list (a fixed memory budget after start-up, an allocator owned by another
component); its scratch is a static device array shared by every call.  Cell
lists are integer data, so the two entry points must agree exactly, on two
calls in a row (the second call must not see the first one's leftovers).
This file is collected last on purpose."""
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


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    s = W.spheres_256()
    pos = torch.tensor(s.pos, device="cuda")
    start = torch.empty(42 ** 3 + 1, dtype=torch.int32, device="cuda")
    idx = torch.empty(s.n, dtype=torch.int32, device="cuda")
    with pytest.raises(lib.HPMCError) as e:
        lib.hpmc_cell_list_noalloc(s.n, 100.0, 42, pos, 1, 0, 0, start, idx)
    assert e.value.code == -6
