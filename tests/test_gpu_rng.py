"""The device Philox4x32-10 against the published known-answer vectors and
against the oracle's generator, through the C ABI (hpmc_philox).

Every random stream of the method (schedule, moves, Poisson counts, depletant
points, CB trials, acceptance) is a Philox4x32-10 draw, so a device generator
that matches the known answers and agrees with the oracle's on random
counters and keys pins both independent implementations to the published
function, in both of the device's forms (key bumped per round, and the ten
round keys precomputed)."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07077_gb300 import build, hpmc
    build.build()
    hpmc.load()
    return hpmc


def _device_words(lib, ctr, key, variant):
    c = torch.tensor(np.asarray(ctr, dtype=np.uint32).view(np.int32), device="cuda")
    k = torch.tensor(np.asarray(key, dtype=np.uint32).view(np.int32), device="cuda")
    out = torch.zeros_like(c)
    lib.hpmc_philox(c, k, out, variant)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("variant", [0, 1])
def test_device_philox_known_answers(lib, variant):
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.json")) as f:
        vecs = json.load(f)["vectors"]
    ctr = [[int(x, 16) for x in v["ctr"]] for v in vecs]
    key = [[int(x, 16) for x in v["key"]] for v in vecs]
    want = np.array([[int(x, 16) for x in v["out"]] for v in vecs], dtype=np.uint32)
    got = _device_words(lib, ctr, key, variant)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("variant", [0, 1])
def test_device_philox_equals_oracle_on_random_counters(lib, oracle, variant):
    rng = np.random.default_rng(11)
    n = 1000   # several CTAs of the hook kernel and a ragged tail
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    got = _device_words(lib, ctr, key, variant)
    want = np.array([oracle.philox(ctr[i], key[i]) for i in range(n)], dtype=np.uint32)
    assert np.array_equal(got, want)


def test_empty_and_invalid(lib):
    z = torch.zeros((0, 4), dtype=torch.int32, device="cuda")
    lib.hpmc_philox(z, torch.zeros((0, 2), dtype=torch.int32, device="cuda"), z)
    c = torch.zeros((2, 4), dtype=torch.int32, device="cuda")
    k = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(lib.HPMCError):
        lib.hpmc_philox(c, k, torch.zeros_like(c), variant=2)


def test_library_kernels_are_sm103(lib):
    """The runtime reports the kernels' binary as compiled for compute
    capability 10.3 (sm_103a) from the 10.3 virtual architecture."""
    binary, ptx = lib.hpmc_kernel_arch()
    assert binary == 103
    assert ptx in (0, 103)
