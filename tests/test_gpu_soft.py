"""GPU parity of the soft (Hertz) colloid-depletant interaction (FP64 form)
against the oracle, through the C ABI: positions and every trajectory counter
identical (the blocking probability is evaluated in the specification's
operation order, with the written-out e^-y, on both sides)."""
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


def _compare(oracle, lib, s, sweeps, eps, *, d_max=0.05, warps=1, v0=0, seed=1):
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=d_max, seed=seed, warps=warps,
                      precision=0, v0=v0, soft_eps=eps)
    smp.sweep(sweeps)
    pos, _, sweep, cnt = smp.state()
    smp.close()
    ref, _, rc, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=d_max, seed=seed,
                               n_sweeps=sweeps, v0_mode=v0, soft_eps=eps)
    for k in oracle.PARITY_COUNTERS:
        assert cnt[k] == rc[k], (k, cnt[k], rc[k])
    assert np.array_equal(pos, ref)
    return cnt


@pytest.mark.parametrize("eps", [2.0, 30.0, 300.0])
def test_soft_spheres_256(oracle, lib, eps):
    cnt = _compare(oracle, lib, W.spheres_256(seed=3), 30, eps, d_max=0.08)
    assert cnt["accept"] > 0 and cnt["reject_depletant"] > 0


@pytest.mark.parametrize("warps", [2, 8])
def test_soft_launch_shapes(oracle, lib, warps):
    _compare(oracle, lib, W.spheres_256(seed=4), 8, 20.0, d_max=0.08, warps=warps)


def test_soft_with_the_cube(oracle, lib):
    _compare(oracle, lib, W.spheres_256(seed=5), 10, 20.0, d_max=0.08, v0=2)


def test_soft_spheres_16384_first_sweeps(oracle, lib):
    _compare(oracle, lib, W.spheres_16384(0.2), 2, 10.0)


def test_soft_argument_errors(lib):
    s = W.spheres_256()
    for kw in (dict(precision=1), dict(n_trial=2), dict(v0=1)):
        smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, soft_eps=5.0, **kw)
        with pytest.raises(lib.HPMCError):
            smp.sweep(1)
        smp.close()
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r)
    with pytest.raises(lib.HPMCError):
        lib.hpmc_set_soft(smp.ctx, -1.0)
    smp.close()
