"""GPU parity of the soft (Hertz) colloid-depletant interaction, both forms,
against the oracle, through the C ABI: positions and every trajectory counter
identical (the blocking probability is evaluated in the specification's
operation order, with the written-out e^-y, on both sides; the FP32 form
settles only the certain early exits in FP32)."""
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


def _compare(oracle, lib, s, sweeps, eps, *, d_max=0.05, warps=1, v0=0, seed=1, precision=0,
             margin=0.0):
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=d_max, seed=seed, warps=warps,
                      precision=precision, v0=v0, soft_eps=eps)
    if margin:
        lib.hpmc_set_fp32_margin(smp.ctx, margin)
    smp.sweep(sweeps)
    pos, _, sweep, cnt = smp.state()
    smp.close()
    ref, _, rc, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=d_max, seed=seed,
                               n_sweeps=sweeps, v0_mode=v0, soft_eps=eps)
    for k in oracle.PARITY_COUNTERS:
        assert cnt[k] == rc[k], (k, cnt[k], rc[k])
    assert np.array_equal(pos, ref)
    return cnt


PRECISIONS = [0, 1]   # FP64; FP32 early exits with the FP64 statement inside the bands


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("eps", [2.0, 30.0, 300.0])
def test_soft_spheres_256(oracle, lib, eps, precision):
    cnt = _compare(oracle, lib, W.spheres_256(seed=3), 30, eps, d_max=0.08, precision=precision)
    assert cnt["accept"] > 0 and cnt["reject_depletant"] > 0


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("warps", [2, 8])
def test_soft_launch_shapes(oracle, lib, warps, precision):
    _compare(oracle, lib, W.spheres_256(seed=4), 8, 20.0, d_max=0.08, warps=warps,
             precision=precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_soft_with_the_cube(oracle, lib, precision):
    _compare(oracle, lib, W.spheres_256(seed=5), 10, 20.0, d_max=0.08, v0=2, precision=precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_soft_spheres_16384_first_sweeps(oracle, lib, precision):
    _compare(oracle, lib, W.spheres_16384(0.2), 2, 10.0, precision=precision)


@pytest.mark.parametrize("eps", [0.5, 1000.0])
def test_soft_fp32_exact_paths(oracle, lib, eps):
    """A margin of 1 sends every FP32 decision of the soft form (ball test,
    both early exits) to the FP64 statement: the trajectory must not change;
    very soft and very stiff interactions stress the energy bands."""
    s = W.spheres_256(seed=6)
    _compare(oracle, lib, s, 6, eps, d_max=0.08, precision=1, margin=1.0)
    _compare(oracle, lib, s, 12, eps, d_max=0.08, precision=1)


def test_soft_argument_errors(lib):
    s = W.spheres_256()
    for kw in (dict(n_trial=2), dict(v0=1)):
        smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, soft_eps=5.0, **kw)
        with pytest.raises(lib.HPMCError):
            smp.sweep(1)
        smp.close()
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r)
    with pytest.raises(lib.HPMCError):
        lib.hpmc_set_soft(smp.ctx, -1.0)
    smp.close()
