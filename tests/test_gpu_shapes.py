"""GPU parity of the anisotropic shapes (hemispheres, discoids; Sec. V) with
translation and rotation moves, against the oracle, through the C ABI.

Positions, orientations and every trajectory counter must be bit-identical:
both sides implement the same written specification (quaternion algebra,
point-to-body tests, portal refinement for pairs) with correctly rounded FP64
and no contraction.  Small systems run many sweeps, the full-size systems
(32768 hemispheres, 65536 discoids) their first sweeps."""
import numpy as np
import pytest

from paper_1508_07077_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(W.HEMISPHERE, 0.25, 0.10, 0.30), (W.SPHEROID, 0.30, 0.10, 0.25)]


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07077_gb300 import build, hpmc
    build.build()
    hpmc.load()
    return hpmc


PRECISIONS = [0, 1]   # HPMC_FP64, HPMC_FP32_RECHECK


def _compare(oracle, lib, s, sweeps, *, n_trial=0, d_max=0.08, a_max=0.2, p_translate=0.5,
             warps=1, seed=1, precision=0, n_cell=0, sweep0=0, margin=0.0):
    smp = lib.Sampler(s.pos, s.L, quat=s.quat, shape=s.shape, shape_params=s.shape_params,
                      q=s.q, n_r=s.n_r, n_trial=n_trial, d_max=d_max, a_max=a_max,
                      p_translate=p_translate, seed=seed, warps=warps, precision=precision,
                      n_cell=n_cell)
    if margin:
        lib.hpmc_set_fp32_margin(smp.ctx, margin)
    if sweep0:
        lib.hpmc_set_state(smp.ctx, s.pos, s.quat, sweep0)
    smp.sweep(sweeps)
    pos, quat, sweep, cnt = smp.state(with_quat=True)
    smp.close()
    ref, refq, rc, _ = oracle.run(s.pos, s.L, shape=s.shape, shape_params=s.shape_params,
                                  quat=s.quat, q=s.q, n_r=s.n_r, n_trial=n_trial,
                                  d_max=d_max, a_max=a_max, p_translate=p_translate,
                                  seed=seed, n_cell=n_cell, n_sweeps=sweeps, sweep0=sweep0)
    assert sweep == sweep0 + sweeps
    for k in oracle.PARITY_COUNTERS:
        assert cnt[k] == rc[k], (k, cnt[k], rc[k])
    assert np.array_equal(pos, ref)
    assert np.array_equal(quat, refq)
    return cnt


def _small(shape, phi, q, eta, n=256, seed=1):
    return W.make_system("small", shape, n, phi, q, eta, seed=seed)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape,phi,q,eta", SHAPES)
def test_small_system_many_sweeps(oracle, lib, shape, phi, q, eta, precision):
    cnt = _compare(oracle, lib, _small(shape, phi, q, eta), 30, precision=precision)
    assert cnt["accept"] > 0 and cnt["reject_overlap"] > 0 and cnt["reject_depletant"] > 0
    assert 0 < cnt["translate"] < cnt["moves"]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape,phi,q,eta", SHAPES)
@pytest.mark.parametrize("n_trial", [1, 3])
def test_configurational_bias(oracle, lib, shape, phi, q, eta, n_trial, precision):
    cnt = _compare(oracle, lib, _small(shape, phi, q, eta, seed=2), 8, n_trial=n_trial,
                   precision=precision)
    assert cnt["reject_cb"] > 0


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape,phi,q,eta", SHAPES)
def test_many_reinsertion_trials(oracle, lib, shape, phi, q, eta, precision):
    """n_trial = 24: each CB factor's trial streams span several warp passes."""
    _compare(oracle, lib, _small(shape, phi, q, eta, seed=4), 4, n_trial=24, precision=precision)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape,phi,q,eta", SHAPES)
@pytest.mark.parametrize("warps", [2, 8])
def test_launch_shapes(oracle, lib, shape, phi, q, eta, warps, precision):
    s = _small(shape, phi, q, eta, seed=3)
    _compare(oracle, lib, s, 5, warps=warps, precision=precision)
    _compare(oracle, lib, s, 3, warps=warps, n_trial=2, precision=precision)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape,phi,q,eta", SHAPES)
def test_move_mixes(oracle, lib, shape, phi, q, eta, precision):
    s = _small(shape, phi, q, eta, n=108, seed=4)
    kw = dict(precision=precision)
    _compare(oracle, lib, s, 6, p_translate=0.0, **kw)                  # rotations only
    _compare(oracle, lib, s, 6, a_max=0.0, **kw)                        # translations only
    _compare(oracle, lib, s, 6, a_max=1.5, p_translate=0.3, sweep0=777, **kw)
    # two cells per side: the deduplicated stencil
    _compare(oracle, lib, _small(shape, phi, q, eta, n=32, seed=4), 6, n_cell=2, **kw)


@pytest.mark.parametrize("shape,phi,q,eta", SHAPES)
@pytest.mark.parametrize("n_trial", [0, 2])
def test_fp32_exact_paths(oracle, lib, shape, phi, q, eta, n_trial):
    """A margin of 1 sends every FP32 depletant test and every pair
    certificate to the exact FP64 re-take: the trajectory must not change,
    and the recheck counter shows the exact paths ran."""
    s = _small(shape, phi, q, eta, n=108, seed=5)
    cnt = _compare(oracle, lib, s, 3, n_trial=n_trial, precision=1, margin=1.0)
    assert cnt["rechecks"] > cnt["moves"]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_full_size_hemispheres(oracle, lib, precision):
    _compare(oracle, lib, W.hemispheres_32768(), 2, d_max=0.05, precision=precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_full_size_discoids(oracle, lib, precision):
    _compare(oracle, lib, W.discoids_65536(), 1, d_max=0.05, precision=precision)


def test_overlapping_start_is_rejected(lib):
    s = _small(W.HEMISPHERE, 0.25, 0.1, 0.3, n=108)
    pos = s.pos.copy()
    quat = s.quat.copy()
    pos[1] = pos[0] + np.array([0.0, 0.0, 0.3])
    pos[1] %= s.L
    quat[0] = quat[1] = [1.0, 0.0, 0.0, 0.0]
    smp = lib.Sampler(pos, s.L, quat=quat, shape=s.shape, shape_params=s.shape_params,
                      q=s.q, n_r=s.n_r)
    with pytest.raises(lib.HPMCError):
        smp.sweep(1)
    smp.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_autotuner_keeps_the_trajectory(oracle, lib, precision):
    """Tuning times candidate launch shapes and cell counts on the live system
    and restores it: the trajectory continues as if nothing ran, with the
    chosen cell count from then on.  A cell count whose bins would overflow
    (two cells per side here) is skipped."""
    s = _small(W.HEMISPHERE, 0.25, 0.1, 0.3, n=256, seed=6)
    kw = dict(q=s.q, n_r=s.n_r, d_max=0.08, a_max=0.2, p_translate=0.5)
    smp = lib.Sampler(s.pos, s.L, quat=s.quat, shape=s.shape, shape_params=s.shape_params,
                      seed=1, precision=precision, **kw)
    smp.sweep(2)
    warps, ncell, ms = lib.hpmc_autotune(smp.ctx, warps=(1, 2), cells=(0, 2), n_sweeps=2)
    assert warps in (1, 2) and ncell == 0 and ms > 0
    smp.sweep(3)
    pos, quat, sweep, cnt = smp.state(with_quat=True)
    smp.close()
    p1, q1, c1, _ = oracle.run(s.pos, s.L, shape=s.shape, shape_params=s.shape_params,
                               quat=s.quat, seed=1, n_sweeps=2, **kw)
    p2, q2, c2, _ = oracle.run(p1, s.L, shape=s.shape, shape_params=s.shape_params, quat=q1,
                               seed=1, n_sweeps=3, sweep0=2, n_cell=ncell, **kw)
    assert sweep == 5
    assert np.array_equal(pos, p2) and np.array_equal(quat, q2)
    for k in oracle.PARITY_COUNTERS:
        assert cnt[k] == c1[k] + c2[k], k
