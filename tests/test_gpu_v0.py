"""GPU parity of the alternative depletant regions V_0 (Sec. III.C) against
the oracle, through the C ABI: the shell-restricted V_0 (spheres,
translations; the closing remark of Sec. III.C) and the cube around the
circumsphere (every shape, no rejection step).

Positions and every trajectory counter must be bit-identical to the oracle's
mode: the level rule is integer-only, the shell point is FP64 in the
specification's order, and the FP32 form certifies its shell decisions (or
re-takes them in FP64)."""
import numpy as np
import pytest

from paper_1508_07077_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHELL = 1
PRECISIONS = [0, 1]   # HPMC_FP64, HPMC_FP32_RECHECK


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07077_gb300 import build, hpmc
    build.build()
    hpmc.load()
    return hpmc


def _compare(oracle, lib, s, sweeps, *, n_trial=0, d_max=0.05, warps=1, n_cell=0, seed=1,
             precision=0, sweep0=0, margin=0.0):
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, n_trial=n_trial, d_max=d_max, seed=seed,
                      warps=warps, n_cell=n_cell, precision=precision, v0=SHELL)
    if margin:
        lib.hpmc_set_fp32_margin(smp.ctx, margin)
    if sweep0:
        lib.hpmc_set_state(smp.ctx, s.pos, None, sweep0)
    smp.sweep(sweeps)
    pos, _, sweep, cnt = smp.state()
    smp.close()
    ref, _, rc, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, n_trial=n_trial, d_max=d_max,
                               seed=seed, n_cell=n_cell, n_sweeps=sweeps, sweep0=sweep0,
                               v0_mode=SHELL)
    assert sweep == sweep0 + sweeps
    for k in oracle.PARITY_COUNTERS:
        assert cnt[k] == rc[k], (k, cnt[k], rc[k])
    assert np.array_equal(pos, ref)
    return cnt, rc


@pytest.mark.parametrize("precision", PRECISIONS)
def test_spheres_256_shell_50_sweeps(oracle, lib, precision):
    s = W.spheres_256()
    cnt, _ = _compare(oracle, lib, s, 50, d_max=0.1, precision=precision)
    assert cnt["reject_depletant"] > 0 and cnt["accept"] > 0
    # fewer depletants than the circumsphere draws for the same moves
    _, _, rc0, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.1, seed=1, n_sweeps=50)
    assert cnt["dep_drawn"] < 0.6 * rc0["dep_drawn"]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n_trial", [1, 3])
def test_shell_configurational_bias(oracle, lib, n_trial, precision):
    cnt, _ = _compare(oracle, lib, W.spheres_256(seed=2), 10, d_max=0.1, n_trial=n_trial,
                      precision=precision)
    assert cnt["reject_cb"] > 0 and cnt["cb_fwd_ok"] > 0


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("warps", [2, 8])
def test_shell_launch_shapes(oracle, lib, warps, precision):
    s = W.spheres_256(seed=3)
    _compare(oracle, lib, s, 5, d_max=0.1, warps=warps, precision=precision)
    _compare(oracle, lib, s, 3, d_max=0.1, warps=warps, n_trial=2, precision=precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_shell_levels_down_to_the_full_ball(oracle, lib, precision):
    """d_max = 0.4: sqrt(3) d_max exceeds R_s, so the thickest levels have
    R_in = 0 (the whole circumsphere); dilute enough for moves to succeed."""
    s = W.make_system("dilute", W.SPHERE, 128, 0.05, 0.2, 0.2, seed=4)
    cnt, _ = _compare(oracle, lib, s, 8, d_max=0.4, precision=precision)
    assert cnt["accept"] > 0


@pytest.mark.parametrize("precision", PRECISIONS)
def test_shell_tiny_box_and_resume(oracle, lib, precision):
    s = W.make_system("tiny", W.SPHERE, 16, 0.2, 0.2, 0.2, seed=5)
    _compare(oracle, lib, s, 20, d_max=0.1, n_cell=2, precision=precision)
    _compare(oracle, lib, W.spheres_256(seed=6), 4, d_max=0.1, precision=precision,
             sweep0=123456)


@pytest.mark.parametrize("n_trial", [0, 2])
def test_shell_fp32_exact_paths(oracle, lib, n_trial):
    """A margin of 1 sends every FP32 shell decision and distance test to the
    exact FP64 re-take: the trajectory must not change."""
    cnt, _ = _compare(oracle, lib, W.spheres_256(seed=7), 3, d_max=0.1, n_trial=n_trial,
                      precision=1, margin=1.0)
    assert cnt["rechecks"] > cnt["dep_evaluated"]


def test_shell_zero_fugacity(oracle, lib):
    s = W.make_system("hs", W.SPHERE, 256, 0.3, 0.2, 0.0, seed=8)
    for precision in PRECISIONS:
        cnt, _ = _compare(oracle, lib, s, 10, d_max=0.1, precision=precision)
        assert cnt["dep_drawn"] == 0


@pytest.mark.parametrize("precision", PRECISIONS)
def test_shell_spheres_16384_first_sweeps(oracle, lib, precision):
    _compare(oracle, lib, W.spheres_16384(0.2), 2, d_max=0.1, precision=precision)


def test_shell_batch_replicas(oracle, lib):
    reps = W.batched_replicas(4, seed=9, n_min=60, n_max=900)
    desc = [{"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r, "n_trial": 0,
             "d_max": 0.04 + 0.02 * k, "replica": s.replica} for k, s in enumerate(reps)]
    for precision in PRECISIONS:
        ctx = lib.hpmc_init_batch(desc, seed=5, precision=precision)
        lib.hpmc_set_v0(ctx, SHELL)
        lib.hpmc_sweep(ctx, 5)
        for k, r in enumerate(desc):
            pos, _, cnt = lib.hpmc_get_replica(ctx, k, r["n"])
            ref, _, rc, _ = oracle.run(r["pos"], r["box_l"], q=r["q"], n_r=r["n_r"],
                                       d_max=r["d_max"], seed=5, replica=r["replica"],
                                       n_sweeps=5, v0_mode=SHELL)
            assert np.array_equal(pos, ref), k
            for name in oracle.PARITY_COUNTERS:
                assert cnt[name] == rc[name], (k, name)
        lib.hpmc_destroy(ctx)


def test_shell_switches_back(oracle, lib):
    """Shell for 3 sweeps, then the circumsphere: each leg equals the oracle's."""
    s = W.spheres_256(seed=10)
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.1, seed=1, precision=1, v0=SHELL)
    smp.sweep(3)
    lib.hpmc_set_v0(smp.ctx, 0)
    smp.sweep(2)
    pos, _, sweep, _ = smp.state()
    smp.close()
    p1, _, _, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.1, seed=1, n_sweeps=3,
                             v0_mode=SHELL)
    p2, _, _, _ = oracle.run(p1, s.L, q=s.q, n_r=s.n_r, d_max=0.1, seed=1, n_sweeps=2,
                             sweep0=3)
    assert sweep == 5 and np.array_equal(pos, p2)


def test_shell_is_for_spheres_only(lib):
    s = W.make_system("h", W.HEMISPHERE, 108, 0.25, 0.1, 0.3, seed=1)
    smp = lib.Sampler(s.pos, s.L, quat=s.quat, shape=s.shape, shape_params=s.shape_params,
                      q=s.q, n_r=s.n_r)
    with pytest.raises(lib.HPMCError):
        lib.hpmc_set_v0(smp.ctx, SHELL)
    with pytest.raises(lib.HPMCError):
        lib.hpmc_set_v0(smp.ctx, 3)
    lib.hpmc_set_v0(smp.ctx, 2)        # the cube is for every shape
    smp.close()


# --------------------------------------------------------------------------
# cube V_0
# --------------------------------------------------------------------------
CUBE = 2


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n_trial", [0, 2])
def test_cube_spheres(oracle, lib, precision, n_trial):
    s = W.spheres_256(seed=11)
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, n_trial=n_trial, d_max=0.1, seed=3,
                      precision=precision, v0=CUBE)
    smp.sweep(12)
    pos, _, sweep, cnt = smp.state()
    smp.close()
    ref, _, rc, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, n_trial=n_trial, d_max=0.1,
                               seed=3, n_sweeps=12, v0_mode=CUBE)
    for k in oracle.PARITY_COUNTERS:
        assert cnt[k] == rc[k], (k, cnt[k], rc[k])
    assert np.array_equal(pos, ref)
    assert cnt["accept"] > 0 and cnt["reject_depletant" if n_trial == 0 else "reject_cb"] > 0


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shape,phi,q,eta", [(W.HEMISPHERE, 0.25, 0.10, 0.12),
                                             (W.SPHEROID, 0.30, 0.10, 0.12)])
def test_cube_anisotropic_with_rotations(oracle, lib, precision, shape, phi, q, eta):
    # (the cube holds 1.9x the circumsphere's depletants: eta_r is kept below
    # the Poisson table's mean limit of 700)
    s = W.make_system("c", shape, 256, phi, q, eta, seed=12)
    kw = dict(q=s.q, n_r=s.n_r, d_max=0.08, a_max=0.2, p_translate=0.5)
    smp = lib.Sampler(s.pos, s.L, quat=s.quat, shape=s.shape, shape_params=s.shape_params,
                      seed=4, precision=precision, v0=CUBE, **kw)
    smp.sweep(6)
    pos, quat, _, cnt = smp.state(with_quat=True)
    smp.close()
    ref, refq, rc, _ = oracle.run(s.pos, s.L, shape=s.shape, shape_params=s.shape_params,
                                  quat=s.quat, seed=4, n_sweeps=6, v0_mode=CUBE, **kw)
    for k in oracle.PARITY_COUNTERS:
        assert cnt[k] == rc[k], (k, cnt[k], rc[k])
    assert np.array_equal(pos, ref) and np.array_equal(quat, refq)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_cube_spheres_16384_first_sweeps(oracle, lib, precision):
    s = W.spheres_16384(0.2)
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.1, seed=1, precision=precision,
                      v0=CUBE)
    smp.sweep(2)
    pos, _, _, cnt = smp.state()
    smp.close()
    ref, _, rc, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.1, seed=1, n_sweeps=2,
                               v0_mode=CUBE)
    for k in oracle.PARITY_COUNTERS:
        assert cnt[k] == rc[k], (k, cnt[k], rc[k])
    assert np.array_equal(pos, ref)


def test_cube_fp32_exact_paths(oracle, lib):
    """Margin 1: every FP32 decision of the cube lens kernel goes to FP64."""
    s = W.spheres_256(seed=13)
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.1, seed=3, precision=1, v0=CUBE)
    lib.hpmc_set_fp32_margin(smp.ctx, 1.0)
    smp.sweep(4)
    pos, _, _, cnt = smp.state()
    smp.close()
    ref, _, rc, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.1, seed=3, n_sweeps=4,
                               v0_mode=CUBE)
    for k in oracle.PARITY_COUNTERS:
        assert cnt[k] == rc[k], (k, cnt[k], rc[k])
    assert np.array_equal(pos, ref)
    assert cnt["rechecks"] > cnt["dep_evaluated"]
