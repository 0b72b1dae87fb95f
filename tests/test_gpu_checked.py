"""The checked build (libhpmc_dep_checked.so, -DHPMC_CHECKED) on small
systems of the FP32 form, spheres and (last test) hemispheres and discoids.
On the sphere path every cell, bin, neighbour, shared-memory and colloid
index is bounds-checked, and every colloid a move reads is checked to sit in
its own cell or in a cell that is not active in the same colour phase
(Sec. III.E), in both colour-phase schedules.  On every path each decision
FP32 takes as certain (ball, new and old pose, cell exit, colloid pair, lens
point against the neighbours, CB trials) is re-taken in FP64 and must agree,
which checks the certified margins on every test, not only on those that
reach the trajectory.  The error word must stay zero and the trajectories
must be the oracle's, bit for bit (the checks observe, they change
nothing)."""
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
    prev = hpmc.use(hpmc.CHECKED_LIB_PATH)
    yield hpmc
    hpmc.use(prev)


CASES = {
    "spheres_256": lambda: W.spheres_256(),
    "spheres_2048_phi0.30_q0.15": lambda: W.make_system("c2", W.SPHERE, 2048, 0.30, 0.15, 0.2,
                                                        seed=3),
    "tiny_two_cells": lambda: W.System("tiny", W.SPHERE, 8, 2.6, 0.2, 30.0,
                                       W.tiny_spheres(8, 2.6), None),
}


@pytest.mark.parametrize("schedule", [1, 0])
@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("n_trial", [0, 3])
def test_checked_build_is_clean_and_exact(oracle, lib, case, schedule, n_trial):
    s = CASES[case]()
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, n_trial=n_trial, d_max=0.06, seed=2,
                      precision=1, schedule=schedule)
    try:
        smp.sweep(6)
        lib.hpmc_sync(smp.ctx)            # raises on a recorded check
        pos, _, sweep, cnt = smp.state()
    finally:
        smp.close()
    ref, _, rc, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, n_trial=n_trial, d_max=0.06, seed=2,
                               n_sweeps=6)
    assert sweep == 6
    assert np.array_equal(pos, ref)
    for k in oracle.PARITY_COUNTERS:
        assert cnt[k] == rc[k], k


@pytest.mark.parametrize("soft,v0", [(10.0, 0), (0.0, 1), (0.0, 2)])
def test_checked_build_batched_variants(oracle, lib, soft, v0):
    """A batch of uneven replicas with the soft interaction, the shell and
    the cube V_0."""
    rng = np.random.default_rng(4)
    sys = [W.make_system("r%d" % k, W.SPHERE, int(rng.integers(80, 600)),
                         float(rng.uniform(0.1, 0.3)), float(rng.choice([0.1, 0.15, 0.2])),
                         float(rng.uniform(0.05, 0.3)), seed=4, replica=k) for k in range(6)]
    reps = [{"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r, "d_max": 0.05,
             "replica": k} for k, s in enumerate(sys)]
    ctx = lib.hpmc_init_batch(reps, seed=4, precision=1)
    try:
        if soft:
            lib.hpmc_set_soft(ctx, soft)
        if v0:
            lib.hpmc_set_v0(ctx, v0)
        lib.hpmc_sweep(ctx, 5)
        lib.hpmc_sync(ctx)
        got = [lib.hpmc_get_replica(ctx, k, r["n"]) for k, r in enumerate(reps)]
    finally:
        lib.hpmc_destroy(ctx)
    for k, r in enumerate(reps):
        ref, _, rc, _ = oracle.run(r["pos"], r["box_l"], q=r["q"], n_r=r["n_r"], d_max=0.05,
                                   seed=4, replica=k, n_sweeps=5, soft_eps=soft, v0_mode=v0)
        assert np.array_equal(got[k][0], ref), k
        for name in oracle.PARITY_COUNTERS:
            assert got[k][2][name] == rc[name], (k, name)


ANISO = [(W.HEMISPHERE, 0.25, 0.10, 0.30), (W.SPHEROID, 0.30, 0.10, 0.25)]


@pytest.mark.parametrize("shape,phi,q,eta", ANISO)
@pytest.mark.parametrize("n_trial", [0, 3])
def test_checked_build_anisotropic(oracle, lib, shape, phi, q, eta, n_trial):
    """Hemispheres and discoids with rotation moves in the FP32 form: every
    shape decision FP32 takes as certain (ball, new and old pose in the lens
    kernel, colloid pairs, lens points against the neighbours, CB trials) is
    re-taken in FP64 and must agree; the trajectory is the oracle's."""
    s = W.make_system("small", shape, 256, phi, q, eta, seed=1)
    smp = lib.Sampler(s.pos, s.L, quat=s.quat, shape=s.shape, shape_params=s.shape_params,
                      q=s.q, n_r=s.n_r, n_trial=n_trial, d_max=0.08, a_max=0.2, p_translate=0.5,
                      seed=2, precision=1)
    try:
        smp.sweep(4)
        lib.hpmc_sync(smp.ctx)            # raises on a recorded check
        pos, quat, sweep, cnt = smp.state(with_quat=True)
    finally:
        smp.close()
    ref, refq, rc, _ = oracle.run(s.pos, s.L, shape=s.shape, shape_params=s.shape_params,
                                  quat=s.quat, q=s.q, n_r=s.n_r, n_trial=n_trial, d_max=0.08,
                                  a_max=0.2, p_translate=0.5, seed=2, n_sweeps=4)
    assert sweep == 4
    assert np.array_equal(pos, ref)
    assert np.array_equal(quat, refq)
    for k in oracle.PARITY_COUNTERS:
        assert cnt[k] == rc[k], k
    # (with CB a blocked move counts as a CB rejection)
    assert cnt["reject_depletant"] + cnt["reject_cb"] > 0 and cnt["reject_overlap"] > 0
