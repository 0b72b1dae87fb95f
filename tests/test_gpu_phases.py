"""The persistent colour-phase schedule (all eight phases of a sweep in one
launch, per-cell readiness counters) and the looping phase grids (waves of
resident CTAs sharing a phase's cells) against the eight-launch schedule
with a CTA per cell, and the persistent schedule's bounded waits.

Both schedules run the same per-cell work in an order Sec. III.E allows (a
cell moves only after the non-empty cells of its neighbourhood that belong to
earlier phases), so trajectories and every counter must be identical.  The
bounded waits are exercised by host-side fault injection: one cell's
readiness is never published, the waits of its later-phase neighbours run
out, the sweep still finishes, the next synchronising call reports
HPMC_ERR_TIMEOUT, and the context keeps working after a state upload."""
import numpy as np
import pytest

from paper_1508_07077_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HPMC_ERR_TIMEOUT = -4
BENCH_DMAX = {0.1: 0.0223, 0.2: 0.0112, 0.3: 0.0075, 0.4: 0.0056}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07077_gb300 import build, hpmc
    build.build()
    hpmc.load()
    return hpmc


def _run(lib, reps, schedule, sweeps, **kw):
    ctx = lib.hpmc_init_batch(reps, seed=kw.get("seed", 1), precision=1)
    try:
        lib.hpmc_set_launch(ctx, 1, schedule)
        lib.hpmc_set_phase_waves(ctx, kw.get("waves", -1))
        if kw.get("soft"):
            lib.hpmc_set_soft(ctx, kw["soft"])
        if kw.get("v0"):
            lib.hpmc_set_v0(ctx, kw["v0"])
        lib.hpmc_sweep(ctx, sweeps)
        pos = np.empty((sum(r["n"] for r in reps), 3))
        sweep, cnt = lib.hpmc_get_state(ctx, pos)
        per = [lib.hpmc_get_replica(ctx, k, r["n"])[2] for k, r in enumerate(reps)]
    finally:
        lib.hpmc_destroy(ctx)
    return pos, sweep, cnt, per


def test_persistent_equals_launches_full_size(lib):
    systems = [W.spheres_16384(eta, seed=1) for eta in BENCH_DMAX]
    reps = [{"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r,
             "d_max": BENCH_DMAX[eta], "replica": k}
            for k, (s, eta) in enumerate(zip(systems, BENCH_DMAX))]
    a = _run(lib, reps, 1, 6)
    b = _run(lib, reps, 0, 6)
    assert np.array_equal(a[0], b[0])
    assert a[1] == b[1] == 6
    for k in a[2]:
        assert a[2][k] == b[2][k], k
    assert a[3] == b[3]
    assert a[2]["accept"] > 0


@pytest.mark.parametrize("n_trial,soft,v0", [(0, 0.0, 0), (3, 0.0, 0), (0, 10.0, 0),
                                              (0, 0.0, 1), (0, 0.0, 2)])
def test_persistent_equals_launches_batched(lib, n_trial, soft, v0):
    """Uneven replicas (N 60..900, n_c from 2 upwards), with CB, the soft
    interaction and the shell and cube V_0."""
    rng = np.random.default_rng(9)
    sys = [W.make_system("r%d" % k, W.SPHERE, int(rng.integers(60, 900)),
                         float(rng.uniform(0.1, 0.3)), float(rng.choice([0.1, 0.15, 0.2])),
                         float(rng.uniform(0.05, 0.25)), seed=9, replica=k) for k in range(24)]
    reps = [{"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r, "n_trial": n_trial,
             "d_max": 0.05, "replica": k} for k, s in enumerate(sys)]
    # and a box of two cells per side (the stencil is the whole box)
    reps.append({"n": 8, "box_l": 2.6, "pos": W.tiny_spheres(8, 2.6), "q": 0.2, "n_r": 30.0,
                 "n_trial": n_trial, "d_max": 0.08, "replica": 24})
    a = _run(lib, reps, 1, 8, soft=soft, v0=v0)
    b = _run(lib, reps, 0, 8, soft=soft, v0=v0)
    assert np.array_equal(a[0], b[0])
    for k in a[2]:
        assert a[2][k] == b[2][k], k


@pytest.mark.parametrize("waves", [1, 3, -1])
def test_phase_waves_equal_a_cta_per_cell_full_size(lib, waves):
    """4 x 16384 spheres: 8788 cells per phase, so one wave of the looping
    grid (24 CTAs per SM) gives some CTAs two cells or more."""
    systems = [W.spheres_16384(eta, seed=1) for eta in BENCH_DMAX]
    reps = [{"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r,
             "d_max": BENCH_DMAX[eta], "replica": k}
            for k, (s, eta) in enumerate(zip(systems, BENCH_DMAX))]
    a = _run(lib, reps, 0, 6, waves=waves)
    b = _run(lib, reps, 0, 6, waves=0)
    assert np.array_equal(a[0], b[0])
    for k in a[2]:
        assert a[2][k] == b[2][k], k
    assert a[3] == b[3]


@pytest.mark.parametrize("n_trial,soft,v0", [(3, 0.0, 0), (0, 10.0, 0), (0, 0.0, 1)])
def test_phase_waves_equal_a_cta_per_cell_batched(lib, n_trial, soft, v0):
    """96 uneven replicas (N 200..3000, down to two cells per side) with CB,
    the soft interaction and the shell V_0, one wave against a CTA per
    cell."""
    rng = np.random.default_rng(13)
    sys = [W.make_system("w%d" % k, W.SPHERE, int(rng.integers(200, 3000)),
                         float(rng.uniform(0.1, 0.3)), float(rng.choice([0.1, 0.15, 0.2])),
                         float(rng.uniform(0.05, 0.25)), seed=13, replica=k) for k in range(95)]
    reps = [{"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r, "n_trial": n_trial,
             "d_max": 0.05, "replica": k} for k, s in enumerate(sys)]
    reps.append({"n": 8, "box_l": 2.6, "pos": W.tiny_spheres(8, 2.6), "q": 0.2, "n_r": 30.0,
                 "n_trial": n_trial, "d_max": 0.08, "replica": 95})
    a = _run(lib, reps, 0, 6, soft=soft, v0=v0, waves=1)
    b = _run(lib, reps, 0, 6, soft=soft, v0=v0, waves=0)
    assert np.array_equal(a[0], b[0])
    for k in a[2]:
        assert a[2][k] == b[2][k], k


def test_bounded_wait_runs_out_and_the_context_recovers(lib):
    s = W.spheres_16384(0.2, seed=1)
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.0112, seed=1, precision=1,
                      schedule=lib.HPMC_PHASES_PERSISTENT)
    ctx = smp.ctx
    try:
        lib.hpmc_set_wait_limit(ctx, 0.02)
        lib.hpmc_debug_withhold_cell(ctx, 1000)
        timed_out = False
        for _ in range(16):      # the cell is non-empty and not in the last phase soon
            lib.hpmc_sweep(ctx, 1)
            try:
                lib.hpmc_sync(ctx)
            except lib.HPMCError as e:
                assert e.code == HPMC_ERR_TIMEOUT
                timed_out = True
                break
        assert timed_out
        # the kernel finished: the state can be read, and after an upload (which
        # clears the error) the context sweeps normally again
        pos = np.empty((s.n, 3))
        with pytest.raises(lib.HPMCError) as e:
            lib.hpmc_get_state(ctx, pos)
        assert e.value.code == HPMC_ERR_TIMEOUT
        assert np.all((pos >= 0.0) & (pos < s.L))
        lib.hpmc_debug_withhold_cell(ctx, -1)
        lib.hpmc_set_wait_limit(ctx, 1.0)
        sweep0 = 100
        lib.hpmc_set_state(ctx, pos, None, sweep0)
        lib.hpmc_sweep(ctx, 3)          # re-validates: HPMC_ERR_OVERLAP if a move went wrong
        lib.hpmc_sync(ctx)
        sweep, cnt = lib.hpmc_get_state(ctx, pos)
        assert sweep == sweep0 + 3
    finally:
        smp.close()


def test_wait_limit_arguments(lib):
    s = W.spheres_256()
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, precision=1)
    try:
        for bad in (0.0, -1.0, 100.0, float("nan")):
            with pytest.raises(lib.HPMCError):
                lib.hpmc_set_wait_limit(smp.ctx, bad)
        with pytest.raises(lib.HPMCError):
            lib.hpmc_debug_withhold_cell(smp.ctx, -2)
        with pytest.raises(lib.HPMCError):
            lib.hpmc_set_launch(smp.ctx, 1, 2)
        for bad in (-2, 65):
            with pytest.raises(lib.HPMCError):
                lib.hpmc_set_phase_waves(smp.ctx, bad)
        lib.hpmc_set_phase_waves(smp.ctx, 64)
        lib.hpmc_sweep(smp.ctx, 1)
    finally:
        smp.close()
