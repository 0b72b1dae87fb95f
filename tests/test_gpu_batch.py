"""GPU parity of batched replicas: one context, one set of launches per sweep
for all replicas, each replica bit-identical to the oracle run of the same
system alone (its own state point, size and RNG key)."""
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


def _replicas(count=5, seed=3):
    reps = W.batched_replicas(count, seed=seed, n_min=60, n_max=900)
    out = []
    for k, s in enumerate(reps):
        out.append({"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r,
                    "n_trial": 0, "d_max": 0.06, "replica": s.replica, "sys": s})
    return out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n_trial", [0, 2])
def test_batch_replicas_match_oracle(oracle, lib, precision, n_trial):
    reps = _replicas()
    for r in reps:
        r["n_trial"] = n_trial
    ctx = lib.hpmc_init_batch(reps, seed=7, precision=precision)
    sweeps = 6
    lib.hpmc_sweep(ctx, sweeps)
    allpos = np.empty((sum(r["n"] for r in reps), 3))
    sweep, tot = lib.hpmc_get_state(ctx, allpos)
    assert sweep == sweeps
    off = 0
    summed = {k: 0 for k in oracle.PARITY_COUNTERS}
    for k, r in enumerate(reps):
        pos, _, cnt = lib.hpmc_get_replica(ctx, k, r["n"])
        ref, _, rc, _ = oracle.run(r["pos"], r["box_l"], q=r["q"], n_r=r["n_r"],
                                   n_trial=n_trial, d_max=r["d_max"], seed=7,
                                   replica=r["replica"], n_sweeps=sweeps)
        assert np.array_equal(pos, ref), k
        assert np.array_equal(allpos[off:off + r["n"]], ref)
        for name in oracle.PARITY_COUNTERS:
            assert cnt[name] == rc[name], (k, name)
            summed[name] += rc[name]
        off += r["n"]
    for name in oracle.PARITY_COUNTERS:
        assert tot[name] == summed[name]
    lib.hpmc_destroy(ctx)


def test_batch_per_replica_moves_and_resume(oracle, lib):
    reps = _replicas(3, seed=11)
    ctx = lib.hpmc_init_batch(reps, seed=2, precision=1)
    lib.hpmc_set_replica_moves(ctx, 1, 0.02)
    lib.hpmc_sweep(ctx, 4)
    mid = np.empty((sum(r["n"] for r in reps), 3))
    sweep, _ = lib.hpmc_get_state(ctx, mid)
    lib.hpmc_set_state(ctx, mid, None, sweep)
    lib.hpmc_sweep(ctx, 3)
    for k, r in enumerate(reps):
        pos, _, _ = lib.hpmc_get_replica(ctx, k, r["n"])
        d = 0.02 if k == 1 else r["d_max"]
        ref, _, _, _ = oracle.run(r["pos"], r["box_l"], q=r["q"], n_r=r["n_r"], d_max=d,
                                  seed=2, replica=r["replica"], n_sweeps=7)
        assert np.array_equal(pos, ref), k
    lib.hpmc_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_mixed_configurational_bias(oracle, lib, precision):
    """Replicas with and without configurational bias in one batch: the
    rejections of the n_trial = 0 replicas count as depletant rejections."""
    reps = _replicas(4, seed=5)
    for k, r in enumerate(reps):
        r["n_trial"] = 3 if k % 2 else 0
    ctx = lib.hpmc_init_batch(reps, seed=9, precision=precision)
    lib.hpmc_sweep(ctx, 5)
    for k, r in enumerate(reps):
        pos, _, cnt = lib.hpmc_get_replica(ctx, k, r["n"])
        ref, _, rc, _ = oracle.run(r["pos"], r["box_l"], q=r["q"], n_r=r["n_r"],
                                   n_trial=r["n_trial"], d_max=r["d_max"], seed=9,
                                   replica=r["replica"], n_sweeps=5)
        assert np.array_equal(pos, ref), k
        for name in oracle.PARITY_COUNTERS:
            assert cnt[name] == rc[name], (k, name, cnt[name], rc[name])
    lib.hpmc_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_degenerate_replicas_match_oracle(oracle, lib, precision):
    """Replicas at the edges of the batch next to ordinary ones: a single
    colloid (no neighbour ever), two colloids near contact, a replica with no
    depletants (n_r = 0: every move that stays in its cell and overlaps
    nothing is accepted) and a box of two cells per side; each bit-identical
    to the oracle run of the same system alone."""
    reps = _replicas(count=3, seed=11)
    L1 = 4.0
    # (alone, any lens point blocks the move: few depletants, so that it moves)
    reps.append({"n": 1, "box_l": L1, "pos": np.array([[1.3, 2.1, 0.7]]), "q": 0.15,
                 "n_r": 2.0, "n_trial": 0, "d_max": 0.08, "replica": 40})
    reps.append({"n": 2, "box_l": L1, "pos": np.array([[1.0, 1.0, 1.0], [2.0005, 1.0, 1.0]]),
                 "q": 0.15, "n_r": 40.0, "n_trial": 0, "d_max": 0.08, "replica": 41})
    s0 = W.make_system("nodep", W.SPHERE, 300, 0.25, 0.15, 0.0, seed=4, replica=42)
    reps.append({"n": s0.n, "box_l": s0.L, "pos": s0.pos, "q": s0.q, "n_r": 0.0,
                 "n_trial": 0, "d_max": 0.06, "replica": 42})
    reps.append({"n": 8, "box_l": 2.6, "pos": W.tiny_spheres(8, 2.6), "q": 0.2, "n_r": 30.0,
                 "n_trial": 0, "d_max": 0.08, "replica": 43})
    ctx = lib.hpmc_init_batch(reps, seed=9, precision=precision)
    sweeps = 12
    lib.hpmc_sweep(ctx, sweeps)
    for k, r in enumerate(reps):
        pos, _, cnt = lib.hpmc_get_replica(ctx, k, r["n"])
        ref, _, rc, _ = oracle.run(r["pos"], r["box_l"], q=r["q"], n_r=r["n_r"],
                                   n_trial=0, d_max=r["d_max"], seed=9,
                                   replica=r["replica"], n_sweeps=sweeps)
        assert np.array_equal(pos, ref), k
        for name in oracle.PARITY_COUNTERS:
            assert cnt[name] == rc[name], (k, name)
    # the single colloid moved; the replica without depletants drew none
    c1 = lib.hpmc_get_replica(ctx, 3, 1)[2]
    assert c1["accept"] > 0
    c_nodep = lib.hpmc_get_replica(ctx, 5, reps[5]["n"])[2]
    assert c_nodep["dep_drawn"] == 0 and c_nodep["accept"] > 0
    lib.hpmc_destroy(ctx)
