"""GPU parity of the Gibbs-ensemble colloid exchange (Sec. IV.B) against the
oracle, through the C ABI: cycles of checkerboard sweeps of both boxes and
exchange attempts; the boxes' colloids in use, every trajectory counter of
each box and the pair's exchange counters must be identical."""
import numpy as np
import pytest

from paper_1508_07077_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

Q = 0.2


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07077_gb300 import build, hpmc
    build.build()
    hpmc.load()
    return hpmc


def _pair(n0, phi0, n1, phi1, eta, seed):
    a = W.make_system("g0", W.SPHERE, n0, phi0, Q, eta, seed=seed)
    b = W.make_system("g1", W.SPHERE, n1, phi1, Q, eta, seed=seed + 1)
    return a, b


def _compare(oracle, lib, pairs, cycles, sweeps, exchanges, precision, seed=3, margin=0.0):
    gp = lib.GibbsPairs([((a.pos, a.L), (b.pos, b.L), prm) for a, b, prm in pairs],
                        seed=seed, precision=precision)
    if margin:
        lib.hpmc_set_fp32_margin(gp.ctx, margin)
    for _ in range(cycles):
        gp.cycle(sweeps, exchanges)
    boxes = gp.boxes()
    gib = [lib.hpmc_get_gibbs(gp.ctx, p) for p in range(len(pairs))]
    gp.close()
    for p, (a, b, prm) in enumerate(pairs):
        dm = prm.get("d_max", 0.1)
        p0, p1, c0, c1, g = oracle.gibbs_run(
            a.pos, b.pos, a.L, b.L, q=prm["q"], n_r=prm["n_r"], n_trial=prm["n_trial"],
            d_max=(dm, dm), seed=seed, replicas=(2 * p, 2 * p + 1), n_cycles=cycles,
            sweeps_per_cycle=sweeps, ex_per_cycle=exchanges)
        step, gc = gib[p]
        assert step == cycles * exchanges
        assert gc == g, (gc, g)
        for (pos, cnt), ref, rc in ((boxes[2 * p], p0, c0), (boxes[2 * p + 1], p1, c1)):
            assert pos.shape == ref.shape
            assert np.array_equal(pos, ref)
            for k in oracle.PARITY_COUNTERS:
                assert cnt[k] == rc[k], (p, k, cnt[k], rc[k])
    return gib


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n_trial,eta", [(0, 0.003), (8, 0.05), (40, 0.08)])
def test_gibbs_pair_matches_oracle(oracle, lib, precision, n_trial, eta):
    a, b = _pair(48, 0.15, 24, 0.06, eta, seed=5)
    prm = {"q": Q, "n_r": a.n_r, "n_trial": n_trial, "d_max": 0.1}
    gib = _compare(oracle, lib, [(a, b, prm)], 8, 1, 12, precision)
    g = gib[0][1]
    assert g["accept"] > 0 and g["reject_ratio"] > 0


@pytest.mark.parametrize("precision", [0, 1])
def test_two_pairs_in_one_context(oracle, lib, precision):
    a, b = _pair(40, 0.12, 30, 0.10, 0.04, seed=7)
    c, d = _pair(20, 0.05, 50, 0.20, 0.01, seed=9)
    pairs = [(a, b, {"q": Q, "n_r": a.n_r, "n_trial": 6, "d_max": 0.08}),
             (c, d, {"q": Q, "n_r": c.n_r, "n_trial": 0, "d_max": 0.12})]
    _compare(oracle, lib, pairs, 6, 2, 8, precision)


def test_gibbs_empty_box_and_many_attempts(oracle, lib):
    """Box 1 starts empty: the first accepted exchanges fill it; attempts that
    pick an empty source are counted and rejected."""
    a = W.make_system("g0", W.SPHERE, 12, 0.05, Q, 0.002, seed=11)
    b = W.make_system("g1", W.SPHERE, 12, 0.05, Q, 0.002, seed=12)
    empty = type(b)(**{**b.__dict__, "n": 0, "pos": np.zeros((0, 3))})
    gib = _compare(oracle, lib, [(a, empty, {"q": Q, "n_r": a.n_r, "n_trial": 0})], 5, 1, 40, 1)
    assert gib[0][1]["accept"] > 0


def test_gibbs_argument_errors(lib):
    a, b = _pair(20, 0.1, 20, 0.1, 0.01, seed=13)
    gp = lib.GibbsPairs([((a.pos, a.L), (b.pos, b.L), {"q": Q, "n_r": a.n_r})])
    with pytest.raises(lib.HPMCError):
        lib.hpmc_set_live(gp.ctx, 0, 41)          # beyond the replica's slots
    gp.close()
    # the exchange inserts its depletants in the circumsphere, hard interaction
    for setter, value in ((lib.hpmc_set_v0, 1), (lib.hpmc_set_v0, 2), (lib.hpmc_set_soft, 3.0)):
        gp = lib.GibbsPairs([((a.pos, a.L), (b.pos, b.L), {"q": Q, "n_r": a.n_r})],
                            precision=0)
        setter(gp.ctx, value)
        with pytest.raises(lib.HPMCError) as e:
            lib.hpmc_gibbs_exchange(gp.ctx, 1)
        assert e.value.code == -1
        gp.close()
    s = W.spheres_256()
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r)
    with pytest.raises(lib.HPMCError):
        lib.hpmc_gibbs_exchange(smp.ctx, 1)       # one replica: no pair
    smp.close()


def test_gibbs_fp32_exact_paths(oracle, lib):
    """A margin of 1 sends every FP32 point test and distance of the exchange
    (and of the sweeps) to FP64: the trajectory must not change."""
    a, b = _pair(40, 0.15, 24, 0.06, 0.05, seed=15)
    prm = {"q": Q, "n_r": a.n_r, "n_trial": 6, "d_max": 0.1}
    _compare(oracle, lib, [(a, b, prm)], 4, 1, 10, 1, margin=1.0)
