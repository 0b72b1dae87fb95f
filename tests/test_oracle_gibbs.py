"""Pins of the Gibbs-ensemble colloid exchange (Sec. IV.B: a colloid moves to
a random position in the other box; depletants are inserted at the new
position and, with configurational bias, reinserted in the old box).

What statistical mechanics fixes:
* detailed balance of one exchange: for boxes of volumes V_s, V_d with N_s,
  N_d colloids, P(s -> d) / P(d -> s) = N_s V_d / ((N_d + 1) V_s) *
  exp(z_p dV_f), where dV_f (free volume gained) = lens(r) - lens(r') for an
  inserted sphere whose new neighbour sits at r and whose old one sat at r'
  (AO lens volumes, Eq. 5-11 with the Gibbs prior; Eq. 12 with CB);
* without depletants and with vanishing excluded volume, the colloid number
  of a box is Binomial(N, V_0 / (V_0 + V_1));
* colloids are conserved and no run leaves an overlap.
"""
import math

import numpy as np
import pytest

from tests.test_oracle_physics import lens

Q = 0.2


def _boxes(r_new, r_old):
    """Box 0 (L = 4): colloid 0 at c0 with a neighbour at distance r_old;
    box 1 (L = 4.4): one colloid at distance r_new from the insertion point."""
    c0 = np.array([1.0, 1.0, 1.0])
    d = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    box0 = np.array([c0, c0 + r_old * d])
    x = np.array([2.0, 2.0, 2.0])
    box1 = np.array([x + r_new * np.array([1.0, 0.0, 0.0])])
    return box0, box1, x


@pytest.mark.parametrize("n_trial,eta", [(0, 0.002), (5, 0.02), (12, 0.04)])
@pytest.mark.parametrize("r_new,r_old", [(1.05, 1.3), (1.3, 1.08)])
def test_exchange_detailed_balance(oracle, n_trial, eta, r_new, r_old):
    z = eta / (math.pi / 6.0 * Q ** 3)
    L0, L1 = 4.0, 4.4
    box0, box1, x = _boxes(r_new, r_old)
    n_rep = 200000
    kw = dict(q=Q, n_r=z, n_trial=n_trial, n_rep=n_rep)
    f, _ = oracle.gibbs_acceptance(box0, box1, L0, L1, 0, 0, x, **kw)
    # the reverse: the inserted colloid (slot 1 of box 1) back to its old place
    rev1 = np.vstack([box1, x])
    rev0 = box0[1:]
    b, _ = oracle.gibbs_acceptance(rev0, rev1, L0, L1, 1, 1, box0[0], step0=10 ** 7, **kw)
    G = (2 * L1 ** 3) / (2 * L0 ** 3)
    expect = G * math.exp(z * float(lens(r_new) - lens(r_old)))
    ratio = f / b
    se = ratio * math.sqrt(1.0 / f + 1.0 / b)
    assert min(f, b) > 2000, (f, b)
    assert abs(ratio - expect) < 4.0 * se, (ratio, expect, se)


def test_exchange_without_cb_power(oracle):
    """At the CB cases' fugacity, n_trial = 0 almost never accepts an
    insertion (the point of the reinsertion scheme)."""
    z = 0.04 / (math.pi / 6.0 * Q ** 3)
    box0, box1, x = _boxes(1.3, 1.3)
    a0, _ = oracle.gibbs_acceptance(box0, box1, 4.0, 4.4, 0, 0, x, q=Q, n_r=z, n_rep=20000)
    a12, _ = oracle.gibbs_acceptance(box0, box1, 4.0, 4.4, 0, 0, x, q=Q, n_r=z, n_trial=12,
                                     n_rep=20000)
    assert a0 < 20 and a12 > 2000, (a0, a12)


def test_ideal_gas_box_occupancy_is_binomial(oracle):
    """z_p = 0 and spheres of diameter 0.02: N_0 ~ Binomial(N, V_0/(V_0+V_1))."""
    N, L0, L1 = 10, 3.0, 3.6
    p = L0 ** 3 / (L0 ** 3 + L1 ** 3)
    rng = np.random.default_rng(4)
    counts = np.zeros(N + 1)
    per_seed = []
    for seed in range(1, 9):
        pos0 = rng.uniform(0, L0, size=(N // 2, 3))
        pos1 = rng.uniform(0, L1, size=(N - N // 2, 3))
        h = np.zeros(N + 1)
        sweep, step = 0, 0
        for cycle in range(2500):
            pos0, pos1, _, _, g = oracle.gibbs_run(pos0, pos1, L0, L1, diameter=0.02, q=0.0,
                                                   seed=seed, sweep0=sweep, step0=step,
                                                   n_cycles=1, sweeps_per_cycle=0,
                                                   ex_per_cycle=3)
            step += 3
            h[len(pos0)] += 1
        counts += h
        per_seed.append(h / h.sum())
    per_seed = np.array(per_seed)
    m, se = per_seed.mean(0), per_seed.std(0, ddof=1) / math.sqrt(len(per_seed))
    expect = np.array([math.comb(N, k) * p ** k * (1 - p) ** (N - k) for k in range(N + 1)])
    sel = expect > 0.01
    z = (m[sel] - expect[sel]) / np.maximum(se[sel], 1e-4)
    assert np.all(np.abs(z) < 4.5), (m, expect)


def test_pair_run_conserves_and_stays_valid(oracle):
    from paper_1508_07077_gb300 import workloads as W
    a = W.make_system("g0", W.SPHERE, 64, 0.15, Q, 0.05, seed=3)
    b = W.make_system("g1", W.SPHERE, 40, 0.08, Q, 0.05, seed=4)
    b_pos = b.pos * (b.L / b.L)
    p0, p1, c0, c1, g = oracle.gibbs_run(a.pos, b_pos, a.L, b.L, q=Q, n_r=a.n_r, n_trial=8,
                                         d_max=(0.1, 0.1), seed=2, n_cycles=20, ex_per_cycle=10)
    assert len(p0) + len(p1) == 104
    assert g["attempts"] == 200 and g["accept"] > 0
    assert g["accept"] + sum(g[k] for k in ("reject_empty", "reject_ratio", "reject_overlap",
                                            "reject_depletant", "reject_cb")) == 200
    for p, L in ((p0, a.L), (p1, b.L)):
        assert np.all((p >= 0) & (p < L))
        d = p[:, None, :] - p[None, :, :]
        d -= L * np.round(d / L)
        r2 = (d ** 2).sum(-1) + 4.0 * np.eye(len(p))
        assert r2.min() >= 1.0
    assert c0["moves"] > 0 and c1["moves"] > 0
