"""Statistical pins of the oracle against what the paper and textbook
statistical mechanics fix.

* Detailed balance (Sec. III.B-C, Eqs. 5-11): for a fixed pair of colloid
  configurations, P_acc(M->M') / P_acc(M'->M) = exp(z_p [V_f(M') - V_f(M)]).
  With two spheres V_f changes only by the Asakura-Oosawa lens volume.
  Checked for n_trial = 0 and for the configurational-bias weight (Eq. 12).
* The Asakura-Oosawa two-colloid distribution P(r) ~ r^2 exp(z_p V_lens(r))
  that the semigrand weight exp(z_p V_f - beta H_cc) (Eq. 2) implies.
* The hard-sphere limit z_p = 0: contact value vs Carnahan-Starling, and the
  scaled-particle-theory free-volume fraction (Sec. IV.A observable).
* The exact free-volume fraction of a single colloid.
* Detailed balance with three spheres whose excluded spheres share a region
  (q = 0.4): the acceptance ratio of a move and its reverse is
  exp(z_p Delta V_f), V_f from inclusion-exclusion with the triple-overlap
  volume, which the pairwise prediction misses.
* The many-body reduction: for q < 2/sqrt(3) - 1 no point lies in three
  excluded spheres, so the free volume is V minus the excluded spheres plus
  their pairwise lens overlaps, and the implicit-depletant chain samples
  exactly the pairwise Asakura-Oosawa fluid; its pair statistics near contact
  must equal those of a plain Metropolis chain of that pair potential (written
  here, sharing nothing with the oracle).
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import pairwise_ao as PA
from paper_1508_07077_gb300 import workloads as W

Q, R_S, Z_P, L2 = 0.2, 0.6, 47.7464829275686, 2.4


def lens(r, R=R_S):
    """Overlap volume of two spheres of radius R at centre distance r."""
    r = np.asarray(r, dtype=float)
    return np.where(r < 2 * R, math.pi / 12.0 * (4 * R + r) * (2 * R - r) ** 2, 0.0)


def _pair(r):
    a = np.array([0.2, 0.2, 0.2])
    d = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    return a, a + r * d


def _ratio(oracle, r0, r1, n_trial, cb_mode, n_rep):
    a, b0 = _pair(r0)
    _, b1 = _pair(r1)
    f, _ = oracle.acceptance(np.array([a, b0]), L2, 1, b1, q=Q, n_r=Z_P,
                             n_trial=n_trial, cb_mode=cb_mode, n_rep=n_rep)
    b, _ = oracle.acceptance(np.array([a, b1]), L2, 1, b0, q=Q, n_r=Z_P,
                             n_trial=n_trial, cb_mode=cb_mode, n_rep=n_rep,
                             sweep0=10 ** 7)
    ratio = f / b
    se = ratio * math.sqrt(1.0 / f + 1.0 / b)
    expect = math.exp(Z_P * float(lens(r1) - lens(r0)))
    return ratio, se, expect


@pytest.mark.parametrize("n_trial", [0, 1, 3, 10])
@pytest.mark.parametrize("r0,r1", [(1.05, 1.10), (1.02, 1.09)])
def test_detailed_balance_of_acceptance(oracle, n_trial, r0, r1):
    ratio, se, expect = _ratio(oracle, r0, r1, n_trial, 0, 150000)
    assert abs(ratio - expect) < 4.0 * se, (ratio, expect, se)


def test_literal_printed_cb_weight_breaks_detailed_balance(oracle):
    """The alternative, literal reading of Eq. (12), with the extra factor
    (N_i + 1)/N_i and n_trial fresh reverse trials, fails the same test: the
    test has the power to reject a wrong weight."""
    ratio, se, expect = _ratio(oracle, 1.02, 1.09, 10, 1, 150000)
    assert abs(ratio - expect) > 6.0 * se, (ratio, expect, se)


@pytest.mark.parametrize("n_trial", [0, 5])
def test_asakura_oosawa_pair_distribution(oracle, n_trial):
    bins, rmax, lo = 24, 1.2, 20          # bins of 0.05 starting at contact
    edges = np.linspace(0.0, rmax, bins + 1)
    expect = []
    for b in range(lo, bins):
        r = np.linspace(edges[b], edges[b + 1], 401)
        expect.append(np.trapezoid(r ** 2 * np.exp(Z_P * lens(r)), r))
    expect = np.array(expect) / np.sum(expect)
    a, b = _pair(1.5)
    hs = []
    for seed in range(1, 9):
        _, _, _, h = oracle.run(np.array([a, b]), L2, q=Q, n_r=Z_P, n_trial=n_trial,
                                d_max=0.03, seed=seed, n_sweeps=60000,
                                hist_bins=bins, hist_rmax=rmax)
        h = h[lo:].astype(float)
        hs.append(h / h.sum())
    hs = np.array(hs)
    m, se = hs.mean(0), hs.std(0, ddof=1) / math.sqrt(len(hs))
    z = (m - expect) / se
    assert np.all(np.abs(z) < 4.0), z
    # the depletion attraction is visible: contact bin well above r^2 alone
    r2 = np.array([(edges[b + 1] ** 3 - edges[b] ** 3) for b in range(lo, bins)])
    assert m[0] / m[-1] > 2.0 * r2[0] / r2[-1]


def _hard_spheres(oracle, phi, n_eq=2000, n_run=8000):
    s = W.make_system("hs", W.SPHERE, 256, phi, 0.2, 0.0)
    pos, _, _, _ = oracle.run(s.pos, s.L, q=0.2, n_r=0.0, d_max=0.1, n_sweeps=n_eq)
    bins, rmax = 130, 1.3
    pos2, _, _, h = oracle.run(pos, s.L, q=0.2, n_r=0.0, d_max=0.1, n_sweeps=n_run,
                               sweep0=n_eq, hist_bins=bins, hist_rmax=rmax)
    return s, pos2, h, bins, rmax, n_run


@pytest.mark.parametrize("phi", [0.2, 0.3])
def test_hard_sphere_limit_carnahan_starling(oracle, phi):
    s, pos, h, bins, rmax, n_run = _hard_spheres(oracle, phi)
    edges = np.linspace(0.0, rmax, bins + 1)
    rho = s.n / s.L ** 3
    shell = 4.0 * math.pi / 3.0 * (edges[1:] ** 3 - edges[:-1] ** 3)
    g = h / (n_run * s.n / 2.0 * rho * shell)
    mid = 0.5 * (edges[1:] + edges[:-1])
    sel = (mid > 1.0) & (mid < 1.08)
    g1 = np.polyval(np.polyfit(mid[sel], g[sel], 2), 1.0)
    Z = 1.0 + 4.0 * phi * g1
    Z_cs = (1 + phi + phi ** 2 - phi ** 3) / (1 - phi) ** 3
    assert abs(Z / Z_cs - 1.0) < 0.025, (Z, Z_cs)
    # free-volume fraction of a q=0.2 test sphere vs scaled-particle theory
    alpha = oracle.free_volume(pos, s.L, 0.2, n_probe=100000)
    gam, q = phi / (1 - phi), 0.2
    A, B, C = 3 * q + 3 * q * q + q ** 3, 4.5 * q * q + 3 * q ** 3, 3 * q ** 3
    spt = (1 - phi) * math.exp(-A * gam - B * gam ** 2 - C * gam ** 3)
    assert abs(alpha / spt - 1.0) < 0.02, (alpha, spt)


def test_single_colloid_free_volume_exact(oracle):
    L, q = 3.0, 0.3
    alpha = oracle.free_volume(np.array([[1.0, 2.0, 0.5]]), L, q, n_probe=400000)
    exact = 1.0 - 4.0 / 3.0 * math.pi * (0.5 + q / 2) ** 3 / L ** 3
    assert abs(alpha - exact) < 4.0 * math.sqrt(exact * (1 - exact) / 400000)


def _mb_oracle(oracle, z_p, n_eq=4000, n_run=12000):
    """Pair counts per colloid and sweep in the bins from contact to 1.2, one
    row per independent oracle chain (seeds 1..16, from the same start)."""
    L, _, pos0 = PA.system()

    def chain(seed):
        p, _, _, _ = oracle.run(pos0, L, q=PA.Q, n_r=z_p, d_max=0.03, n_sweeps=n_eq, seed=seed)
        _, _, _, h = oracle.run(p, L, q=PA.Q, n_r=z_p, d_max=0.03, n_sweeps=n_run, seed=seed,
                                sweep0=n_eq, hist_bins=PA.BINS, hist_rmax=PA.RMAX)
        return h[PA.LO:].astype(float) / (n_run * PA.N)

    with ThreadPoolExecutor(max_workers=8) as ex:
        return np.array(list(ex.map(chain, range(1, PA.GROUPS + 1))))


def test_many_body_reduction_to_pairwise_asakura_oosawa(oracle):
    """Below q = 2/sqrt(3) - 1 the implicit-depletant chain of 32 spheres has
    the pair statistics of the pairwise Asakura-Oosawa fluid (chi^2 of the four
    bins from contact to r = 1.2 below its 0.999 quantile).  Two controls: the
    attraction is visible (the contact bin well above the hard spheres'), and
    the test has the power to reject a wrong potential (the oracle at
    0.75 z_p fails it)."""
    _, z_p, _ = PA.system()
    ref = PA.pairwise_counts()
    got = _mb_oracle(oracle, z_p)
    chi2, z = PA.chi2(got, ref)
    assert chi2 < PA.CHI2_999, z
    hard = _mb_oracle(oracle, 0.0, n_eq=1000, n_run=4000)
    assert got.mean(0)[0] > 1.2 * hard.mean(0)[0], (got.mean(0), hard.mean(0))
    wrong = _mb_oracle(oracle, 0.75 * z_p)
    chi2_w, z_w = PA.chi2(wrong, ref)
    assert chi2_w > 30.0, z_w


# three spheres whose excluded spheres (radius 0.7 at q = 0.4) share a region;
# colloid i moves away from the other two and the shared region shrinks
Q3, L3, Z3 = 0.4, 4.0, 20.0
R3 = 0.5 + Q3 / 2.0
J3, K3 = np.array([1.4, 1.5, 2.0]), np.array([2.5, 1.5, 2.0])
I3_OLD, I3_NEW = np.array([1.95, 2.45, 2.0]), np.array([1.95, 2.55, 2.0])


def _triple_volume(a, b, c, m=20):
    """Volume common to three spheres of radius R3 about a, b, c: the fraction
    of 2^m scrambled Sobol points of the box around the common part that lie
    in all three."""
    from scipy.stats import qmc
    lo = np.maximum(np.maximum(a, b), c) - R3
    hi = np.minimum(np.minimum(a, b), c) + R3
    if np.any(hi <= lo):
        return 0.0
    x = qmc.Sobol(3, scramble=True, seed=5).random_base2(m) * (hi - lo) + lo
    inside = np.ones(len(x), dtype=bool)
    for centre in (a, b, c):
        inside &= ((x - centre) ** 2).sum(1) < R3 * R3
    return float(inside.mean() * np.prod(hi - lo))


@pytest.mark.parametrize("n_trial", [0, 3])
def test_detailed_balance_with_a_triple_overlap(oracle, n_trial):
    """P_acc(M->M')/P_acc(M'->M) = exp(z_p [V_f(M') - V_f(M)]) when three
    excluded spheres overlap: V_f = V - |union|, |union| = sum of spheres -
    sum of pair lenses + triple volume (exact lenses, the triple volume by
    quasi-Monte Carlo).  Without and with CB.  The pairwise prediction (the
    triple volume dropped) is rejected: the test sees the many-body term."""
    def lens3(x, y):
        return float(lens(np.linalg.norm(x - y), R3))
    d_pair = (lens3(I3_NEW, J3) + lens3(I3_NEW, K3)) - (lens3(I3_OLD, J3) + lens3(I3_OLD, K3))
    d_tri = _triple_volume(I3_OLD, J3, K3) - _triple_volume(I3_NEW, J3, K3)
    f, _ = oracle.acceptance(np.array([J3, K3, I3_OLD]), L3, 2, I3_NEW, q=Q3, n_r=Z3,
                             n_trial=n_trial, n_rep=150000)
    b, _ = oracle.acceptance(np.array([J3, K3, I3_NEW]), L3, 2, I3_OLD, q=Q3, n_r=Z3,
                             n_trial=n_trial, n_rep=150000, sweep0=10 ** 7)
    ratio = f / b
    se = ratio * math.sqrt(1.0 / f + 1.0 / b)
    expect = math.exp(Z3 * (d_pair + d_tri))
    assert abs(ratio - expect) < 4.0 * se, (ratio, expect, se)
    assert abs(ratio - math.exp(Z3 * d_pair)) > 6.0 * se, (ratio, math.exp(Z3 * d_pair), se)
