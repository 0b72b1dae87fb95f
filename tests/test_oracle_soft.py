"""Pins of the soft (Hertz) colloid-depletant interaction (Sec. VI remarks
that the scheme generalises to soft potentials such as the Hertz one).

Reading: a depletant at x blocks a move M -> M' with probability
b(x) = e^{-U_others(x)} max(0, e^{-u_old(x)} - e^{-u_new(x)}), so that
P(M->M') / P(M'->M) = exp(z_p Int [e^{-U'(x)} - e^{-U(x)}] dx), the ratio of
semigrand weights exp(z_p Int [e^{-U} - 1] dx).  What is fixed:
* the exponential the two sides share by specification: e^{-y} within a few
  ulp of the library's, exact at 0;
* detailed balance of a move against that integral, computed here by
  quadrature;
* the two-colloid distribution P(r) ~ r^2 exp(z_p I(r)),
  I(r) = Int (1 - e^{-u_a})(1 - e^{-u_b}) dx, by quadrature;
* the hard limit: a very stiff potential reproduces the hard acceptance.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from tests.test_oracle_physics import L2, Q, R_S, _pair

SIGMA = R_S          # contact distance colloid-depletant: (d + q) / 2


def _u(r, eps):
    r = np.asarray(r, dtype=float)
    t = np.clip(1.0 - r / SIGMA, 0.0, None)
    return eps * t ** 2.5


def test_exp_neg_matches_the_library(oracle):
    rng = np.random.default_rng(1)
    ys = np.concatenate([rng.uniform(0, 1, 4000), rng.uniform(0, 50, 4000),
                         rng.uniform(0, 699, 2000), [0.0, 1e-300, 0.5 * math.log(2), 1.0]])
    for y in ys:
        got, ref = oracle.exp_neg(y), math.exp(-y)
        assert abs(got - ref) <= 4.0 * math.ulp(ref), (y, got, ref)
    assert oracle.exp_neg(0.0) == 1.0
    assert oracle.exp_neg(701.0) == 0.0


def test_hertz_energy(oracle):
    eps = 3.0
    for r in (0.0, 0.1, 0.3, 0.59, 0.6, 0.7):
        assert oracle.hertz(eps, SIGMA, r * r) == pytest.approx(float(_u(r, eps)), rel=1e-13,
                                                               abs=1e-300)


def _delta_integral(r0, r1, eps):
    """Int [e^{-U'} - e^{-U}] dx for colloids a at 0 and b moving r0 -> r1 along
    x: = Int e^{-u_a} (e^{-u_b1} - e^{-u_b0}), axisymmetric quadrature."""
    def f(rho, x):
        ra = math.hypot(x, rho)
        g1 = math.exp(-_u(math.hypot(x - r1, rho), eps)) - math.exp(-_u(math.hypot(x - r0, rho), eps))
        return 2 * math.pi * rho * math.exp(-_u(ra, eps)) * g1
    lo, hi = min(r0, r1) - SIGMA, max(r0, r1) + SIGMA
    val, err = integrate.dblquad(f, lo, hi, 0.0, SIGMA, epsabs=1e-11, epsrel=1e-10)
    return val


@pytest.mark.parametrize("eps,z,r0,r1", [(2.0, 10.0, 1.05, 1.10), (300.0, 30.0, 1.02, 1.09),
                                         (300.0, 30.0, 1.10, 1.04)])
def test_soft_detailed_balance(oracle, eps, z, r0, r1):
    a, b0 = _pair(r0)
    _, b1 = _pair(r1)
    n_rep = 150000
    f, _ = oracle.acceptance(np.array([a, b0]), L2, 1, b1, q=Q, n_r=z, soft_eps=eps, n_rep=n_rep)
    b, _ = oracle.acceptance(np.array([a, b1]), L2, 1, b0, q=Q, n_r=z, soft_eps=eps,
                             n_rep=n_rep, sweep0=10 ** 7)
    expect = math.exp(z * _delta_integral(r0, r1, eps))
    ratio = f / b
    se = ratio * math.sqrt(1.0 / f + 1.0 / b)
    assert min(f, b) > 5000
    assert abs(ratio - expect) < 4.0 * se, (ratio, expect, se)


def _I(r, eps):
    def f(rho, x):
        ua = _u(math.hypot(x, rho), eps)
        ub = _u(math.hypot(x - r, rho), eps)
        return 2 * math.pi * rho * (1.0 - math.exp(-ua)) * (1.0 - math.exp(-ub))
    if r >= 2 * SIGMA:
        return 0.0
    val, _ = integrate.dblquad(f, r - SIGMA, SIGMA, 0.0, SIGMA, epsabs=1e-11, epsrel=1e-9)
    return val


def test_soft_pair_distribution(oracle):
    eps, z = 1000.0, 60.0
    bins, rmax, lo = 24, 1.2, 20
    edges = np.linspace(0.0, rmax, bins + 1)
    grid = np.linspace(1.0, 1.2, 41)
    Ig = np.array([_I(r, eps) for r in grid])
    expect = []
    for k in range(lo, bins):
        r = np.linspace(edges[k], edges[k + 1], 201)
        expect.append(np.trapezoid(r ** 2 * np.exp(z * np.interp(r, grid, Ig)), r))
    expect = np.array(expect) / np.sum(expect)
    a, b = _pair(1.5)
    hs = []
    for seed in range(1, 9):
        _, _, _, h = oracle.run(np.array([a, b]), L2, q=Q, n_r=z, soft_eps=eps, d_max=0.03,
                                seed=seed, n_sweeps=60000, hist_bins=bins, hist_rmax=rmax)
        h = h[lo:].astype(float)
        hs.append(h / h.sum())
    hs = np.array(hs)
    m, se = hs.mean(0), hs.std(0, ddof=1) / math.sqrt(len(hs))
    assert np.all(np.abs((m - expect) / se) < 4.0), (m, expect)
    # the test has power: the distribution without the depletion term is rejected
    r2 = np.array([edges[k + 1] ** 3 - edges[k] ** 3 for k in range(lo, bins)])
    r2 /= r2.sum()
    assert np.max(np.abs((m - r2) / se)) > 6.0


def test_stiff_limit_is_hard(oracle):
    """eps = 1e4: e^{-u} is 0 except in a shell of width ~1e-2 sigma at the
    contact distance, so the acceptance is the hard one within statistics."""
    a, b0 = _pair(1.05)
    _, b1 = _pair(1.10)
    n_rep = 100000
    z = 8.0
    fs, _ = oracle.acceptance(np.array([a, b0]), L2, 1, b1, q=Q, n_r=z, soft_eps=1e4, n_rep=n_rep)
    fh, _ = oracle.acceptance(np.array([a, b0]), L2, 1, b1, q=Q, n_r=z, n_rep=n_rep, sweep0=999)
    ps, ph = fs / n_rep, fh / n_rep
    assert abs(ps - ph) < 4.5 * math.sqrt(ps * (1 - ps) / n_rep + ph * (1 - ph) / n_rep) + 0.01


def test_soft_argument_validation(oracle):
    s = np.array([[0.5, 0.5, 0.5], [1.6, 0.5, 0.5]])
    with pytest.raises(ValueError):
        oracle.run(s, 3.0, q=0.2, n_r=1.0, soft_eps=1.0, n_trial=2)      # no CB
    with pytest.raises(ValueError):
        oracle.run(s, 3.0, q=0.2, n_r=1.0, soft_eps=1.0, v0_mode=1)     # not the shell
    with pytest.raises(ValueError):
        oracle.run(s, 3.0, q=0.2, n_r=1.0, soft_eps=-1.0)


def test_soft_with_the_cube_has_the_same_acceptance(oracle):
    """The cube V_0 holds the new circumsphere, so the soft acceptance
    probability is the circumsphere's (the blocking uniform is each
    attempt's fourth word in both)."""
    a, b0 = _pair(1.05)
    _, b1 = _pair(1.10)
    n_rep = 60000
    p = []
    for mode, sweep0 in ((0, 1), (2, 5 * 10 ** 6)):
        f, _ = oracle.acceptance(np.array([a, b0]), L2, 1, b1, q=Q, n_r=10.0, soft_eps=20.0,
                                 v0_mode=mode, n_rep=n_rep, sweep0=sweep0)
        p.append(f / n_rep)
    se = math.sqrt(sum(x * (1 - x) for x in p) / n_rep)
    assert 0.05 < p[0] < 0.95 and abs(p[0] - p[1]) < 4.5 * se, (p, se)
