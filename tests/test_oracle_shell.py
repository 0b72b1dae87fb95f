"""Pins of the alternative depletant regions V_0 (Sec. III.C: any convenient
region that contains every point overlapping the new configuration but not
the old one).

Shell (closing remark of Sec. III.C): for a translated sphere, depletants may
be sampled in the shell of the moved colloid's excluded volume that can hold
points overlapping the new pose but not the old one, instead of in the whole
circumsphere.  Cube: the axis-aligned cube around the circumsphere, sampled
with no rejection (every attempt is a depletant), for every shape.

What mathematics fixes, and what is checked here:
* geometry: a point within R_s of the new centre and at least R_s from the
  old one lies at distance >= R_s - |D| from the new centre, so every lens
  point is in the shell of a level whose thickness exceeds |D|; the level a
  move's words select always has that property, and is the thinnest one up
  to the rounding of the integer rule;
* the generator: points uniform in the shell (radial CDF (r^3 - R_in^3) /
  (R_s^3 - R_in^3), isotropic directions) at the acceptance rate the
  thinning step implies, (pi/6) (1 + rho + rho^2) / 3 with rho = R_in / R_s;
* N_p ~ Poisson(z_p |shell|);
* the acceptance probability of every move is the circumsphere's (the
  blocking depletants form the same Poisson process on the lens), so
  detailed balance (Eqs. 5-11, 12) and the Asakura-Oosawa pair distribution
  hold unchanged.
"""
import math

import numpy as np
import pytest

from tests.test_oracle_physics import L2, Q, R_S, Z_P, _pair, lens

K = 32


def _s11(w):
    return (np.asarray(w, dtype=np.float64) + 0.5) / 2.0 ** 31 - 1.0


def _levels(oracle, words):
    return np.array([oracle.shell_level(*w) for w in words])


def test_level_holds_the_lens_and_is_thinnest(oracle):
    d_max = 0.1
    dd = math.sqrt(3.0) * d_max / K
    rng = np.random.default_rng(11)
    words = rng.integers(0, 2 ** 32, size=(20000, 3), dtype=np.uint64).astype(np.uint32)
    # corners and the centre of the displacement cube
    words = np.vstack([words, [[0, 0, 0], [2 ** 32 - 1] * 3, [2 ** 31] * 3,
                               [2 ** 31 - 1, 2 ** 31, 2 ** 31 - 1], [0, 2 ** 32 - 1, 0]]])
    k = _levels(oracle, words.astype(np.uint32))
    D = np.linalg.norm(d_max * _s11(words), axis=1)
    assert k.min() >= 1 and k.max() <= K
    assert np.all(D < k * dd)                                      # holds the lens
    assert np.all((k - 1) * dd < D + math.sqrt(3.0) * d_max * 2.0 ** -16)  # thinnest
    assert k[-5] == K and k[-4] == K and k[-3] == 1 and k[-2] == 1
    # the level histogram follows |D| for D uniform in the cube
    assert abs(np.mean(k) - np.mean(np.ceil(D[:-5] / dd))) < 0.01


def test_lens_points_lie_in_the_shell(oracle):
    """Brute force: uniform points of the new circumsphere that overlap the
    new pose and not the old one all lie at >= R_s - k dd from the centre,
    and the closest possible lens point, R_s - |D| along D, does too."""
    d_max = 0.1
    dd = math.sqrt(3.0) * d_max / K
    rng = np.random.default_rng(12)
    for _ in range(40):
        w = rng.integers(0, 2 ** 32, size=3, dtype=np.uint64).astype(np.uint32)
        k = oracle.shell_level(*w)
        D = d_max * _s11(w)
        o = -D                                   # old centre relative to the new one
        e = rng.uniform(-R_S, R_S, size=(200000, 3))
        r = np.linalg.norm(e, axis=1)
        in_lens = (r < R_S) & (np.linalg.norm(e - o, axis=1) >= R_S)
        R_in = R_S - k * dd
        assert np.all(r[in_lens] >= R_in)
        nearest = R_S - np.linalg.norm(D)
        assert nearest > R_in


@pytest.mark.parametrize("d_max,lvl", [(0.1, 1), (0.1, 12), (0.1, 32), (0.35, 32)])
def test_shell_points_are_uniform_in_the_shell(oracle, d_max, lvl):
    n_att = 200000
    e = oracle.shell_points(R_S, d_max, lvl, n_att, seed=3, sweep=5, tag=7)
    dd = math.sqrt(3.0) * d_max / K
    R_in = max(0.0, R_S - (lvl * dd + 1e-9 * R_S))
    rho = R_in / R_S
    r = np.linalg.norm(e, axis=1)
    assert r.min() >= R_in * (1 - 1e-12) and r.max() < R_S
    # acceptance rate of the thinning step
    p = math.pi / 6.0 * (1.0 + rho + rho * rho) / 3.0
    se = math.sqrt(p * (1 - p) / n_att)
    assert abs(len(e) / n_att - p) < 4.5 * se, (len(e) / n_att, p)
    # radial CDF: (r^3 - R_in^3) / (R_s^3 - R_in^3) is uniform (KS)
    u = np.sort((r ** 3 - R_in ** 3) / (R_S ** 3 - R_in ** 3))
    n = len(u)
    ks = max(np.max(np.arange(1, n + 1) / n - u), np.max(u - np.arange(n) / n))
    assert ks < 1.63 / math.sqrt(n), ks            # 1% critical value
    # isotropy: mean direction ~ 0, second moments ~ I/3
    nhat = e / r[:, None]
    assert np.all(np.abs(nhat.mean(0)) < 4.5 * math.sqrt(1.0 / 3.0 / n))
    m2 = nhat.T @ nhat / n
    assert np.allclose(m2, np.eye(3) / 3.0, atol=4.5 * math.sqrt(4.0 / 45.0 / n))


def _move(r0, r1):
    a, b0 = _pair(r0)
    _, b1 = _pair(r1)
    return np.array([a, b0]), b1


@pytest.mark.parametrize("r0,r1", [(1.05, 1.10), (1.10, 1.03)])
def test_shell_draws_poisson_of_the_shell_volume(oracle, r0, r1):
    pos, xn = _move(r0, r1)
    d_max = 0.05
    dd = math.sqrt(3.0) * d_max / K
    n_rep = 40000
    _, c = oracle.acceptance(pos, L2, 1, xn, q=Q, n_r=Z_P, v0_mode=1, d_max=d_max,
                             n_rep=n_rep)
    delta = abs(r1 - r0)
    k = math.ceil(delta / dd)
    R_in = R_S - k * dd
    lam = Z_P * 4.0 * math.pi / 3.0 * (R_S ** 3 - R_in ** 3)
    mean = c["dep_drawn"] / n_rep
    assert abs(mean - lam) < 4.5 * math.sqrt(lam / n_rep), (mean, lam)
    # far fewer than the circumsphere's z_p (4 pi / 3) R_s^3
    assert lam < 0.5 * Z_P * 4.0 * math.pi / 3.0 * R_S ** 3


@pytest.mark.parametrize("n_trial", [0, 3])
def test_acceptance_equals_the_circumsphere(oracle, n_trial):
    """Same configuration and move, independent streams: the acceptance
    probabilities and the mean number of blocking depletants agree."""
    rng = np.random.default_rng(5)
    pos = np.array([[1.2, 1.2, 1.2], [2.25, 1.2, 1.2], [1.2, 2.27, 1.25],
                    [0.2, 1.0, 1.3], [1.3, 0.15, 1.9]])
    L = 3.2
    xn = pos[0] + np.array([0.04, 0.03, -0.02])
    n_rep = 60000
    res = []
    for mode in (0, 1):
        a, c = oracle.acceptance(pos, L, 0, xn, q=Q, n_r=Z_P, n_trial=n_trial, v0_mode=mode,
                                 d_max=0.05, n_rep=n_rep, sweep0=int(rng.integers(1 << 20)))
        res.append((a / n_rep, c))
    (p0, c0), (p1, c1) = res
    se = math.sqrt(p0 * (1 - p0) / n_rep + p1 * (1 - p1) / n_rep)
    assert 0.05 < p0 < 0.95
    assert abs(p0 - p1) < 4.5 * se, (p0, p1, se)
    assert c1["dep_drawn"] < 0.5 * c0["dep_drawn"]
    if n_trial > 0:
        b0, b1 = c0["dep_blocking"] / n_rep, c1["dep_blocking"] / n_rep
        assert abs(b0 - b1) < 4.5 * math.sqrt((b0 + b1) / n_rep), (b0, b1)


@pytest.mark.parametrize("n_trial", [0, 3])
@pytest.mark.parametrize("r0,r1", [(1.05, 1.10), (1.02, 1.09)])
def test_detailed_balance_with_the_shell(oracle, n_trial, r0, r1):
    pos0, x1 = _move(r0, r1)
    pos1, x0 = _move(r1, r0)
    kw = dict(q=Q, n_r=Z_P, n_trial=n_trial, v0_mode=1, d_max=0.05, n_rep=150000)
    f, _ = oracle.acceptance(pos0, L2, 1, x1, **kw)
    b, _ = oracle.acceptance(pos1, L2, 1, x0, sweep0=10 ** 7, **kw)
    ratio = f / b
    se = ratio * math.sqrt(1.0 / f + 1.0 / b)
    expect = math.exp(Z_P * float(lens(r1) - lens(r0)))
    assert abs(ratio - expect) < 4.0 * se, (ratio, expect, se)


def test_asakura_oosawa_pair_distribution_with_the_shell(oracle):
    """The full sampler (cell list, level from the move words, shell tables)
    reproduces P(r) ~ r^2 exp(z_p V_lens(r)) of two depletion-attracting
    spheres, and draws fewer depletants than with the circumsphere."""
    bins, rmax, lo = 24, 1.2, 20
    edges = np.linspace(0.0, rmax, bins + 1)
    expect = []
    for b in range(lo, bins):
        r = np.linspace(edges[b], edges[b + 1], 401)
        expect.append(np.trapezoid(r ** 2 * np.exp(Z_P * lens(r)), r))
    expect = np.array(expect) / np.sum(expect)
    a, b = _pair(1.5)
    hs, drawn = [], [0, 0]
    for seed in range(1, 9):
        _, _, c, h = oracle.run(np.array([a, b]), L2, q=Q, n_r=Z_P, v0_mode=1, d_max=0.03,
                                seed=seed, n_sweeps=60000, hist_bins=bins, hist_rmax=rmax)
        h = h[lo:].astype(float)
        hs.append(h / h.sum())
        drawn[1] += c["dep_drawn"]
        if seed == 1:
            _, _, c0, _ = oracle.run(np.array([a, b]), L2, q=Q, n_r=Z_P, d_max=0.03,
                                     seed=seed, n_sweeps=60000)
            drawn[0] = c0["dep_drawn"]
    hs = np.array(hs)
    m, se = hs.mean(0), hs.std(0, ddof=1) / math.sqrt(len(hs))
    z = (m - expect) / se
    assert np.all(np.abs(z) < 4.0), z
    assert drawn[1] / 8 < 0.5 * drawn[0]


def test_shell_argument_validation(oracle):
    s = np.array([[0.5, 0.5, 0.5], [1.6, 0.5, 0.5]])
    with pytest.raises(ValueError):   # shells are for spheres only
        oracle.run(s, 3.0, shape=oracle.SHAPE_HEMISPHERE, shape_params=(1.0,),
                   quat=np.tile([1.0, 0, 0, 0], (2, 1)), q=0.2, n_r=1.0, v0_mode=1)
    with pytest.raises(ValueError):
        oracle.run(s, 3.0, q=0.2, n_r=1.0, v0_mode=3)
    with pytest.raises(ValueError):   # move longer than the largest level
        oracle.acceptance(s, 3.0, 1, s[1] + 0.2, q=0.2, n_r=1.0, v0_mode=1, d_max=0.05)
    with pytest.raises(ValueError):
        oracle.shell_points(0.6, 0.1, 33, 10)


# --------------------------------------------------------------------------
# cube V_0
# --------------------------------------------------------------------------

def test_cube_draws_poisson_of_the_cube_volume(oracle):
    pos, xn = _move(1.05, 1.10)
    n_rep = 40000
    _, c = oracle.acceptance(pos, L2, 1, xn, q=Q, n_r=Z_P, v0_mode=2, n_rep=n_rep)
    lam = Z_P * (2.0 * R_S) ** 3
    mean = c["dep_drawn"] / n_rep
    assert abs(mean - lam) < 4.5 * math.sqrt(lam / n_rep), (mean, lam)
    assert abs(oracle.lib().oracle_cube_lambda(R_S, Z_P) - lam) < 1e-9 * lam


@pytest.mark.parametrize("n_trial", [0, 3])
def test_cube_acceptance_equals_the_circumsphere(oracle, n_trial):
    pos = np.array([[1.2, 1.2, 1.2], [2.25, 1.2, 1.2], [1.2, 2.27, 1.25],
                    [0.2, 1.0, 1.3], [1.3, 0.15, 1.9]])
    xn = pos[0] + np.array([0.04, 0.03, -0.02])
    n_rep = 60000
    p = []
    for mode, sweep0 in ((0, 11), (2, 77777)):
        a, _ = oracle.acceptance(pos, 3.2, 0, xn, q=Q, n_r=Z_P, n_trial=n_trial, v0_mode=mode,
                                 n_rep=n_rep, sweep0=sweep0)
        p.append(a / n_rep)
    se = math.sqrt(sum(x * (1 - x) for x in p) / n_rep)
    assert 0.05 < p[0] < 0.95 and abs(p[0] - p[1]) < 4.5 * se, (p, se)


def test_cube_acceptance_of_a_rotation_equals_the_circumsphere(oracle):
    """Anisotropic colloids: a fixed rotation of a hemisphere next to another."""
    shape, params = oracle.SHAPE_HEMISPHERE, (1.0,)
    pos = np.array([[1.5, 1.5, 1.5], [1.5, 1.5, 2.55]])
    quat = np.array([[1.0, 0.0, 0.0, 0.0], [0.0, 1.0, 0.0, 0.0]])
    th = 0.15
    qn = np.array([math.cos(th / 2), math.sin(th / 2), 0.0, 0.0])
    n_rep = 40000
    p = []
    for mode, sweep0 in ((0, 5), (2, 99999)):
        a, _ = oracle.acceptance(pos, 3.5, 0, pos[0], shape=shape, shape_params=params, q=0.1,
                                 n_r=40.0, v0_mode=mode, quat=quat, qn=qn, n_rep=n_rep,
                                 sweep0=sweep0)
        p.append(a / n_rep)
    se = math.sqrt(sum(x * (1 - x) for x in p) / n_rep)
    assert 0.05 < p[0] < 0.95 and abs(p[0] - p[1]) < 4.5 * se, (p, se)


@pytest.mark.parametrize("n_trial", [0, 3])
def test_detailed_balance_with_the_cube(oracle, n_trial):
    pos0, x1 = _move(1.02, 1.09)
    pos1, x0 = _move(1.09, 1.02)
    kw = dict(q=Q, n_r=Z_P, n_trial=n_trial, v0_mode=2, n_rep=150000)
    f, _ = oracle.acceptance(pos0, L2, 1, x1, **kw)
    b, _ = oracle.acceptance(pos1, L2, 1, x0, sweep0=10 ** 7, **kw)
    ratio = f / b
    se = ratio * math.sqrt(1.0 / f + 1.0 / b)
    expect = math.exp(Z_P * float(lens(1.09) - lens(1.02)))
    assert abs(ratio - expect) < 4.0 * se, (ratio, expect, se)


def test_asakura_oosawa_pair_distribution_with_the_cube(oracle):
    bins, rmax, lo = 24, 1.2, 20
    edges = np.linspace(0.0, rmax, bins + 1)
    expect = []
    for b in range(lo, bins):
        r = np.linspace(edges[b], edges[b + 1], 401)
        expect.append(np.trapezoid(r ** 2 * np.exp(Z_P * lens(r)), r))
    expect = np.array(expect) / np.sum(expect)
    a, b = _pair(1.5)
    hs = []
    for seed in range(1, 9):
        _, _, c, h = oracle.run(np.array([a, b]), L2, q=Q, n_r=Z_P, v0_mode=2, d_max=0.03,
                                seed=seed, n_sweeps=40000, hist_bins=bins, hist_rmax=rmax)
        h = h[lo:].astype(float)
        hs.append(h / h.sum())
        assert c["dep_evaluated"] <= c["dep_drawn"]
    hs = np.array(hs)
    m, se = hs.mean(0), hs.std(0, ddof=1) / math.sqrt(len(hs))
    assert np.all(np.abs((m - expect) / se) < 4.0)
