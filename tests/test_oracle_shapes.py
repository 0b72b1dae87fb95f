"""Pins of the oracle's anisotropic shapes (Sec. V): hemispheres (Sec. V.A) and
the discoid, an oblate spheroid a = b = 0.5, c = 0.25 (Sec. V.B), with
quaternion rotation moves.

Each primitive is checked against something other than itself:

* depletant-colloid tests against the point-to-body distance found by a
  general constrained minimiser (scipy SLSQP on the convex body's own
  inequalities) and against closed forms on symmetry axes;
* colloid-colloid tests against separation distance / common-point depth
  found by the same minimiser, against touching distances along symmetry
  axes, and against the sphere test when a = c;
* the excluded volume of one colloid against the Steiner formula of integral
  geometry, V(K + rB) = V + S r + 2 pi wbar r^2 + 4/3 pi r^3 (wbar = mean width);
* the rotation proposal against its angle distribution, axis isotropy and
  symmetry;
* detailed balance of rotation moves against exp(z_p dV_f) with the free
  volume change measured by Monte Carlo on an explicit union-of-solids
  description of the excluded region;
* cell-list neighbours against brute force for whole anisotropic trajectories.
"""
import math

import numpy as np
import pytest

from paper_1508_07077_gb300 import workloads as W

optimize = pytest.importorskip("scipy.optimize")
Rotation = pytest.importorskip("scipy.spatial.transform").Rotation

HEMI, SPHD = 1, 2
HEMI_P = (1.0,)
SPHD_P = (0.5, 0.25)


def _rot(q):
    """scipy rotation of quaternion (s, x, y, z) (scipy stores x, y, z, w)."""
    return Rotation.from_quat([q[1], q[2], q[3], q[0]])


def _rand_quat(rng):
    v = rng.normal(size=4)
    return v / np.linalg.norm(v)


# body-frame inequality descriptions g_k(x) >= 0 (smooth, concave)
def _body_cons(shape, params):
    if shape == HEMI:
        R = 0.5 * params[0]
        return [lambda x: R * R - x @ x, lambda x: x[2]]
    a, c = params
    return [lambda x: 1.0 - (x[0] ** 2 + x[1] ** 2) / a ** 2 - x[2] ** 2 / c ** 2]


def _interior(shape, params):
    if shape == HEMI:
        return np.array([0.0, 0.0, 0.25 * params[0]])
    return np.zeros(3)


def _point_distance(shape, params, p):
    """min |x - p| over the body, body frame, by SLSQP."""
    cons = [{"type": "ineq", "fun": g} for g in _body_cons(shape, params)]
    best = None
    for x0 in (_interior(shape, params), 0.5 * _interior(shape, params)):
        r = optimize.minimize(lambda x: (x - p) @ (x - p), x0, jac=lambda x: 2 * (x - p),
                              constraints=cons, method="SLSQP",
                              options={"ftol": 1e-14, "maxiter": 500})
        # a feasible point bounds the distance from above; SLSQP may stop with
        # a line-search complaint at the optimum, so feasibility is the check
        if min(g(r.x) for g in _body_cons(shape, params)) > -1e-9:
            d = math.sqrt(max(r.fun, 0.0))
            best = d if best is None else min(best, d)
    return best


@pytest.mark.parametrize("shape,params", [(HEMI, HEMI_P), (SPHD, SPHD_P)])
def test_depletant_test_equals_minimised_distance(oracle, shape, params):
    rng = np.random.default_rng(11 + shape)
    q = 0.2
    r = q / 2
    R_s = 0.5 + r
    checked = 0
    for _ in range(500):
        v = rng.uniform(-R_s, R_s, 3)
        if v @ v >= R_s * R_s:
            continue
        quat = _rand_quat(rng)
        p = _rot(quat).inv().apply(v)          # body frame, independent rotation
        d = _point_distance(shape, params, p)
        assert d is not None
        if abs(d - r) < 1e-6:
            continue
        got = oracle.dep_overlap(v, q, shape=shape, shape_params=params, quat=quat)
        assert got == (d < r), (v, quat, d)
        checked += 1
    assert checked > 250


def test_depletant_closed_forms_on_axes(oracle):
    q, r = 0.1, 0.05
    eps = 1e-9
    # spheroid: along the symmetry axis dist = |z| - c, in the equator rho - a
    for z in (0.25 + r - eps, 0.25 + r + eps, -(0.25 + r) + eps):
        assert oracle.dep_overlap([0, 0, z], q, shape=SPHD, shape_params=SPHD_P) == \
            (abs(z) - 0.25 < r)
    for x in (0.5 + r - eps, 0.5 + r + eps):
        assert oracle.dep_overlap([x, 0, 0], q, shape=SPHD, shape_params=SPHD_P) == \
            (x - 0.5 < r)
    # hemisphere (flat face at z = 0, dome z >= 0): on the axis below the face
    # dist = -z, above it dist = z - R; below the rim dist = sqrt(dz^2 + dr^2)
    for z in (-r + eps, -r - eps, 0.5 + r - eps, 0.5 + r + eps):
        d = -z if z < 0 else z - 0.5
        assert oracle.dep_overlap([0, 0, z], q, shape=HEMI, shape_params=HEMI_P) == (d < r)
    s = r / math.sqrt(2.0)
    for k in (1 - 1e-7, 1 + 1e-7):
        v = [0.5 + s * k, 0.0, -s * k]
        assert oracle.dep_overlap(v, q, shape=HEMI, shape_params=HEMI_P) == (k < 1)
    # a rotated body: hemisphere turned so that its dome points along +x
    qy = [math.cos(math.pi / 4), 0.0, math.sin(math.pi / 4), 0.0]
    assert oracle.dep_overlap([0.5 + r - eps, 0, 0], q, shape=HEMI, shape_params=HEMI_P,
                              quat=qy)
    assert not oracle.dep_overlap([-r - eps, 0, 0], q, shape=HEMI, shape_params=HEMI_P,
                                  quat=qy)
    assert oracle.dep_overlap([-r + eps, 0, 0], q, shape=HEMI, shape_params=HEMI_P,
                              quat=qy)


def test_spheroid_with_equal_axes_is_a_sphere(oracle):
    rng = np.random.default_rng(5)
    q = 0.2
    for _ in range(2000):
        v = rng.uniform(-0.6, 0.6, 3)
        d = np.linalg.norm(v)
        if abs(d - 0.6) < 1e-9:
            continue
        assert oracle.dep_overlap(v, q, shape=SPHD, shape_params=(0.5, 0.5),
                                  quat=_rand_quat(rng)) == (d < 0.6)
    for _ in range(300):
        rr = rng.uniform(-1.0, 1.0, 3)
        d = np.linalg.norm(rr)
        if abs(d - 1.0) < 1e-9:
            continue
        got = oracle.pair_overlap(rr, shape=SPHD, shape_params=(0.5, 0.5),
                                  qa=_rand_quat(rng), qb=_rand_quat(rng))
        assert got == (d < 1.0), (rr, d)


def _pair_classify(shape, params, r, qa, qb):
    """+1 overlap, 0 separated, None undecided (within 1e-6 of contact), from
    two convex programs solved by SLSQP in the lab frame."""
    Ra, Rb = _rot(qa), _rot(qb)
    ga = _body_cons(shape, params)
    ca = Ra.apply(_interior(shape, params))
    cb = Rb.apply(_interior(shape, params)) + r

    def in_a(x):
        return Ra.inv().apply(x)

    def in_b(x):
        return Rb.inv().apply(x - r)

    # separation: min |x - y|, x in A, y in B
    cons = [{"type": "ineq", "fun": (lambda z, g=g: g(in_a(z[:3])))} for g in ga]
    cons += [{"type": "ineq", "fun": (lambda z, g=g: g(in_b(z[3:])))} for g in ga]
    res = optimize.minimize(lambda z: (z[:3] - z[3:]) @ (z[:3] - z[3:]),
                            np.concatenate([ca, cb]), constraints=cons, method="SLSQP",
                            options={"ftol": 1e-14, "maxiter": 800})
    sep = math.sqrt(max(res.fun, 0.0)) if res.success else None
    # depth: max t with every constraint of both bodies >= t at one point x
    cons = [{"type": "ineq", "fun": (lambda z, g=g: g(in_a(z[:3])) - z[3])} for g in ga]
    cons += [{"type": "ineq", "fun": (lambda z, g=g: g(in_b(z[:3])) - z[3])} for g in ga]
    x0 = 0.5 * (ca + cb)
    t0 = min(min(g(in_a(x0)) for g in ga), min(g(in_b(x0)) for g in ga)) - 0.1
    res2 = optimize.minimize(lambda z: -z[3], np.concatenate([x0, [t0]]), constraints=cons,
                             method="SLSQP", options={"ftol": 1e-14, "maxiter": 800})
    depth = -res2.fun
    feasible = all(c["fun"](res2.x) >= -1e-12 for c in cons)
    # a feasible point of depth t > 0 proves an overlap; a separation needs
    # both programs to agree (each alone only bounds its optimum from one side)
    if feasible and depth > 1e-6:
        return 1
    if sep is not None and sep > 1e-6 and depth < -1e-6:
        return 0
    return None


@pytest.mark.parametrize("shape,params", [(HEMI, HEMI_P), (SPHD, SPHD_P)])
def test_pair_test_equals_convex_programs(oracle, shape, params):
    rng = np.random.default_rng(21 + shape)
    seen = {0: 0, 1: 0}
    for _ in range(240):
        r = rng.uniform(-1.0, 1.0, 3)
        if r @ r >= 1.0:
            continue
        qa, qb = _rand_quat(rng), _rand_quat(rng)
        want = _pair_classify(shape, params, r, qa, qb)
        if want is None:
            continue
        got = oracle.pair_overlap(r, shape=shape, shape_params=params, qa=qa, qb=qb)
        assert int(got) == want, (r, qa, qb)
        seen[want] += 1
    assert seen[0] > 20 and seen[1] > 20, seen


def _qaxis(ax, ang):
    ax = np.asarray(ax, dtype=float)
    ax = ax / np.linalg.norm(ax)
    return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * ax])


def _qmul(a, b):
    s1, v1, s2, v2 = a[0], a[1:], b[0], b[1:]
    return np.concatenate([[s1 * s2 - v1 @ v2], s1 * v2 + s2 * v1 + np.cross(v1, v2)])


def test_pair_test_near_parallel_flat_faces(oracle):
    """Hemispheres face to face, faces nearly parallel, gaps and overlaps from
    1e-7 to 1e-2: the flat faces make the difference body partly flat, the
    hardest case for the portal method."""
    rng = np.random.default_rng(1)
    flip = np.array([0.0, 1.0, 0.0, 0.0])
    seen = {0: 0, 1: 0}
    for _ in range(200):
        qa = _qmul(_qaxis(rng.normal(size=3), 10 ** rng.uniform(-6, -1)), flip)
        qb = _qaxis(rng.normal(size=3), 10 ** rng.uniform(-6, -1))
        lat = rng.uniform(-0.9, 0.9, 2)
        r = np.array([lat[0], lat[1], rng.choice([-1, 1]) * 10 ** rng.uniform(-7, -2)])
        if r @ r >= 1.0:
            continue
        want = _pair_classify(HEMI, HEMI_P, r, qa, qb)
        if want is None:
            continue
        assert int(oracle.pair_overlap(r, shape=HEMI, shape_params=HEMI_P, qa=qa, qb=qb)) == want
        seen[want] += 1
    assert seen[0] > 10 and seen[1] > 10, seen


def test_pair_touching_distances_along_axes(oracle):
    e = 1e-9
    up = [1.0, 0.0, 0.0, 0.0]
    flip = [0.0, 1.0, 0.0, 0.0]                  # 180 deg about x: dome toward -z
    rx = [math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0, 0.0]   # body z -> lab -y
    R = 0.5

    def hemi(r, qa, qb):
        return oracle.pair_overlap(r, shape=HEMI, shape_params=HEMI_P, qa=qa, qb=qb)

    def sphd(r, qa, qb):
        return oracle.pair_overlap(r, shape=SPHD, shape_params=SPHD_P, qa=qa, qb=qb)

    # stacked, same orientation: B's face at s meets A's dome tip at R
    assert hemi([0, 0, R - e], up, up) and not hemi([0, 0, R + e], up, up)
    assert hemi([0, 0, -R + e], up, up) and not hemi([0, 0, -R - e], up, up)
    # dome to dome: tips meet at s = 2R
    assert hemi([0, 0, 2 * R - e], up, flip) and not hemi([0, 0, 2 * R + e], up, flip)
    # face to face (A's dome down, B's dome up): faces touch at s = 0
    assert hemi([0, 0, -e], flip, up) and not hemi([0, 0, e], flip, up)
    assert hemi([0.3, 0.2, -e], flip, up) and not hemi([0.3, 0.2, e], flip, up)
    # side by side
    assert hemi([2 * R - e, 0, 0], up, up) and not hemi([2 * R + e, 0, 0], up, up)
    # discoids: stacked along the axis, side by side, crossed
    assert sphd([0, 0, 0.5 - e], up, up) and not sphd([0, 0, 0.5 + e], up, up)
    assert sphd([1.0 - e, 0, 0], up, up) and not sphd([1.0 + e, 0, 0], up, up)
    assert sphd([0, 0.75 - e, 0], up, rx) and not sphd([0, 0.75 + e, 0], up, rx)
    assert sphd([1.0 - e, 0, 0], up, rx) and not sphd([1.0 + e, 0, 0], up, rx)


def _mean_width_spheroid(a, c):
    from scipy.integrate import quad
    val, _ = quad(lambda t: math.sqrt(a * a * (1 - t * t) + c * c * t * t), 0.0, 1.0,
                  epsabs=1e-13)
    return 2.0 * val


@pytest.mark.parametrize("shape", [HEMI, SPHD])
def test_single_colloid_excluded_volume_steiner(oracle, shape):
    q = 0.2
    r = q / 2
    if shape == HEMI:
        R = 0.5
        V, S, wbar = 2 / 3 * math.pi * R ** 3, 3 * math.pi * R ** 2, R * (1 + math.pi / 4)
        params = HEMI_P
    else:
        a, c = SPHD_P
        e = math.sqrt(1 - c * c / (a * a))
        V = 4 / 3 * math.pi * a * a * c
        S = 2 * math.pi * a * a * (1 + (1 - e * e) / e * math.atanh(e))
        wbar = _mean_width_spheroid(a, c)
        params = SPHD_P
    v_excl = V + S * r + 2 * math.pi * wbar * r * r + 4 / 3 * math.pi * r ** 3
    L, n_probe = 1.6, 1000000
    quat = _rand_quat(np.random.default_rng(3))
    alpha = oracle.free_volume(np.array([[0.3, 1.1, 0.7]]), L, q, shape=shape,
                               shape_params=params, quat=quat[None, :], n_probe=n_probe)
    exact = 1.0 - v_excl / L ** 3
    assert abs(alpha - exact) < 4.0 * math.sqrt(exact * (1 - exact) / n_probe), (alpha, exact)


def test_rotation_proposal_distribution(oracle):
    a_max, n = 0.4, 20000
    alpha = math.tan(a_max / 2)
    ident = np.array([1.0, 0.0, 0.0, 0.0])
    qs = np.array([oracle.rotation_proposal(ident, a_max, tag=t) for t in range(n)])
    assert np.all(np.abs(np.linalg.norm(qs, axis=1) - 1.0) < 4e-16)
    vec = qs[:, 1:]
    sv = np.linalg.norm(vec, axis=1)
    theta = 2.0 * np.arctan2(sv, qs[:, 0])
    assert theta.max() <= a_max + 1e-12
    # P(theta <= x) = (tan(x/2)/alpha)^3 for v uniform in the unit ball
    from scipy import stats
    ks = stats.kstest(theta, lambda x: np.clip(np.tan(x / 2) / alpha, 0, 1) ** 3)
    assert ks.pvalue > 1e-4, ks
    axis = vec / sv[:, None]
    assert np.all(np.abs(axis.mean(0)) < 4.0 / math.sqrt(3 * n))
    m2 = axis.T @ axis / n
    assert np.all(np.abs(m2 - np.eye(3) / 3) < 0.02)
    # q' = q_r q: the left factor does not depend on q
    rng = np.random.default_rng(2)
    for t in range(50):
        q = _rand_quat(rng)
        qn = oracle.rotation_proposal(q, a_max, tag=t)
        left = (_rot(qn) * _rot(q).inv()).as_quat()
        ref = _rot(qs[t]).as_quat()
        assert min(np.abs(left - ref).max(), np.abs(left + ref).max()) < 1e-14


def _hemi_excluded(p, x, quat, R, r):
    """Points p (n x 3) in the excluded region of a hemisphere at x: union of
    the dome ball cap, the slab under the face and the tube around the rim."""
    b = _rot(quat).inv().apply(p - x)
    rho = np.hypot(b[:, 0], b[:, 1])
    dome = (b[:, 2] >= 0) & (np.einsum("ij,ij->i", b, b) < (R + r) ** 2)
    slab = (b[:, 2] < 0) & (b[:, 2] > -r) & (rho <= R)
    tube = (b[:, 2] < 0) & ((rho - R) ** 2 + b[:, 2] ** 2 < r * r)
    return dome | slab | tube


@pytest.mark.parametrize("n_trial", [0, 3])
def test_detailed_balance_of_rotation_moves(oracle, n_trial):
    R, q = 0.5, 0.2
    r = q / 2
    z = 70.0
    L = 4.0
    x0 = np.array([1.0, 1.0, 1.0])
    x1 = x0 + np.array([0.95, 0.0, 0.1])
    q1 = np.array([math.cos(5 * math.pi / 12), 0.0, math.sin(5 * math.pi / 12), 0.0])
    qa = np.array([1.0, 0.0, 0.0, 0.0])
    qb = np.array([math.cos(0.1), 0.0, math.sin(0.1), 0.0])     # 0.2 rad about y
    pos = np.array([x0, x1])
    for qq in (qa, qb):
        assert not oracle.pair_overlap(x1 - x0, shape=HEMI, shape_params=HEMI_P, qa=qq, qb=q1)
    # intersection volumes |X_a n X_1| and |X_b n X_1| by Monte Carlo in the
    # ball of radius R + r around colloid 0 (which holds X_a and X_b)
    rng = np.random.default_rng(9)
    m = 3000000
    pts = rng.uniform(-(R + r), R + r, size=(m, 3))
    pts = pts[np.einsum("ij,ij->i", pts, pts) < (R + r) ** 2] + x0
    vball = 4 / 3 * math.pi * (R + r) ** 3
    in1 = _hemi_excluded(pts, x1, q1, R, r)
    fa = np.mean(in1 & _hemi_excluded(pts, x0, qa, R, r))
    fb = np.mean(in1 & _hemi_excluded(pts, x0, qb, R, r))
    dv = vball * (fb - fa)
    dv_se = vball * math.sqrt((fa + fb) / len(pts))
    n_rep = 300000
    f, _ = oracle.acceptance(pos, L, 0, x0, shape=HEMI, shape_params=HEMI_P, q=q, n_r=z,
                             n_trial=n_trial, quat=np.array([qa, q1]), qn=qb, n_rep=n_rep)
    b, _ = oracle.acceptance(pos, L, 0, x0, shape=HEMI, shape_params=HEMI_P, q=q, n_r=z,
                             n_trial=n_trial, quat=np.array([qb, q1]), qn=qa, n_rep=n_rep,
                             sweep0=10 ** 7)
    ratio = f / b
    se = ratio * math.sqrt(1.0 / f + 1.0 / b)
    expect = math.exp(z * dv)
    assert abs(dv) * z > 0.1                     # the test has something to detect
    assert abs(ratio - expect) < 4.0 * math.hypot(se, expect * z * dv_se), (ratio, expect)


@pytest.mark.parametrize("shape", [HEMI, SPHD])
def test_anisotropic_cell_list_equals_brute_force(oracle, shape):
    params = HEMI_P if shape == HEMI else SPHD_P
    n, phi, q = 108, 0.25, 0.1
    L = W.box_length(n, phi, shape)
    pos = W.fcc_positions(n, L, seed=4)
    quat = W.random_quaternions(n, seed=4)
    kw = dict(shape=shape, shape_params=params, q=q, n_r=W.fugacity(0.2, q), d_max=0.08,
              a_max=0.3, p_translate=0.5, quat=quat, n_sweeps=4, seed=3)
    pa, qa_, ca, _ = oracle.run(pos, L, **kw)
    pb, qb_, cb, _ = oracle.run(pos, L, brute_force=True, **kw)
    assert np.array_equal(pa, pb) and np.array_equal(qa_, qb_)
    assert ca == cb
    assert ca["accept"] > 0 and ca["translate"] < ca["moves"]
    # the final configuration is free of overlaps
    for i in range(n):
        for j in range(i + 1, n):
            d = pb[j] - pb[i]
            d -= L * np.round(d / L)
            assert not oracle.pair_overlap(d, shape=shape, shape_params=params,
                                           qa=qb_[i], qb=qb_[j])
