"""Python access to the CPU oracle (``oracle/hpmc_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product path (``paper_1508_07077_gb300``) never imports this module.

The oracle is a plain serial FP64 C program compiled with ``-ffp-contract=off``
so that every floating-point expression is evaluated exactly in the order the
specification fixes.  See ``hpmc_oracle.c`` for the paper sections it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hpmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SHAPE_SPHERE, SHAPE_HEMISPHERE, SHAPE_SPHEROID = 0, 1, 2
V0_CIRCUMSPHERE, V0_SHELL, V0_CUBE = 0, 1, 2

# counter slots of oracle_run
COUNTERS = ("moves", "accept", "reject_cell", "reject_overlap", "reject_depletant",
            "reject_cb", "dep_drawn", "dep_blocking", "cb_fwd_ok", "cb_rev_ok",
            "cap_hits", "translate", "dep_evaluated")
N_COUNTERS = 16
# counters that are a pure function of the trajectory (identical on any
# correct implementation of the specification)
PARITY_COUNTERS = ("moves", "accept", "reject_cell", "reject_overlap",
                   "reject_depletant", "reject_cb", "dep_drawn", "translate",
                   "dep_evaluated")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2,
    -ffp-contract=off, no -march so the result is the same on x86 and Arm)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.oracle_philox4x32_10.restype = None
            for name in ("oracle_u01", "oracle_s11"):
                getattr(L, name).argtypes = [ctypes.c_uint32]
                getattr(L, name).restype = ctypes.c_double
            L.oracle_u53.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.oracle_u53.restype = ctypes.c_double
            L.oracle_lambda.argtypes = [ctypes.c_double, ctypes.c_double]
            L.oracle_lambda.restype = ctypes.c_double
            L.oracle_poisson_table.argtypes = [ctypes.c_double, dp, ctypes.c_int]
            L.oracle_poisson_table.restype = ctypes.c_int
            L.oracle_schedule.argtypes = [ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.c_uint32, ctypes.c_double, dp, ip]
            L.oracle_schedule.restype = None
            L.oracle_cell_list.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                           dp, ctypes.c_uint64, ctypes.c_uint32,
                                           ctypes.c_uint32, ip, ip]
            L.oracle_cell_list.restype = ctypes.c_int
            L.oracle_auto_cells.argtypes = [ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double]
            L.oracle_auto_cells.restype = ctypes.c_int
            L.oracle_run.argtypes = [
                ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, ctypes.c_int,
                ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                dp, dp, ctypes.c_uint64, ctypes.c_int, u64p,
                ctypes.c_int, ctypes.c_double, u64p]
            L.oracle_run.restype = ctypes.c_int
            L.oracle_run_threads.argtypes = L.oracle_run.argtypes + [ctypes.c_int]
            L.oracle_run_threads.restype = ctypes.c_int
            L.oracle_poisson_sample.argtypes = [dp, ctypes.c_int, ctypes.c_double]
            L.oracle_poisson_sample.restype = ctypes.c_int
            L.oracle_acceptance.argtypes = [
                ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, ctypes.c_int,
                ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, dp, dp, ctypes.c_int, dp, dp, ctypes.c_uint64,
                ctypes.c_long, u64p]
            L.oracle_acceptance.restype = ctypes.c_long
            L.oracle_free_volume.argtypes = [
                ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, ctypes.c_double,
                dp, dp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_long]
            L.oracle_free_volume.restype = ctypes.c_long
            L.oracle_dep_overlap.argtypes = [ctypes.c_int, dp, ctypes.c_int,
                                             ctypes.c_double, dp, dp]
            L.oracle_dep_overlap.restype = ctypes.c_int
            L.oracle_pair_overlap.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, dp, dp]
            L.oracle_pair_overlap.restype = ctypes.c_int
            L.oracle_rotation_proposal.argtypes = [ctypes.c_uint64, ctypes.c_uint32,
                                                   ctypes.c_uint32, ctypes.c_uint32,
                                                   ctypes.c_double, dp, dp]
            L.oracle_rotation_proposal.restype = ctypes.c_int
            L.oracle_shell_level.argtypes = [u32p]
            L.oracle_shell_level.restype = ctypes.c_int
            L.oracle_s21.argtypes = [ctypes.c_uint32]
            L.oracle_s21.restype = ctypes.c_double
            L.oracle_paired_points.argtypes = [ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_uint32, ctypes.c_uint32, dp]
            L.oracle_paired_points.restype = None
            L.oracle_shell_lambda.argtypes = [ctypes.c_double] * 3
            L.oracle_shell_lambda.restype = ctypes.c_double
            L.oracle_shell_points.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                              ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_uint32, dp]
            L.oracle_shell_points.restype = ctypes.c_long
            L.oracle_cube_lambda.argtypes = [ctypes.c_double, ctypes.c_double]
            L.oracle_cube_lambda.restype = ctypes.c_double
            ip = ctypes.POINTER(ctypes.c_int)
            L.oracle_gibbs_run.argtypes = [
                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ip, dp, dp,
                ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                u64p, u64p]
            L.oracle_gibbs_run.restype = ctypes.c_int
            L.oracle_gibbs_acceptance.argtypes = [
                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int, dp,
                ctypes.c_uint64, ctypes.c_long, u64p]
            L.oracle_gibbs_acceptance.restype = ctypes.c_long
            L.oracle_exp_neg.argtypes = [ctypes.c_double]
            L.oracle_exp_neg.restype = ctypes.c_double
            L.oracle_hertz.argtypes = [ctypes.c_double] * 3
            L.oracle_hertz.restype = ctypes.c_double
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def philox(ctr, key):
    """Philox4x32-10 of one counter (4 x u32) under one key (2 x u32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32),
                               _p(out, ctypes.c_uint32))
    return out


def u01(w):
    return lib().oracle_u01(int(w))


def s11(w):
    return lib().oracle_s11(int(w))


def u53(w0, w1):
    return lib().oracle_u53(int(w0), int(w1))


def poisson_lambda(R_s, n_r):
    """lambda = z_p * |V_0| for the sampling sphere of radius R_s."""
    return lib().oracle_lambda(float(R_s), float(n_r))


def poisson_table(lam, cap=8192):
    F = np.zeros(cap, dtype=np.float64)
    n = lib().oracle_poisson_table(float(lam), _p(F, ctypes.c_double), cap)
    if n < 0:
        raise ValueError("poisson table: lambda out of range")
    return F[:n].copy()


def poisson_sample(F, u):
    """N_p = #{k : F[k] <= u} for one 53-bit uniform u."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    return lib().oracle_poisson_sample(_p(F, ctypes.c_double), len(F), float(u))


def acceptance(pos, L, i, xn, *, shape=SHAPE_SPHERE, shape_params=(1.0,), q=0.0,
               n_r=0.0, n_trial=0, cb_mode=0, v0_mode=0, soft_eps=0.0, d_max=0.0, seed=1,
               quat=None, qn=None, sweep0=0, n_rep=1000):
    """How many of n_rep independent evaluations accept the fixed proposed move
    of colloid i to position xn (and orientation qn).  Returns (count, counters).
    v0_mode 1 samples depletants in the thinnest shell level (of a system with
    step size d_max) that holds the move's lens."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    sp = np.ascontiguousarray(shape_params, dtype=np.float64)
    x = np.ascontiguousarray(xn, dtype=np.float64)
    qa = None if quat is None else np.ascontiguousarray(quat, dtype=np.float64)
    qb = None if qn is None else np.ascontiguousarray(qn, dtype=np.float64)
    cnt = np.zeros(N_COUNTERS, dtype=np.uint64)
    a = lib().oracle_acceptance(
        pos.shape[0], float(L), int(shape), _p(sp, ctypes.c_double), len(sp),
        float(q), float(n_r), int(n_trial), int(cb_mode), int(v0_mode), float(soft_eps),
        float(d_max), int(seed), _p(pos, ctypes.c_double),
        _p(qa, ctypes.c_double) if qa is not None else None, int(i),
        _p(x, ctypes.c_double), _p(qb, ctypes.c_double) if qb is not None else None,
        int(sweep0), int(n_rep), _p(cnt, ctypes.c_uint64))
    if a < 0:
        raise ValueError("oracle_acceptance rejected its arguments")
    return int(a), {name: int(cnt[k]) for k, name in enumerate(COUNTERS)}


def schedule(seed, replica, sweep, w):
    sigma = np.zeros(3)
    perm = np.zeros(8, dtype=np.int32)
    lib().oracle_schedule(int(seed), int(replica), int(sweep), float(w),
                          _p(sigma, ctypes.c_double), _p(perm, ctypes.c_int))
    return sigma, perm


def auto_cells(L, R_circ, q):
    return lib().oracle_auto_cells(float(L), float(R_circ), float(q))


def cell_list(pos, L, nc, seed, replica, sweep):
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    n = pos.shape[0]
    start = np.zeros(nc ** 3 + 1, dtype=np.int32)
    idx = np.zeros(max(n, 1), dtype=np.int32)
    rc = lib().oracle_cell_list(n, float(L), int(nc), _p(pos, ctypes.c_double),
                                int(seed), int(replica), int(sweep),
                                _p(start, ctypes.c_int), _p(idx, ctypes.c_int))
    if rc != 0:
        raise ValueError("oracle_cell_list failed")
    return start, idx[:n]


def run(pos, L, *, shape=SHAPE_SPHERE, shape_params=(1.0,), q=0.0, n_r=0.0,
        n_trial=0, cb_mode=0, v0_mode=0, soft_eps=0.0, d_max=0.1, a_max=0.0, p_translate=1.0, seed=1,
        replica=0, n_cell=0, brute_force=False, quat=None, sweep0=0, n_sweeps=1,
        hist_bins=0, hist_rmax=0.0, threads=1):
    """Run the sampler in place on copies of pos/quat (threads > 1: the active
    cells of each colour phase on that many threads, identical results).

    Returns (pos, quat, counters dict, hist or None)."""
    pos = np.array(pos, dtype=np.float64, order="C").reshape(-1, 3)
    n = pos.shape[0]
    qa = None
    if quat is not None:
        qa = np.array(quat, dtype=np.float64, order="C").reshape(-1, 4)
    sp = np.ascontiguousarray(shape_params, dtype=np.float64)
    cnt = np.zeros(N_COUNTERS, dtype=np.uint64)
    hist = np.zeros(max(hist_bins, 1), dtype=np.uint64) if hist_bins > 0 else None
    rc = lib().oracle_run_threads(
        n, float(L), int(shape), _p(sp, ctypes.c_double), len(sp), float(q),
        float(n_r), int(n_trial), int(cb_mode), int(v0_mode), float(soft_eps), float(d_max),
        float(a_max),
        float(p_translate), int(seed), int(replica), int(n_cell),
        int(bool(brute_force)), _p(pos, ctypes.c_double),
        _p(qa, ctypes.c_double) if qa is not None else None,
        int(sweep0), int(n_sweeps), _p(cnt, ctypes.c_uint64),
        int(hist_bins), float(hist_rmax),
        _p(hist, ctypes.c_uint64) if hist is not None else None, int(threads))
    if rc != 0:
        raise ValueError("oracle_run rejected its arguments (rc=%d)" % rc)
    counters = {name: int(cnt[i]) for i, name in enumerate(COUNTERS)}
    return pos, qa, counters, hist


def exp_neg(y):
    return lib().oracle_exp_neg(float(y))


def hertz(eps, sigma, r2):
    return lib().oracle_hertz(float(eps), float(sigma), float(r2))


def shell_level(w0, w1, w2):
    """Shell level (1..32) of a translation drawn from move words w0..w2."""
    w = np.array([w0, w1, w2], dtype=np.uint32)
    return lib().oracle_shell_level(_p(w, ctypes.c_uint32))


def s21(a):
    return lib().oracle_s21(int(a))


def paired_points(R_s, n_att, *, seed=1, sweep=0, tag=0):
    """The points (n_att x 3) of attempts 0 .. n_att - 1 of a paired depletant
    stream (two attempts per Philox call), in or out of the ball."""
    e = np.zeros((max(n_att, 1), 3))
    lib().oracle_paired_points(float(R_s), int(seed), int(sweep), int(tag), int(n_att),
                               _p(e, ctypes.c_double))
    return e[:n_att].copy()


def shell_lambda(R_s, R_in, n_r):
    return lib().oracle_shell_lambda(float(R_s), float(R_in), float(n_r))


def shell_points(R_s, d_max, lvl, n_att, *, seed=1, sweep=0, tag=0):
    """Points the shell generator accepts among n_att attempts (n x 3)."""
    e = np.zeros((max(n_att, 1), 3))
    m = lib().oracle_shell_points(float(R_s), float(d_max), int(lvl), int(seed), int(sweep),
                                  int(tag), int(n_att), _p(e, ctypes.c_double))
    if m < 0:
        raise ValueError("oracle_shell_points rejected its arguments")
    return e[:m].copy()


GIBBS_COUNTERS = ("attempts", "accept", "reject_empty", "reject_ratio", "reject_overlap",
                  "reject_depletant", "reject_cb", "dep_drawn")


def gibbs_run(pos0, pos1, L0, L1, *, diameter=1.0, q=0.0, n_r=0.0, n_trial=0, d_max=(0.1, 0.1),
              seed=1, replicas=(0, 1), sweep0=0, step0=0, n_cycles=1, sweeps_per_cycle=1,
              ex_per_cycle=1):
    """A Gibbs pair of sphere boxes: cycles of sweeps of both boxes, then
    exchange attempts.  Returns (pos0, pos1, counters0, counters1, gibbs
    counters) with the boxes' live colloids."""
    a = np.ascontiguousarray(pos0, dtype=np.float64).reshape(-1, 3)
    b = np.ascontiguousarray(pos1, dtype=np.float64).reshape(-1, 3)
    cap = a.shape[0] + b.shape[0]
    p0 = np.zeros((cap, 3))
    p1 = np.zeros((cap, 3))
    p0[:a.shape[0]] = a
    p1[:b.shape[0]] = b
    n = np.array([a.shape[0], b.shape[0]], dtype=np.int32)
    cnt = np.zeros(2 * N_COUNTERS, dtype=np.uint64)
    g = np.zeros(len(GIBBS_COUNTERS), dtype=np.uint64)
    rc = lib().oracle_gibbs_run(
        float(diameter), float(q), float(n_r), int(n_trial), float(d_max[0]), float(d_max[1]),
        int(seed), int(replicas[0]), int(replicas[1]), float(L0), float(L1),
        _p(n, ctypes.c_int), _p(p0, ctypes.c_double), _p(p1, ctypes.c_double), int(sweep0),
        int(step0), int(n_cycles), int(sweeps_per_cycle), int(ex_per_cycle),
        _p(cnt, ctypes.c_uint64), _p(g, ctypes.c_uint64))
    if rc != 0:
        raise ValueError("oracle_gibbs_run rejected its arguments")
    c0 = {name: int(cnt[k]) for k, name in enumerate(COUNTERS)}
    c1 = {name: int(cnt[N_COUNTERS + k]) for k, name in enumerate(COUNTERS)}
    gc = {name: int(g[k]) for k, name in enumerate(GIBBS_COUNTERS)}
    return p0[:n[0]].copy(), p1[:n[1]].copy(), c0, c1, gc


def gibbs_acceptance(pos0, pos1, L0, L1, src, i, xn, *, diameter=1.0, q=0.0, n_r=0.0,
                     n_trial=0, seed=1, replica=0, step0=0, n_rep=1000):
    """How many of n_rep evaluations accept moving slot i of box src to xn
    in the other box.  Returns (count, gibbs counters)."""
    a = np.ascontiguousarray(pos0, dtype=np.float64).reshape(-1, 3)
    b = np.ascontiguousarray(pos1, dtype=np.float64).reshape(-1, 3)
    x = np.ascontiguousarray(xn, dtype=np.float64)
    g = np.zeros(len(GIBBS_COUNTERS), dtype=np.uint64)
    acc = lib().oracle_gibbs_acceptance(
        float(diameter), float(q), float(n_r), int(n_trial), int(seed), int(replica),
        float(L0), float(L1), a.shape[0], b.shape[0], _p(a, ctypes.c_double),
        _p(b, ctypes.c_double), int(src), int(i), _p(x, ctypes.c_double), int(step0),
        int(n_rep), _p(g, ctypes.c_uint64))
    if acc < 0:
        raise ValueError("oracle_gibbs_acceptance rejected its arguments")
    return int(acc), {name: int(g[k]) for k, name in enumerate(GIBBS_COUNTERS)}


def free_volume(pos, L, q, *, shape=SHAPE_SPHERE, shape_params=(1.0,), quat=None,
                seed=7, sample=0, n_probe=100000):
    """Fraction of n_probe uniform points free of every colloid."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    sp = np.ascontiguousarray(shape_params, dtype=np.float64)
    qa = None if quat is None else np.ascontiguousarray(quat, dtype=np.float64)
    c = lib().oracle_free_volume(pos.shape[0], float(L), int(shape),
                                 _p(sp, ctypes.c_double), float(q),
                                 _p(pos, ctypes.c_double),
                                 _p(qa, ctypes.c_double) if qa is not None else None,
                                 int(seed), int(sample), int(n_probe))
    if c < 0:
        raise ValueError("oracle_free_volume failed")
    return c / float(n_probe)


def _opt(a, n):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64).reshape(n)


def dep_overlap(v, q, *, shape=SHAPE_SPHERE, shape_params=(1.0,), quat=None):
    """Does a depletant of diameter q at v (relative to the colloid's reference
    point, lab frame) overlap the colloid of orientation quat?"""
    sp = np.ascontiguousarray(shape_params, dtype=np.float64)
    vv = _opt(v, 3)
    qq = _opt(quat, 4)
    r = lib().oracle_dep_overlap(int(shape), _p(sp, ctypes.c_double), len(sp), float(q),
                                 _p(vv, ctypes.c_double),
                                 _p(qq, ctypes.c_double) if qq is not None else None)
    if r < 0:
        raise ValueError("oracle_dep_overlap rejected its arguments")
    return bool(r)


def pair_overlap(r, *, shape=SHAPE_SPHERE, shape_params=(1.0,), qa=None, qb=None):
    """Do two colloids with reference points separated by r (first to second)
    and orientations qa, qb overlap?"""
    sp = np.ascontiguousarray(shape_params, dtype=np.float64)
    rr = _opt(r, 3)
    a = _opt(qa, 4)
    b = _opt(qb, 4)
    res = lib().oracle_pair_overlap(int(shape), _p(sp, ctypes.c_double), len(sp),
                                    _p(rr, ctypes.c_double),
                                    _p(a, ctypes.c_double) if a is not None else None,
                                    _p(b, ctypes.c_double) if b is not None else None)
    if res < 0:
        raise ValueError("oracle_pair_overlap rejected its arguments")
    return bool(res)


def rotation_proposal(q, a_max, *, seed=1, replica=0, sweep=0, tag=0):
    """The rotated orientation proposed for colloid `tag` in `sweep`, or None
    if the attempt stream hit its cap."""
    qi = _opt(q, 4)
    qo = np.zeros(4)
    rc = lib().oracle_rotation_proposal(int(seed), int(replica), int(sweep), int(tag),
                                        float(a_max), _p(qi, ctypes.c_double),
                                        _p(qo, ctypes.c_double))
    if rc < 0:
        raise ValueError("oracle_rotation_proposal rejected its arguments")
    return qo if rc == 1 else None
