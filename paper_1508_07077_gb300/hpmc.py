"""Thin Python binding of ``libhpmc_dep.so`` (see ``include/hpmc_dep.h``).

Argument marshalling only: every step of the Monte Carlo path runs in the
library's CUDA kernels.  Functions carry the C names; negative return codes
raise :class:`HPMCError`.  Device buffers may be torch CUDA tensors (their
``data_ptr()`` is passed), host buffers numpy arrays.  The library is loaded
from the package's in-tree ``_lib/``; if it is missing the import fails loudly
(there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIBDIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib")
LIB_PATH = os.path.join(_LIBDIR, "libhpmc_dep.so")
# the same library with bounds and checkerboard-invariant checks (HPMC_CHECKED)
CHECKED_LIB_PATH = os.path.join(_LIBDIR, "libhpmc_dep_checked.so")

HPMC_OK = 0
HPMC_SPHERE, HPMC_HEMISPHERE, HPMC_SPHEROID = 0, 1, 2
HPMC_FP64, HPMC_FP32_RECHECK = 0, 1
HPMC_HOST, HPMC_DEVICE = 0, 1
HPMC_V0_CIRCUMSPHERE, HPMC_V0_SHELL, HPMC_V0_CUBE = 0, 1, 2
HPMC_PHASES_LAUNCHES, HPMC_PHASES_PERSISTENT = 0, 1

EXPORTS = ("hpmc_init", "hpmc_init_batch", "hpmc_get_replica", "hpmc_set_replica_moves",
           "hpmc_set_shape", "hpmc_set_depletant", "hpmc_set_moves",
           "hpmc_set_cells", "hpmc_set_launch", "hpmc_set_phase_waves", "hpmc_set_wait_limit",
           "hpmc_debug_withhold_cell", "hpmc_autotune", "hpmc_set_fp32_margin",
           "hpmc_set_v0", "hpmc_set_soft", "hpmc_set_live", "hpmc_get_live", "hpmc_gibbs_exchange",
           "hpmc_get_gibbs", "hpmc_set_timing",
           "hpmc_get_timing", "hpmc_sweep", "hpmc_get_state",
           "hpmc_set_state", "hpmc_reset_counters", "hpmc_sync", "hpmc_cell_list",
           "hpmc_cell_list_noalloc", "hpmc_philox", "hpmc_kernel_arch", "hpmc_free_volume", "hpmc_get_size", "hpmc_strerror",
           "hpmc_destroy")


class HPMCError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, strerror(code), code))


class hpmc_replica_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("box_l", ctypes.c_double),
                ("pos", ctypes.c_void_p), ("quat", ctypes.c_void_p),
                ("q", ctypes.c_double), ("n_r", ctypes.c_double), ("n_trial", ctypes.c_int),
                ("d_max", ctypes.c_double), ("a_max", ctypes.c_double),
                ("p_translate", ctypes.c_double), ("replica", ctypes.c_uint32),
                ("n_cell", ctypes.c_int)]


class hpmc_counters(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in (
        "moves", "accept", "reject_cell", "reject_overlap", "reject_depletant",
        "reject_cb", "dep_drawn", "translate", "dep_evaluated", "dep_blocking",
        "cb_fwd_ok", "cb_rev_ok", "cap_hits", "rechecks")] + [
        ("reserved", ctypes.c_uint64 * 2)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_
                if name != "reserved"}


_lib = None
_lib_path = LIB_PATH


def load(path: str = LIB_PATH):
    """Load the shared library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libhpmc_dep.so not built (run __graft_entry__.build()): " + path)
    L = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    L.hpmc_init.argtypes = [ctypes.POINTER(vp), ip, ctypes.c_double, vp, vp, ip,
                            ctypes.c_uint64, ctypes.c_uint32, ip, ip]
    L.hpmc_init_batch.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(hpmc_replica_desc), ip,
                                  dp, ip, ctypes.c_uint64, ip, ip]
    L.hpmc_get_replica.argtypes = [vp, ip, vp, vp, ctypes.POINTER(hpmc_counters)]
    L.hpmc_set_replica_moves.argtypes = [vp, ip, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double]
    L.hpmc_set_shape.argtypes = [vp, ip, dp, ip]
    L.hpmc_set_depletant.argtypes = [vp, ctypes.c_double, ctypes.c_double, ip]
    L.hpmc_set_moves.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.hpmc_set_cells.argtypes = [vp, ip]
    L.hpmc_set_launch.argtypes = [vp, ip, ip]
    L.hpmc_set_wait_limit.argtypes = [vp, ctypes.c_double]
    L.hpmc_set_phase_waves.argtypes = [vp, ip]
    L.hpmc_debug_withhold_cell.argtypes = [vp, ip]
    L.hpmc_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ip, ctypes.POINTER(ctypes.c_int),
                                ip, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_double)]
    L.hpmc_set_fp32_margin.argtypes = [vp, ctypes.c_double]
    L.hpmc_set_v0.argtypes = [vp, ip]
    L.hpmc_set_soft.argtypes = [vp, ctypes.c_double]
    L.hpmc_set_live.argtypes = [vp, ip, ip]
    L.hpmc_get_live.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.hpmc_gibbs_exchange.argtypes = [vp, ip, vp]
    L.hpmc_get_gibbs.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.POINTER(ctypes.c_uint64)]
    L.hpmc_set_timing.argtypes = [vp, ip]
    L.hpmc_get_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_uint64), ip]
    L.hpmc_sweep.argtypes = [vp, ip, vp]
    L.hpmc_get_state.argtypes = [vp, vp, vp, ip, ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.POINTER(hpmc_counters), vp]
    L.hpmc_set_state.argtypes = [vp, vp, vp, ip, ctypes.c_uint64, vp]
    L.hpmc_reset_counters.argtypes = [vp]
    L.hpmc_sync.argtypes = [vp]
    L.hpmc_cell_list.argtypes = [ip, ctypes.c_double, ip, vp, ctypes.c_uint64,
                                 ctypes.c_uint32, ctypes.c_uint64, vp, vp, vp]
    L.hpmc_cell_list_noalloc.argtypes = L.hpmc_cell_list.argtypes
    L.hpmc_philox.argtypes = [ip, vp, vp, vp, ip, vp]
    L.hpmc_kernel_arch.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.hpmc_free_volume.argtypes = [vp, ip, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
    L.hpmc_get_size.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.hpmc_strerror.argtypes = [ip]
    L.hpmc_strerror.restype = ctypes.c_char_p
    L.hpmc_destroy.argtypes = [vp]
    L.hpmc_destroy.restype = None
    for name in EXPORTS:
        if name not in ("hpmc_strerror", "hpmc_destroy"):
            getattr(L, name).restype = ctypes.c_int
    global _lib_path
    _lib = L
    _lib_path = path
    return L


def use(path: str = LIB_PATH):
    """Make the binding call the library at `path` (e.g. CHECKED_LIB_PATH)
    from now on; returns the path it used before."""
    global _lib, _lib_path
    prev = _lib_path
    _lib = None
    load(path)
    return prev


def strerror(code: int) -> str:
    return load().hpmc_strerror(int(code)).decode()


def _check(rc: int, where: str) -> None:
    if rc != HPMC_OK:
        raise HPMCError(rc, where)


def _ptr(buf):
    """(address, mem kind) of a numpy array (host) or a torch tensor."""
    if buf is None:
        return None, HPMC_HOST
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous or buf.dtype != np.float64:
            raise ValueError("host arrays must be C-contiguous float64")
        return buf.ctypes.data, HPMC_HOST
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous() or str(buf.dtype) != "torch.float64":
            raise ValueError("tensors must be contiguous float64")
        return buf.data_ptr(), (HPMC_DEVICE if buf.is_cuda else HPMC_HOST)
    raise TypeError("unsupported buffer type %r" % type(buf))


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def hpmc_init(n, box_l, pos, quat=None, seed=1, replica=0, precision=HPMC_FP64, device=0):
    p, mem = _ptr(pos)
    q, mem_q = _ptr(quat)
    if quat is not None and mem_q != mem:
        raise ValueError("pos and quat must live in the same memory")
    ctx = ctypes.c_void_p()
    _check(load().hpmc_init(ctypes.byref(ctx), int(n), float(box_l), p, q, mem,
                            int(seed), int(replica), int(precision), int(device)),
           "hpmc_init")
    return ctx


def hpmc_init_batch(replicas, shape=HPMC_SPHERE, shape_params=(1.0,), seed=1,
                    precision=HPMC_FP64, device=0):
    """replicas: list of dicts with keys n, box_l, pos (n x 3 float64), quat
    (optional), q, n_r, n_trial, d_max, a_max, p_translate, replica, n_cell."""
    arr = (hpmc_replica_desc * len(replicas))()
    keep = []
    for k, r in enumerate(replicas):
        pos = np.ascontiguousarray(r["pos"], dtype=np.float64)
        keep.append(pos)
        quat = r.get("quat")
        if quat is not None:
            quat = np.ascontiguousarray(quat, dtype=np.float64)
            keep.append(quat)
        arr[k] = hpmc_replica_desc(
            int(r["n"]), float(r["box_l"]), pos.ctypes.data,
            quat.ctypes.data if quat is not None else None, float(r.get("q", 0.0)),
            float(r.get("n_r", 0.0)), int(r.get("n_trial", 0)), float(r.get("d_max", 0.1)),
            float(r.get("a_max", 0.0)), float(r.get("p_translate", 1.0)),
            int(r.get("replica", k)), int(r.get("n_cell", 0)))
    sp = np.ascontiguousarray(shape_params, dtype=np.float64)
    ctx = ctypes.c_void_p()
    _check(load().hpmc_init_batch(ctypes.byref(ctx), len(replicas), arr, int(shape),
                                  sp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(sp),
                                  int(seed), int(precision), int(device)), "hpmc_init_batch")
    return ctx


def hpmc_get_replica(ctx, r, n, with_quat=False):
    """(pos, quat or None, counters dict) of replica r (n colloids)."""
    pos = np.empty((n, 3))
    quat = np.empty((n, 4)) if with_quat else None
    cnt = hpmc_counters()
    _check(load().hpmc_get_replica(ctx, int(r), pos.ctypes.data,
                                   quat.ctypes.data if quat is not None else None,
                                   ctypes.byref(cnt)), "hpmc_get_replica")
    return pos, quat, cnt.as_dict()


def hpmc_set_replica_moves(ctx, r, d_max, a_max=0.0, p_translate=1.0):
    _check(load().hpmc_set_replica_moves(ctx, int(r), float(d_max), float(a_max),
                                         float(p_translate)), "hpmc_set_replica_moves")


def hpmc_set_shape(ctx, kind, params):
    a = np.ascontiguousarray(params, dtype=np.float64)
    _check(load().hpmc_set_shape(ctx, int(kind), a.ctypes.data_as(
        ctypes.POINTER(ctypes.c_double)), len(a)), "hpmc_set_shape")


def hpmc_set_depletant(ctx, q, n_r, n_trial=0):
    _check(load().hpmc_set_depletant(ctx, float(q), float(n_r), int(n_trial)),
           "hpmc_set_depletant")


def hpmc_set_moves(ctx, d_max, a_max=0.0, p_translate=1.0):
    _check(load().hpmc_set_moves(ctx, float(d_max), float(a_max), float(p_translate)),
           "hpmc_set_moves")


def hpmc_set_cells(ctx, n_cell):
    _check(load().hpmc_set_cells(ctx, int(n_cell)), "hpmc_set_cells")


def hpmc_autotune(ctx, warps=(1, 2, 4), cells=(0,), n_sweeps=5):
    """Time every (warps_per_colloid, cells per side) pair and keep the fastest;
    the state is restored.  Returns (warps, cells, ms_per_sweep)."""
    wa = (ctypes.c_int * len(warps))(*[int(w) for w in warps])
    ca = (ctypes.c_int * len(cells))(*[int(c) for c in cells])
    bw, bc, bm = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(load().hpmc_autotune(ctx, wa, len(warps), ca, len(cells), int(n_sweeps),
                                ctypes.byref(bw), ctypes.byref(bc), ctypes.byref(bm)),
           "hpmc_autotune")
    return bw.value, bc.value, bm.value


def hpmc_free_volume(ctx, q, *, replica=0, seed=7, sample=0, n_probe=1000000):
    """(free probes, n_probe): probes of replica `replica` overlapping no colloid
    as a depletant of diameter q."""
    out = ctypes.c_uint64(0)
    _check(load().hpmc_free_volume(ctx, int(replica), float(q), int(seed), int(sample),
                                   int(n_probe), ctypes.byref(out)), "hpmc_free_volume")
    return out.value, int(n_probe)


def hpmc_set_launch(ctx, warps_per_colloid, phase_schedule=HPMC_PHASES_LAUNCHES):
    _check(load().hpmc_set_launch(ctx, int(warps_per_colloid), int(phase_schedule)),
           "hpmc_set_launch")


def hpmc_set_phase_waves(ctx, waves):
    _check(load().hpmc_set_phase_waves(ctx, int(waves)), "hpmc_set_phase_waves")


def hpmc_set_wait_limit(ctx, seconds):
    _check(load().hpmc_set_wait_limit(ctx, float(seconds)), "hpmc_set_wait_limit")


def hpmc_debug_withhold_cell(ctx, cell):
    _check(load().hpmc_debug_withhold_cell(ctx, int(cell)), "hpmc_debug_withhold_cell")


def hpmc_set_fp32_margin(ctx, margin):
    _check(load().hpmc_set_fp32_margin(ctx, float(margin)), "hpmc_set_fp32_margin")


def hpmc_set_v0(ctx, mode):
    _check(load().hpmc_set_v0(ctx, int(mode)), "hpmc_set_v0")


def hpmc_set_soft(ctx, eps):
    _check(load().hpmc_set_soft(ctx, float(eps)), "hpmc_set_soft")


def hpmc_set_live(ctx, replica, n_live):
    _check(load().hpmc_set_live(ctx, int(replica), int(n_live)), "hpmc_set_live")


def hpmc_get_live(ctx, n_rep):
    out = (ctypes.c_int * n_rep)()
    _check(load().hpmc_get_live(ctx, out), "hpmc_get_live")
    return [int(x) for x in out]


def hpmc_gibbs_exchange(ctx, n_attempts, stream=None):
    _check(load().hpmc_gibbs_exchange(ctx, int(n_attempts), _stream(stream)),
           "hpmc_gibbs_exchange")


GIBBS_COUNTERS = ("attempts", "accept", "reject_empty", "reject_ratio", "reject_overlap",
                  "reject_depletant", "reject_cb", "dep_drawn")


def hpmc_get_gibbs(ctx, pair):
    """(attempt count, counters dict) of Gibbs pair `pair`."""
    step = ctypes.c_uint64(0)
    cnt = (ctypes.c_uint64 * 8)()
    _check(load().hpmc_get_gibbs(ctx, int(pair), ctypes.byref(step), cnt), "hpmc_get_gibbs")
    return int(step.value), {k: int(v) for k, v in zip(GIBBS_COUNTERS, cnt)}


class GibbsPairs:
    """Gibbs-ensemble pairs of sphere boxes in one context: pair p is
    replicas 2p, 2p + 1, each with one slot per colloid of the pair."""

    def __init__(self, pairs, *, diameter=1.0, seed=1, precision=HPMC_FP64, device=0,
                 replica0=0):
        """pairs: list of ((pos0, L0), (pos1, L1), params) with params a dict
        of q, n_r, n_trial, d_max (per box: d_max may be a pair).  Box k of
        pair p is replica replica0 + 2 p + k (its RNG key)."""
        reps, self.live = [], []
        for p, ((a, L0), (b, L1), prm) in enumerate(pairs):
            a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1, 3)
            b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1, 3)
            cap = a.shape[0] + b.shape[0]
            dm = prm.get("d_max", 0.1)
            dm = dm if isinstance(dm, (tuple, list)) else (dm, dm)
            for k, (x, L) in enumerate(((a, L0), (b, L1))):
                slots = np.zeros((cap, 3))
                slots[:x.shape[0]] = x
                reps.append({"n": cap, "box_l": L, "pos": slots, "q": prm.get("q", 0.0),
                             "n_r": prm.get("n_r", 0.0), "n_trial": prm.get("n_trial", 0),
                             "d_max": dm[k], "replica": replica0 + 2 * p + k})
                self.live.append(x.shape[0])
        self.reps = reps
        self.ctx = hpmc_init_batch(reps, shape=HPMC_SPHERE, shape_params=(diameter,), seed=seed,
                                   precision=precision, device=device)
        for r, n in enumerate(self.live):
            hpmc_set_live(self.ctx, r, n)

    def cycle(self, sweeps=1, exchanges=1, stream=None):
        if sweeps:
            hpmc_sweep(self.ctx, sweeps, stream)
        if exchanges:
            hpmc_gibbs_exchange(self.ctx, exchanges, stream)

    def boxes(self):
        """[(pos of the colloids in use, counters)] per replica."""
        live = hpmc_get_live(self.ctx, len(self.reps))
        out = []
        for r, rep in enumerate(self.reps):
            pos, _, cnt = hpmc_get_replica(self.ctx, r, rep["n"])
            out.append((pos[:live[r]].copy(), cnt))
        return out

    def close(self):
        if self.ctx is not None:
            hpmc_destroy(self.ctx)
            self.ctx = None


def hpmc_set_timing(ctx, on):
    _check(load().hpmc_set_timing(ctx, int(bool(on))), "hpmc_set_timing")


def hpmc_get_timing(ctx):
    """(ms, launches) per kind: 0 = cell list, 1 = colour-phase kernel,
    2 = depletant lens kernel."""
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_uint64 * 3)()
    _check(load().hpmc_get_timing(ctx, ms, n, 3), "hpmc_get_timing")
    return [float(x) for x in ms], [int(x) for x in n]


def hpmc_sweep(ctx, n_sweeps=1, stream=None):
    _check(load().hpmc_sweep(ctx, int(n_sweeps), _stream(stream)), "hpmc_sweep")


def hpmc_get_size(ctx):
    """(colloid slots, replicas) of a context."""
    n, r = ctypes.c_int(), ctypes.c_int()
    _check(load().hpmc_get_size(ctx, ctypes.byref(n), ctypes.byref(r)), "hpmc_get_size")
    return int(n.value), int(r.value)


def _check_rows(ctx, buf, width, what):
    """A state buffer must hold exactly one row of `width` per colloid slot
    (the device reads and writes pinned and device buffers in place)."""
    if buf is None:
        return
    n = hpmc_get_size(ctx)[0]
    size = buf.size if isinstance(buf, np.ndarray) else buf.numel()
    if size != n * width:
        raise ValueError("%s must hold %d x %d values, got %d" % (what, n, width, size))


def hpmc_get_state(ctx, pos=None, quat=None, stream=None):
    """Fill pos (n x 3) / quat (n x 4) buffers (numpy or CUDA tensors, same
    memory); returns (sweep, counters dict)."""
    _check_rows(ctx, pos, 3, "pos")
    _check_rows(ctx, quat, 4, "quat")
    p, mem = _ptr(pos)
    q, mem_q = _ptr(quat)
    if pos is not None and quat is not None and mem != mem_q:
        raise ValueError("pos and quat must live in the same memory")
    if pos is None:
        mem = mem_q
    sweep = ctypes.c_uint64()
    cnt = hpmc_counters()
    _check(load().hpmc_get_state(ctx, p, q, mem, ctypes.byref(sweep), ctypes.byref(cnt),
                                 _stream(stream)), "hpmc_get_state")
    return int(sweep.value), cnt.as_dict()


def hpmc_set_state(ctx, pos=None, quat=None, sweep=0, stream=None):
    _check_rows(ctx, pos, 3, "pos")
    _check_rows(ctx, quat, 4, "quat")
    p, mem = _ptr(pos)
    q, mem_q = _ptr(quat)
    if pos is None:
        mem = mem_q
    _check(load().hpmc_set_state(ctx, p, q, mem, int(sweep), _stream(stream)),
           "hpmc_set_state")


def hpmc_reset_counters(ctx):
    _check(load().hpmc_reset_counters(ctx), "hpmc_reset_counters")


def hpmc_sync(ctx):
    _check(load().hpmc_sync(ctx), "hpmc_sync")


def hpmc_cell_list(n, box_l, n_cell, pos_dev, seed, replica, sweep, cell_start_dev,
                   cell_idx_dev, stream=None):
    _check(load().hpmc_cell_list(int(n), float(box_l), int(n_cell), _ptr(pos_dev)[0],
                                 int(seed), int(replica), int(sweep),
                                 cell_start_dev.data_ptr(), cell_idx_dev.data_ptr(),
                                 _stream(stream)), "hpmc_cell_list")


def hpmc_cell_list_noalloc(n, box_l, n_cell, pos_dev, seed, replica, sweep, cell_start_dev,
                           cell_idx_dev, stream=None):
    """hpmc_cell_list without any device allocation (static scratch; see the
    header for its limits and its one-array-per-device sharing rule)."""
    _check(load().hpmc_cell_list_noalloc(int(n), float(box_l), int(n_cell), _ptr(pos_dev)[0],
                                         int(seed), int(replica), int(sweep),
                                         cell_start_dev.data_ptr(), cell_idx_dev.data_ptr(),
                                         _stream(stream)), "hpmc_cell_list_noalloc")


def hpmc_philox(ctr_dev, key_dev, out_dev, variant=0, stream=None):
    """Device Philox4x32-10 of n counters (n x 4 int32 CUDA tensor) under n
    keys (n x 2) into out_dev (n x 4); words are the tensors' bit patterns."""
    n = int(ctr_dev.shape[0])
    if tuple(ctr_dev.shape) != (n, 4) or tuple(key_dev.shape) != (n, 2) or \
            tuple(out_dev.shape) != (n, 4):
        raise ValueError("ctr, key, out must be n x 4, n x 2, n x 4")
    for t in (ctr_dev, key_dev, out_dev):
        if not t.is_cuda or not t.is_contiguous() or t.element_size() != 4:
            raise ValueError("buffers must be contiguous 32-bit CUDA tensors")
    _check(load().hpmc_philox(n, ctr_dev.data_ptr(), key_dev.data_ptr(), out_dev.data_ptr(),
                              int(variant), _stream(stream)), "hpmc_philox")


def hpmc_kernel_arch():
    """(binary version, PTX version) of the library's kernels on the current
    device, as the CUDA runtime reports them."""
    b, p = ctypes.c_int(), ctypes.c_int()
    _check(load().hpmc_kernel_arch(ctypes.byref(b), ctypes.byref(p)), "hpmc_kernel_arch")
    return b.value, p.value


def hpmc_destroy(ctx):
    if ctx:
        load().hpmc_destroy(ctx)


class Sampler:
    """Owns one context: a convenience wrapper over the calls above."""

    def __init__(self, pos, box_l, *, quat=None, shape=HPMC_SPHERE, shape_params=(1.0,),
                 q=0.0, n_r=0.0, n_trial=0, d_max=0.1, a_max=0.0, p_translate=1.0,
                 seed=1, replica=0, precision=HPMC_FP64, n_cell=0, warps=1,
                 schedule=HPMC_PHASES_LAUNCHES, device=0,
                 v0=HPMC_V0_CIRCUMSPHERE, soft_eps=0.0):
        pos = np.ascontiguousarray(pos, dtype=np.float64) if isinstance(pos, np.ndarray) else pos
        if isinstance(quat, np.ndarray):
            quat = np.ascontiguousarray(quat, dtype=np.float64)
        self.n = int(pos.shape[0])
        self.L = float(box_l)
        self.ctx = hpmc_init(self.n, box_l, pos, quat, seed, replica, precision, device)
        try:
            hpmc_set_shape(self.ctx, shape, shape_params)
            hpmc_set_depletant(self.ctx, q, n_r, n_trial)
            hpmc_set_moves(self.ctx, d_max, a_max, p_translate)
            hpmc_set_cells(self.ctx, n_cell)
            hpmc_set_launch(self.ctx, warps, schedule)
            if v0 != HPMC_V0_CIRCUMSPHERE:
                hpmc_set_v0(self.ctx, v0)
            if soft_eps:
                hpmc_set_soft(self.ctx, soft_eps)
        except Exception:
            self.close()
            raise

    def sweep(self, n=1, stream=None):
        hpmc_sweep(self.ctx, n, stream)

    def state(self, with_quat=False):
        pos = np.empty((self.n, 3))
        quat = np.empty((self.n, 4)) if with_quat else None
        sweep, cnt = hpmc_get_state(self.ctx, pos, quat)
        return pos, quat, sweep, cnt

    def close(self):
        if getattr(self, "ctx", None):
            hpmc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
