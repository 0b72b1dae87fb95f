"""The oracle's threaded sweep (the active cells of one colour phase handed
out to threads) against its serial sweep.

Sec. III.E makes the active cells of one colour independent: a colloid moves
only inside its own cell and interacts only with colloids of the 26
neighbouring cells, none of which is active in the same phase.  So the order
in which the cells of a phase are processed cannot matter, and the threaded
run must give the serial run's positions, orientations and counters exactly,
for every thread count (this is what makes the all-core CPU baseline a
measurement of the same computation)."""
import numpy as np
import pytest

from paper_1508_07077_gb300 import workloads as W


def _both(oracle, s, threads, **kw):
    a = oracle.run(s.pos, s.L, shape=s.shape, shape_params=s.shape_params, quat=s.quat,
                   q=s.q, n_r=s.n_r, a_max=s.a_max, p_translate=s.p_translate, **kw)
    b = oracle.run(s.pos, s.L, shape=s.shape, shape_params=s.shape_params, quat=s.quat,
                   q=s.q, n_r=s.n_r, a_max=s.a_max, p_translate=s.p_translate,
                   threads=threads, **kw)
    return a, b


@pytest.mark.parametrize("threads", [2, 5])
@pytest.mark.parametrize("n_trial,v0", [(0, 0), (3, 0), (0, 1)])
def test_threaded_sweeps_equal_serial_spheres(oracle, threads, n_trial, v0):
    s = W.make_system("par", W.SPHERE, 2048, 0.30, 0.15, 0.2, seed=4)
    a, b = _both(oracle, s, threads, d_max=0.05, n_trial=n_trial, v0_mode=v0, seed=4,
                 n_sweeps=3)
    assert np.array_equal(a[0], b[0])
    assert a[2] == b[2]
    assert a[2]["accept"] > 0


def test_threaded_sweeps_equal_serial_hemispheres(oracle):
    s = W.make_system("par_h", W.HEMISPHERE, 864, 0.20, 0.1, 0.3, seed=6, a_max=0.2,
                      p_translate=0.5)
    a, b = _both(oracle, s, 3, d_max=0.05, seed=6, n_sweeps=2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2] == b[2]


def test_smallest_grid_two_cells_per_side(oracle):
    """n_c = 2: each colour has one cell, the stencil is the whole box."""
    pos = W.tiny_spheres(8, 2.6, seed=3)
    a = oracle.run(pos, 2.6, q=0.2, n_r=20.0, d_max=0.1, n_sweeps=5)
    b = oracle.run(pos, 2.6, q=0.2, n_r=20.0, d_max=0.1, n_sweeps=5, threads=4)
    assert np.array_equal(a[0], b[0]) and a[2] == b[2]
