"""Pins of the oracle's checkerboard sampler (Sec. III.E) that need no
statistics: the cell list, the sweep schedule, brute-force neighbour
enumeration, the hard-core invariant and the counters."""
import math

import numpy as np
import pytest

from paper_1508_07077_gb300 import workloads as W


def _ref_cells(pos, L, nc, sigma):
    """Cell of each particle from the plain definition
    c_d = floor(((x_d - sigma_d) mod L) / w)."""
    w = L / nc
    s = np.mod(pos - sigma[None, :], L)
    c = np.minimum(np.floor(s / w).astype(int), nc - 1)
    return c[:, 0] + nc * (c[:, 1] + nc * c[:, 2])


@pytest.mark.parametrize("sweep", [0, 1, 17, 999])
def test_cell_list_is_a_stable_counting_sort(oracle, sweep):
    s = W.spheres_256()
    nc = oracle.auto_cells(s.L, 0.5, s.q)
    start, idx = oracle.cell_list(s.pos, s.L, nc, 1, 0, sweep)
    sigma, _ = oracle.schedule(1, 0, sweep, s.L / nc)
    cell = _ref_cells(s.pos, s.L, nc, sigma)
    assert start[0] == 0 and start[-1] == s.n and np.all(np.diff(start) >= 0)
    assert sorted(idx.tolist()) == list(range(s.n))
    for c in range(nc ** 3):
        members = idx[start[c]:start[c + 1]]
        assert np.all(np.diff(members) > 0)               # ascending tag
        assert np.all(cell[members] == c)
    counts = np.bincount(cell, minlength=nc ** 3)
    assert np.array_equal(np.diff(start), counts)


def test_schedule_shift_and_colour_permutation(oracle):
    w = 1.4585
    seen = np.zeros((8, 8), dtype=int)
    for sweep in range(4000):
        sigma, perm = oracle.schedule(1, 0, sweep, w)
        assert np.all(sigma > 0.0) and np.all(sigma < w)
        assert sorted(perm.tolist()) == list(range(8))
        seen[np.arange(8), perm] += 1
    # every colour equally likely at every phase position
    assert np.all(np.abs(seen - 500) < 5 * math.sqrt(500 * 7 / 8))


def test_auto_cells_even_and_wide_enough(oracle):
    for L, q in [(8.751, 0.2), (30.58, 0.15), (2.4, 0.2), (5.0, 0.1)]:
        nc = oracle.auto_cells(L, 0.5, q)
        assert nc % 2 == 0 and nc >= 2
        assert L / nc >= 1.0 + q
        assert L / (nc + 2) < 1.0 + q


@pytest.mark.parametrize("n_trial", [0, 3])
def test_cell_neighbours_equal_brute_force(oracle, n_trial):
    """Gathering neighbours from the 27 cells gives the same trajectory as
    testing against every colloid (tiny box with nc = 2, and 256 spheres)."""
    cases = [(W.tiny_spheres(8, 2.6), 2.6, 0.2, 30.0),
             (W.spheres_256().pos, W.spheres_256().L, 0.2, 47.75)]
    for pos, L, q, zp in cases:
        a = oracle.run(pos, L, q=q, n_r=zp, n_trial=n_trial, d_max=0.08, n_sweeps=15)
        b = oracle.run(pos, L, q=q, n_r=zp, n_trial=n_trial, d_max=0.08, n_sweeps=15,
                       brute_force=True)
        assert np.array_equal(a[0], b[0])
        assert a[2] == b[2]


def _min_pair_distance(pos, L):
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    r[np.diag_indices(len(pos))] = np.inf
    return r.min()


def test_hard_core_and_counters(oracle):
    s = W.spheres_256()
    pos, _, c, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, n_trial=2, d_max=0.05,
                              n_sweeps=30)
    assert _min_pair_distance(pos, s.L) >= 1.0
    assert np.all(pos >= 0.0) and np.all(pos < s.L)
    assert c["moves"] == 30 * s.n
    assert c["moves"] == (c["accept"] + c["reject_cell"] + c["reject_overlap"]
                          + c["reject_depletant"] + c["reject_cb"])
    assert c["reject_depletant"] == 0           # n_trial > 0: CB decides
    assert c["cap_hits"] == 0


def test_zero_fugacity_draws_no_depletants(oracle):
    s = W.spheres_256()
    _, _, c, _ = oracle.run(s.pos, s.L, q=s.q, n_r=0.0, d_max=0.1, n_sweeps=5)
    assert c["dep_drawn"] == 0 and c["reject_depletant"] == 0


def test_resume_is_bit_exact(oracle):
    s = W.spheres_256()
    a = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.05, n_sweeps=20)
    h = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.05, n_sweeps=10)
    b = oracle.run(h[0], s.L, q=s.q, n_r=s.n_r, d_max=0.05, n_sweeps=10, sweep0=10)
    assert np.array_equal(a[0], b[0])


def test_argument_validation(oracle):
    s = W.spheres_256()
    with pytest.raises(ValueError):
        oracle.run(s.pos, 2.0, q=0.2, n_r=1.0)            # box below two cells
    with pytest.raises(ValueError):
        oracle.run(s.pos, s.L, q=0.2, n_r=1.0, d_max=5.0)  # step wider than a cell
    with pytest.raises(ValueError):
        oracle.run(s.pos, s.L, q=0.2, n_r=1e6)             # lambda beyond the table
