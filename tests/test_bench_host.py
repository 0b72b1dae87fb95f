"""Host logic of the benchmark: the step-size rule both arms replay, the
checkerboard width it bounds the step by, and the oracle leg's replica
pool (threads over independent replicas give the serial results)."""
import math

import numpy as np

import bench
from paper_1508_07077_gb300 import workloads as W


def test_tune_update_moves_towards_the_target_and_stays_bounded():
    w = 1.2
    assert bench.tune_update(0.01, 30, 100, w) == 0.01          # at the target
    assert bench.tune_update(0.01, 60, 100, w) > 0.01           # too many accepted: larger
    assert bench.tune_update(0.01, 5, 100, w) < 0.01            # too few: smaller
    assert bench.tune_update(0.01, 100, 100, w) == 0.02         # at most a factor 2
    assert bench.tune_update(0.01, 0, 100, w) == 0.005          # at least a factor 1/2
    assert bench.tune_update(0.5, 100, 100, w) == 0.25 * w      # below a quarter cell
    assert bench.tune_update(1e-4, 0, 100, w) == 1e-4           # and above 1e-4
    assert bench.tune_update(0.01, 0, 0, w) == 0.005            # no moves counts as none accepted


def test_cell_width_is_the_largest_even_grid():
    for L, q in ((13.8, 0.2), (30.58, 0.15), (2.4, 0.2), (7.0, 0.1)):
        w = bench.cell_width(L, q)
        nc = round(L / w)
        assert nc % 2 == 0 and w >= 1.0 + q - 1e-12
        assert L / (nc + 2) < 1.0 + q


def test_workload_is_the_128_replica_batch():
    reps, keys, widths = bench.batched_workload(0)
    assert len(reps) == 128 and keys == list(range(128))
    assert sum(s.n for s in reps) == bench.batched_config()["colloids"]
    assert all(500 <= s.n <= 20000 for s in reps)
    _, keys1, _ = bench.batched_workload(1)
    assert keys1 == list(range(128, 256))


def test_oracle_batch_threads_equal_serial(oracle):
    reps = [W.make_system("a", W.SPHERE, 300, 0.2, 0.2, 0.2, seed=2, replica=0),
            W.make_system("b", W.SPHERE, 500, 0.3, 0.15, 0.1, seed=2, replica=1)]
    widths = [bench.cell_width(s.L, s.q) for s in reps]
    one = bench.OracleBatch(reps, [0, 1], cores=1)
    many = bench.OracleBatch(reps, [0, 1], cores=2)
    d1, d2 = one.tune(widths), many.tune(widths)
    assert d1 == d2
    c1, c2 = one.run(d1, 2), many.run(d2, 2)
    assert c1 == c2
    for a, b in zip(one.pos, many.pos):
        assert np.array_equal(a, b)
    assert all(math.isfinite(x) and x > 0 for x in d1)
