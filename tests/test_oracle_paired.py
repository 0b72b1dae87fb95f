"""Pins of the paired depletant stream: the depletant points of a trial move
(hard interactions, circumsphere or cube V_0) take two attempts from each
Philox4x32-10 call, 21-bit coordinates from 126 of its 128 bits; in each
block of 64 attempts the first 32 are the first halves of 32 calls and the
next 32 their second halves.

Checked against what a uniform sampler must satisfy, not against a retyped
formula: the 21-bit map hits the stated interval exactly (and in FP32);
every one of the 21 bits of every coordinate of both halves is a fair coin
(a wrong mask or shift leaves a constant or duplicated bit); the coordinates
are uniform and the two halves of a call and the three coordinates of a
point uncorrelated; points in the ball are accepted at the ball-to-cube
volume ratio and are uniform in radius and direction."""
import math

import numpy as np
from scipy import stats

N_ATT = 200000


def _half(n, h):
    """Attempt indices of half h (blocks of 64: 32 first halves, 32 second)."""
    t = np.arange(n)
    return ((t >> 5) & 1) == h


def _fields(e):
    """The 21-bit integers behind points drawn with R_s = 1 (exact)."""
    a = (e + 1.0) * 2.0 ** 20 - 0.5
    ai = np.rint(a)
    assert np.all(ai == a)
    return ai.astype(np.int64)


def test_s21_map_is_exact_and_symmetric(oracle):
    top = 2 ** 21 - 1
    assert oracle.s21(0) == -1.0 + 2.0 ** -21
    assert oracle.s21(top) == 1.0 - 2.0 ** -21
    for a in (0, 1, 12345, 2 ** 20 - 1, 2 ** 20, top):
        x = oracle.s21(a)
        assert oracle.s21(top - a) == -x
        assert float(np.float32(x)) == x          # representable in FP32


def test_every_bit_of_both_halves_is_fair(oracle):
    e = oracle.paired_points(1.0, N_ATT, seed=11, sweep=3, tag=5)
    a = _fields(e)
    for h in (0, 1):
        half = a[_half(len(a), h)]
        bits = (half[:, :, None] >> np.arange(21)) & 1
        mean = bits.mean(axis=0)
        n = half.shape[0]
        assert np.all(np.abs(mean - 0.5) < 5.0 * 0.5 / math.sqrt(n)), (h, mean)


def test_coordinates_uniform_and_uncorrelated(oracle):
    e = oracle.paired_points(0.7, N_ATT, seed=2, sweep=9, tag=77)
    for col in range(3):
        for h in (0, 1):
            x = e[_half(len(e), h), col] / 0.7
            assert stats.kstest(x, "uniform", args=(-1.0, 2.0)).pvalue > 1e-3
    # the two halves of one call: attempt t and t + 32 in each block of 64
    blocks = len(e) // 64
    b = e[:blocks * 64].reshape(blocks, 2, 32, 3)
    h0, h1 = b[:, 0].reshape(-1, 3), b[:, 1].reshape(-1, 3)
    lim = 5.0 / math.sqrt(h0.shape[0])
    for i in range(3):
        for j in range(3):
            assert abs(np.corrcoef(h0[:, i], h1[:, j])[0, 1]) < lim, (i, j)
            if i != j:
                assert abs(np.corrcoef(h0[:, i], h0[:, j])[0, 1]) < lim
                assert abs(np.corrcoef(h1[:, i], h1[:, j])[0, 1]) < lim


def test_points_in_the_ball_are_uniform(oracle):
    R = 0.575
    e = oracle.paired_points(R, N_ATT, seed=7, sweep=1, tag=2)
    r2 = (e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1]) + e[:, 2] * e[:, 2]
    inside = r2 < R * R
    p = math.pi / 6.0
    n = len(r2)
    assert abs(inside.mean() - p) < 5.0 * math.sqrt(p * (1 - p) / n)
    r = np.sqrt(r2[inside]) / R
    assert stats.kstest(r ** 3, "uniform").pvalue > 1e-3
    u = e[inside] / (np.sqrt(r2[inside])[:, None])
    for col in range(3):                     # isotropic: each direction cosine U(-1, 1)
        assert stats.kstest(u[:, col], "uniform", args=(-1.0, 2.0)).pvalue > 1e-3
    # both halves accepted alike
    a0, a1 = inside[_half(n, 0)].mean(), inside[_half(n, 1)].mean()
    assert abs(a0 - a1) < 5.0 * math.sqrt(2 * p * (1 - p) / (n / 2))
