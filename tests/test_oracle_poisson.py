"""Pins of the Poisson depletant count N_p ~ Poisson(z_p |V_0|) (Sec. III.B
step 2) against the library pmf/cdf and its moments."""
import math

import numpy as np
import pytest
from scipy import stats


@pytest.mark.parametrize("lam", [0.3, 5.0, 43.2, 180.0, 532.0, 699.0])
def test_table_is_the_poisson_cdf(oracle, lam):
    F = oracle.poisson_table(lam)
    k = np.arange(len(F))
    ref = stats.poisson.cdf(k, lam)
    assert np.max(np.abs(F - ref)) < 1e-12
    assert np.all(np.diff(F) >= 0.0)            # monotone: inversion is a count
    assert abs(1.0 - F[-1]) < 1e-13  # rounding of a ~10^3-term sum


def test_zero_mean_draws_nothing(oracle):
    F = oracle.poisson_table(0.0)
    for u in (0.0, 0.5, 1.0 - 2.0 ** -53):
        assert oracle.poisson_sample(F, u) == 0


def test_lambda_is_fugacity_times_sphere_volume(oracle):
    # lambda = z_p (4 pi / 3) R_s^3; e.g. spheres d=1, q=0.2: R_s = 0.6
    assert oracle.poisson_lambda(0.6, 47.7464829275686) == pytest.approx(
        47.7464829275686 * 4.0 / 3.0 * math.pi * 0.216, rel=1e-15)
    assert oracle.poisson_lambda(0.6, 0.0) == 0.0


@pytest.mark.parametrize("lam", [2.5, 43.2, 226.0])
def test_inversion_sampling_moments_and_pmf(oracle, lam):
    F = oracle.poisson_table(lam)
    n = 20000
    rng_words = [oracle.philox([i, 0, 3 << 24, 0], (11, 0)) for i in range(n)]
    draws = np.array([oracle.poisson_sample(F, oracle.u53(w[0], w[1]))
                      for w in rng_words])
    assert abs(draws.mean() - lam) < 5 * math.sqrt(lam / n)
    assert abs(draws.var() / lam - 1.0) < 5 * math.sqrt(2.0 / n)
    lo, hi = int(max(0, lam - 3 * math.sqrt(lam))), int(lam + 3 * math.sqrt(lam))
    edges = np.arange(lo, hi + 1)
    obs = np.array([(draws < lo).sum()] + [(draws == k).sum() for k in edges]
                   + [(draws > hi).sum()])
    pm = stats.poisson.pmf(edges, lam)
    exp = np.concatenate([[stats.poisson.cdf(lo - 1, lam)], pm,
                          [stats.poisson.sf(hi, lam)]]) * n
    keep = exp > 5
    chi2 = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4


def test_exact_boundaries(oracle):
    """u exactly at a table entry counts that entry (strict u < F[k] stops)."""
    F = oracle.poisson_table(4.0)
    assert oracle.poisson_sample(F, F[0]) == 1
    assert oracle.poisson_sample(F, np.nextafter(F[0], 0.0)) == 0
    assert oracle.poisson_sample(F, F[5]) == 6
