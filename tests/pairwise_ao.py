"""Independent reference for the many-body reduction pin (test helper, not a
test module).

For spheres with q < 2/sqrt(3) - 1 no point lies in three excluded spheres of
radius R_s = (1 + q)/2, so the free volume of a configuration is V minus the
excluded spheres plus their pairwise lens overlaps, and the implicit-depletant
weight exp(z_p V_f) is exactly that of the pairwise Asakura-Oosawa potential
beta U(r) = -z_p V_lens(r) (hard core below r = 1).  This module samples that
pair potential with a plain Metropolis chain (numpy, many independent replicas
moved together) and shares nothing with the oracle or the library: both are
compared against it through the pair counts near contact.
"""
import math

import numpy as np

from paper_1508_07077_gb300 import workloads as W

# 32 spheres at phi = 0.2, q = 0.15 (below 2/sqrt(3) - 1 = 0.1547), eta_r = 0.05:
# z_p = 28.3, beta U(1) = -0.55
N, PHI, Q, ETA = 32, 0.2, 0.15, 0.05
BINS, RMAX, LO = 24, 1.2, 20     # the histogram's bins of 0.05; LO.. run from contact to 1.2
GROUPS = 16                      # independent groups of chains on each side
CHI2_999 = 18.47                 # 0.999 quantile of chi^2 with BINS - LO = 4 degrees of freedom


def system():
    """(box length, z_p, the common fcc start)."""
    L = (N * math.pi / 6.0 / PHI) ** (1.0 / 3.0)
    z_p = 6.0 * ETA / (math.pi * Q ** 3)
    return L, z_p, W.fcc_positions(N, L, 1)


def lens(r, R):
    """Overlap volume of two spheres of radius R at centre distance r."""
    r = np.asarray(r, dtype=float)
    return np.where(r < 2 * R, math.pi / 12.0 * (4 * R + r) * (2 * R - r) ** 2, 0.0)


def pairwise_counts(n_rep=32, n_eq=400, n_run=1600, d_max=0.08, seed=7):
    """Pair counts per colloid and sample in the bins from contact to RMAX,
    one row per group of replicas (GROUPS rows), from a Metropolis chain of
    the pairwise AO potential: single-colloid cube moves, every colloid in
    turn, minimum image."""
    L, z_p, pos0 = system()
    R_s = 0.5 + Q / 2.0
    rng = np.random.default_rng(seed)
    X = np.repeat(pos0[None], n_rep, axis=0).copy()
    edges = np.linspace(0.0, RMAX, BINS + 1)[LO:]
    iu = np.triu_indices(N, 1)
    H = np.zeros((n_rep, BINS - LO))
    samples = 0
    for sweep in range(n_eq + n_run):
        for i in range(N):
            xo = X[:, i, :]
            xn = xo + rng.uniform(-d_max, d_max, size=(n_rep, 3))
            do = X - xo[:, None, :]
            do -= L * np.round(do / L)
            dn = X - xn[:, None, :]
            dn -= L * np.round(dn / L)
            ro = np.sqrt((do ** 2).sum(-1))
            rn = np.sqrt((dn ** 2).sum(-1))
            ro[:, i] = np.inf
            rn[:, i] = np.inf
            dU = -z_p * (lens(rn, R_s).sum(1) - lens(ro, R_s).sum(1))
            ok = ~(rn < 1.0).any(1) & (rng.random(n_rep) < np.exp(-dU))
            X[ok, i, :] = xn[ok] % L
        if sweep >= n_eq and sweep % 2 == 0:
            d = X[:, :, None, :] - X[:, None, :, :]
            d -= L * np.round(d / L)
            r = np.sqrt((d ** 2).sum(-1))[:, iu[0], iu[1]]
            for b in range(BINS - LO):
                H[:, b] += ((r >= edges[b]) & (r < edges[b + 1])).sum(1)
            samples += 1
    H /= samples * N
    return H.reshape(GROUPS, -1, BINS - LO).mean(1)


def chi2(a, b):
    """chi^2 over the bins of the difference of two sets of independent group
    means (rows), with the z score of each bin."""
    z = (a.mean(0) - b.mean(0)) / np.sqrt(a.var(0, ddof=1) / len(a) + b.var(0, ddof=1) / len(b))
    return float(np.sum(z ** 2)), z
