"""Long runs of the CUDA path (FP32 certified form unless stated) against what
statistical mechanics and the oracle fix, with many independent replica
chains advanced together in one batch.

* The two-colloid Asakura-Oosawa distribution (Sec. III.A, Eq. 2; the
  semigrand weight exp(z_p V_f) of two spheres): the separation density for
  r < L/2 is proportional to r^2 exp(z_p V_lens(r)).  Checked without and
  with configurational bias (Sec. III.D, Eq. 12), whose weight must leave the
  distribution unchanged.
* The hard-sphere limit z_p = 0: the pressure from the contact value,
  Z = 1 + 4 phi g(1+), against Carnahan-Starling at phi = 0.2 and 0.3.
* The many-body reduction: 32 spheres at q = 0.15 (below 2/sqrt(3) - 1, where
  no point lies in three excluded spheres) sample the pairwise
  Asakura-Oosawa fluid; pair counts near contact against an independent
  Metropolis chain of that pair potential (tests/pairwise_ao.py).
* The state point of the 16384-sphere workload (phi_c 0.30, q 0.15, eta_r 0.2)
  at a size the oracle runs in seconds: acceptance rate and g(r) of
  independent GPU chains against independent oracle chains; the acceptance
  errors by Flyvbjerg-Petersen blocking of each chain's series, the g(r)
  errors from the spread over the independent chains.
* Bit-exact trajectories at the benchmark's own (small, tuned) step sizes on
  the full-size systems: the four 16384-sphere state points for 10 sweeps and
  the 128-replica batch for 3 sweeps.

Every chain is seeded, so each test is deterministic."""
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import pairwise_ao as PA
from paper_1508_07077_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

THREADS = max(1, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07077_gb300 import build, hpmc
    build.build()
    hpmc.load()
    return hpmc


def fp_error(x, min_blocks=16):
    """Flyvbjerg-Petersen blocking: standard error of the mean of a correlated
    series.  The series is halved by pairwise averaging while at least
    min_blocks blocks remain; the largest per-level estimate is returned
    (the plateau, or its conservative bound when the plateau is not reached)."""
    x = np.asarray(x, dtype=float)
    best = 0.0
    while len(x) >= min_blocks:
        n = len(x)
        best = max(best, float(x.std(ddof=1)) / math.sqrt(n))
        m = n // 2
        x = 0.5 * (x[0:2 * m:2] + x[1:2 * m:2])
    return best


def _min_image(d, L):
    return d - L * np.round(d / L)


# --- two colloids: the Asakura-Oosawa distribution ---------------------------

Q, R_S, Z_P, L2 = 0.2, 0.6, 47.7464829275686, 2.4


def _lens(r, R=R_S):
    r = np.asarray(r, dtype=float)
    return np.where(r < 2 * R, math.pi / 12.0 * (4 * R + r) * (2 * R - r) ** 2, 0.0)


def _pairs(m, seed):
    """m non-overlapping sphere pairs, uniform in the box."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < m:
        a, b = rng.uniform(0.0, L2, size=(2, 3))
        d = _min_image(b - a, L2)
        if d @ d >= 1.0:
            out.append(np.array([a, b]))
    return out


@pytest.mark.parametrize("precision,n_trial", [(1, 0), (1, 5), (0, 0)])
def test_asakura_oosawa_pair_distribution_long_run(lib, precision, n_trial):
    # the pair separation relaxes over the box in ~10^3 sweeps at this step
    # size: 5000 sweeps of burn-in from uniform starts, then 40000 sweeps
    m, groups = 2048, 32
    burn, sweeps, every = 5000, 40000, 20
    bins, lo, hi = 8, 1.0, 1.2            # contact to L/2
    starts = _pairs(m, seed=17 + n_trial)
    reps = [{"n": 2, "box_l": L2, "pos": p, "q": Q, "n_r": Z_P, "n_trial": n_trial,
             "d_max": 0.08, "replica": k, "n_cell": 2} for k, p in enumerate(starts)]
    ctx = lib.hpmc_init_batch(reps, seed=3, precision=precision)
    try:
        lib.hpmc_sweep(ctx, burn)
        buf = np.empty((2 * m, 3))
        hist = np.zeros((m, bins))
        for _ in range(sweeps // every):
            lib.hpmc_sweep(ctx, every)
            lib.hpmc_get_state(ctx, buf)
            p = buf.reshape(m, 2, 3)
            d = _min_image(p[:, 1] - p[:, 0], L2)
            r = np.sqrt((d * d).sum(1))
            k = np.floor((r - lo) / (hi - lo) * bins).astype(int)
            ok = (k >= 0) & (k < bins)
            np.add.at(hist, (np.nonzero(ok)[0], k[ok]), 1.0)
        _, cnt = lib.hpmc_get_state(ctx)
    finally:
        lib.hpmc_destroy(ctx)
    assert cnt["moves"] == 2 * m * (burn + sweeps)
    if n_trial:
        assert cnt["cb_fwd_ok"] > 0 and cnt["reject_cb"] > 0
    edges = np.linspace(lo, hi, bins + 1)
    expect = []
    for b in range(bins):
        r = np.linspace(edges[b], edges[b + 1], 401)
        expect.append(np.trapezoid(r ** 2 * np.exp(Z_P * _lens(r)), r))
    expect = np.array(expect) / np.sum(expect)
    g = hist.reshape(groups, m // groups, bins).sum(1)
    g = g / g.sum(1, keepdims=True)
    mean, se = g.mean(0), g.std(0, ddof=1) / math.sqrt(groups)
    z = (mean - expect) / se
    assert np.all(np.abs(z) < 4.0), z
    # the test has power: the r^2-only law (no depletion attraction) is far off
    r2 = np.diff(edges ** 3)
    r2 = r2 / r2.sum()
    assert np.max(np.abs(mean - r2) / se) > 20.0


# --- hard-sphere limit: Carnahan-Starling -----------------------------------

def _pair_hist_device(pos, m, n, L, edges_t):
    """Histogram over all pairs of every replica (on the device)."""
    p = pos.view(m, n, 3)
    d = p[:, :, None, :] - p[:, None, :, :]
    d = d - L * torch.round(d / L)
    r = torch.sqrt((d * d).sum(-1))
    iu = torch.triu_indices(n, n, 1, device=p.device)
    r = r[:, iu[0], iu[1]]
    out = torch.zeros((m, len(edges_t) - 1), dtype=torch.float64, device=p.device)
    k = torch.bucketize(r, edges_t, right=True) - 1
    ok = (k >= 0) & (k < len(edges_t) - 1)
    rows = torch.arange(m, device=p.device)[:, None].expand_as(k)
    out.index_put_((rows[ok], k[ok]), torch.ones_like(r[ok]), accumulate=True)
    return out


@pytest.mark.parametrize("phi", [0.2, 0.3])
def test_hard_sphere_pressure_carnahan_starling_long_run(lib, phi):
    n, m, groups = 256, 64, 16
    burn, sweeps, every = 1000, 4000, 10
    systems = [W.make_system("hs", W.SPHERE, n, phi, 0.2, 0.0, seed=2, replica=k)
               for k in range(m)]
    L = systems[0].L
    reps = [{"n": n, "box_l": L, "pos": s.pos, "q": 0.2, "n_r": 0.0, "d_max": 0.1,
             "replica": k} for k, s in enumerate(systems)]
    ctx = lib.hpmc_init_batch(reps, seed=2, precision=1)
    rmax, width = 1.30, 0.01
    edges = np.arange(0.0, rmax + 0.5 * width, width)
    edges_t = torch.tensor(edges, device="cuda")
    pos = torch.empty((m * n, 3), dtype=torch.float64, device="cuda")
    hist = torch.zeros((m, len(edges) - 1), dtype=torch.float64, device="cuda")
    try:
        lib.hpmc_sweep(ctx, burn)
        for _ in range(sweeps // every):
            lib.hpmc_sweep(ctx, every)
            lib.hpmc_get_state(ctx, pos)
            hist += _pair_hist_device(pos, m, n, L, edges_t)
        _, cnt = lib.hpmc_get_state(ctx)
    finally:
        lib.hpmc_destroy(ctx)
    acc = cnt["accept"] / cnt["moves"]
    assert 0.1 < acc < 0.9
    h = hist.cpu().numpy().reshape(groups, m // groups, -1).sum(1)
    samples = sweeps // every * (m // groups)
    rho = n / L ** 3
    shell = 4.0 * math.pi / 3.0 * (edges[1:] ** 3 - edges[:-1] ** 3)
    g = h / (samples * n / 2.0 * rho * shell)
    mid = 0.5 * (edges[1:] + edges[:-1])
    assert np.all(h[:, mid < 1.0] == 0)          # hard cores never overlap
    sel = (mid > 1.0) & (mid < 1.08)
    g1 = np.array([np.polyval(np.polyfit(mid[sel], gk[sel], 2), 1.0) for gk in g])
    Z = 1.0 + 4.0 * phi * g1
    z_mean, z_se = Z.mean(), Z.std(ddof=1) / math.sqrt(groups)
    z_cs = (1 + phi + phi ** 2 - phi ** 3) / (1 - phi) ** 3
    # statistical error plus 0.5% for the contact extrapolation and N = 256
    # (the oracle's own chains, binned every sweep, land within 0.15%)
    assert abs(z_mean - z_cs) < 3.0 * z_se + 0.005 * z_cs, (z_mean, z_se, z_cs)


# --- many-body reduction: the pairwise Asakura-Oosawa fluid -----------------

@pytest.fixture(scope="module")
def pairwise_reference():
    return PA.pairwise_counts()


@pytest.mark.parametrize("precision", [1, 0])
def test_many_body_reduction_to_pairwise_ao_long_run(lib, pairwise_reference, precision):
    """32 spheres at q = 0.15, below 2/sqrt(3) - 1, where the implicit model is
    exactly the pairwise Asakura-Oosawa fluid: the pair counts from contact to
    r = 1.2 of 64 independent CUDA chains (FP32 certified form and plain FP64,
    16 groups of 4) against a Metropolis chain of the pair potential that
    shares nothing with the library (chi^2 of the four bins below its 0.999
    quantile)."""
    L, z_p, pos0 = PA.system()
    m, n = 64, PA.N
    burn, sweeps, every = 4000, 12000, 10
    reps = [{"n": n, "box_l": L, "pos": pos0, "q": PA.Q, "n_r": z_p, "d_max": 0.03,
             "replica": k} for k in range(m)]
    ctx = lib.hpmc_init_batch(reps, seed=5, precision=precision)
    edges_t = torch.tensor(np.linspace(0.0, PA.RMAX, PA.BINS + 1)[PA.LO:], device="cuda")
    pos = torch.empty((m * n, 3), dtype=torch.float64, device="cuda")
    hist = torch.zeros((m, PA.BINS - PA.LO), dtype=torch.float64, device="cuda")
    try:
        lib.hpmc_sweep(ctx, burn)
        for _ in range(sweeps // every):
            lib.hpmc_sweep(ctx, every)
            lib.hpmc_get_state(ctx, pos)
            hist += _pair_hist_device(pos, m, n, L, edges_t)
        _, cnt = lib.hpmc_get_state(ctx)
    finally:
        lib.hpmc_destroy(ctx)
    assert cnt["moves"] == m * n * (burn + sweeps)
    got = hist.cpu().numpy() / (sweeps // every * n)
    got = got.reshape(PA.GROUPS, m // PA.GROUPS, -1).mean(1)
    chi2, z = PA.chi2(got, pairwise_reference)
    assert chi2 < PA.CHI2_999, z


# --- the 16384-sphere state point: GPU chains against oracle chains ----------

PHI2, Q2, ETA2, D2 = 0.30, 0.15, 0.2, 0.0112


def _chain_series(pos_blocks, counts, L, edges):
    """Per block: acceptance and the pair histogram of the block's end state
    (pair distances binned on the device)."""
    acc = np.array([a / mv for a, mv in counts])
    edges_t = torch.tensor(edges, device="cuda")
    hs = []
    for p in pos_blocks:
        pt = torch.tensor(p, device="cuda")
        n = pt.shape[0]
        hs.append(_pair_hist_device(pt, 1, n, L, edges_t)[0].cpu().numpy())
    return acc, np.array(hs)


def test_state_point_statistics_against_oracle(lib, oracle):
    n, m_gpu, m_or = 1024, 32, 16
    burn, blocks, every = 200, 60, 10
    edges = np.arange(0.9, 2.5 + 1e-9, 0.04)

    def system(k):
        return W.make_system("sp", W.SPHERE, n, PHI2, Q2, ETA2, seed=5, replica=k)

    L = system(0).L
    # GPU: m_gpu chains (keys 0..), one batch
    gs = [system(k) for k in range(m_gpu)]
    reps = [{"n": n, "box_l": L, "pos": s.pos, "q": Q2, "n_r": s.n_r, "d_max": D2,
             "replica": k} for k, s in enumerate(gs)]
    ctx = lib.hpmc_init_batch(reps, seed=5, precision=1)
    g_acc, g_hist = [[] for _ in range(m_gpu)], [[] for _ in range(m_gpu)]
    try:
        lib.hpmc_sweep(ctx, burn)
        buf = np.empty((m_gpu * n, 3))
        prev = [lib.hpmc_get_replica(ctx, k, n)[2] for k in range(m_gpu)]
        for _ in range(blocks):
            lib.hpmc_sweep(ctx, every)
            lib.hpmc_get_state(ctx, buf)
            for k in range(m_gpu):
                c = lib.hpmc_get_replica(ctx, k, n)[2]
                g_acc[k].append((c["accept"] - prev[k]["accept"], c["moves"] - prev[k]["moves"]))
                g_hist[k].append(buf[k * n:(k + 1) * n].copy())
                prev[k] = c
    finally:
        lib.hpmc_destroy(ctx)

    # oracle: m_or independent chains (keys 1000..), run in parallel threads
    def oracle_chain(k):
        s = system(1000 + k)
        pos, _, _, _ = oracle.run(s.pos, L, q=Q2, n_r=s.n_r, d_max=D2, seed=5,
                                  replica=1000 + k, n_sweeps=burn)
        counts, states = [], []
        for b in range(blocks):
            pos, _, c, _ = oracle.run(pos, L, q=Q2, n_r=s.n_r, d_max=D2, seed=5,
                                      replica=1000 + k, sweep0=burn + b * every,
                                      n_sweeps=every)
            counts.append((c["accept"], c["moves"]))
            states.append(pos.copy())
        return counts, states

    with ThreadPoolExecutor(max_workers=min(THREADS, m_or)) as ex:
        ochains = list(ex.map(oracle_chain, range(m_or)))

    def summarise(chains):
        accs, ses, hists = [], [], []
        for counts, states in chains:
            a, h = _chain_series(states, counts, L, edges)
            accs.append(a.mean())
            ses.append(fp_error(a))
            hists.append(h)
        return np.array(accs), np.array(ses), np.array(hists)

    ga, gse, gh = summarise(list(zip(g_acc, g_hist)))
    oa, ose, oh = summarise(ochains)
    # acceptance: mean over chains; the error of each chain's mean by
    # blocking, combined over the (independent) chains
    g_mean, g_err = ga.mean(), math.sqrt(np.sum(gse ** 2)) / m_gpu
    o_mean, o_err = oa.mean(), math.sqrt(np.sum(ose ** 2)) / m_or
    sigma = math.sqrt(g_err ** 2 + o_err ** 2)
    assert 0.15 < g_mean < 0.5
    assert abs(g_mean - o_mean) < 2.0 * sigma, (g_mean, o_mean, sigma)
    # g(r): every bin; the chains are independent, so the error of the mean
    # over chains follows from the spread of the chain means
    def bin_stats(hs, nchain):
        per_chain = hs.mean(axis=1)
        return per_chain.mean(axis=0), per_chain.std(axis=0, ddof=1) / math.sqrt(nchain)

    gm, ge = bin_stats(gh, m_gpu)
    om, oe = bin_stats(oh, m_or)
    live = (ge > 0) & (oe > 0)
    z = (gm - om)[live] / np.sqrt(ge ** 2 + oe ** 2)[live]
    assert np.mean(np.abs(z) < 2.0) >= 0.85, z
    assert np.all(np.abs(z) < 5.0), z
    # the histogram starts at contact (no overlaps) and shows the first shell
    mid = 0.5 * (edges[1:] + edges[:-1])
    assert np.all(gm[mid < 1.0] == 0) and np.all(om[mid < 1.0] == 0)


# --- bit-exact at the benchmark's step sizes, full size ----------------------

BENCH_DMAX = {0.1: 0.0223, 0.2: 0.0112, 0.3: 0.0075, 0.4: 0.0056}


def test_full_size_spheres_at_benchmark_step_sizes(lib, oracle):
    systems = [W.spheres_16384(eta, seed=1) for eta in BENCH_DMAX]
    reps = [{"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r,
             "d_max": BENCH_DMAX[eta], "replica": k}
            for k, (s, eta) in enumerate(zip(systems, BENCH_DMAX))]
    sweeps = 10
    ctx = lib.hpmc_init_batch(reps, seed=1, precision=1)
    try:
        lib.hpmc_sweep(ctx, sweeps)
        got = [lib.hpmc_get_replica(ctx, k, r["n"]) for k, r in enumerate(reps)]
    finally:
        lib.hpmc_destroy(ctx)
    for k, r in enumerate(reps):
        ref, _, rc, _ = oracle.run(r["pos"], r["box_l"], q=r["q"], n_r=r["n_r"],
                                   d_max=r["d_max"], seed=1, replica=k, n_sweeps=sweeps,
                                   threads=THREADS)
        assert np.array_equal(got[k][0], ref), k
        for name in oracle.PARITY_COUNTERS:
            assert got[k][2][name] == rc[name], (k, name)
        assert rc["accept"] > 0.2 * rc["moves"]


def test_batched_128_replicas_at_small_steps(lib, oracle):
    """The 128-replica workload (N log-uniform in [500, 20000], uneven state
    points) for 3 sweeps at step sizes of the order the benchmark tunes."""
    reps_sys = W.batched_replicas(128, seed=1)
    reps = [{"n": s.n, "box_l": s.L, "pos": s.pos, "q": s.q, "n_r": s.n_r,
             "d_max": 0.004 + 0.02 * (k % 5) / 4.0, "replica": k}
            for k, s in enumerate(reps_sys)]
    sweeps = 3
    ctx = lib.hpmc_init_batch(reps, seed=1, precision=1)
    try:
        lib.hpmc_sweep(ctx, sweeps)
        got = [lib.hpmc_get_replica(ctx, k, r["n"]) for k, r in enumerate(reps)]
    finally:
        lib.hpmc_destroy(ctx)

    def ref(k):
        r = reps[k]
        return oracle.run(r["pos"], r["box_l"], q=r["q"], n_r=r["n_r"], d_max=r["d_max"],
                          seed=1, replica=k, n_sweeps=sweeps)

    with ThreadPoolExecutor(max_workers=THREADS) as ex:
        refs = list(ex.map(ref, range(len(reps))))
    for k in range(len(reps)):
        assert np.array_equal(got[k][0], refs[k][0]), k
        for name in oracle.PARITY_COUNTERS:
            assert got[k][2][name] == refs[k][2][name], (k, name)
