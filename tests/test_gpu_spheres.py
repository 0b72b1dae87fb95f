"""GPU parity of the sphere path against the oracle, through the C-ABI.

Decisions (all trajectory counters) and positions must be bit-identical: both
sides implement the same specification with correctly rounded FP64 and no
contraction.  Sizes span several CTAs/tiles and ragged (empty, crowded)
cells; the full-size 16384-sphere system is checked on its first sweeps."""
import numpy as np
import pytest

from paper_1508_07077_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07077_gb300 import build, hpmc
    build.build()
    hpmc.load()
    return hpmc


PRECISIONS = [0, 1]   # HPMC_FP64, HPMC_FP32_RECHECK


def _compare(oracle, lib, s, sweeps, *, n_trial=0, d_max=0.05, warps=1, schedule=1, n_cell=0,
             seed=1, precision=0, sweep0=0, margin=0.0):
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, n_trial=n_trial, d_max=d_max,
                      seed=seed, warps=warps, schedule=schedule, n_cell=n_cell,
                      precision=precision)
    if margin:
        lib.hpmc_set_fp32_margin(smp.ctx, margin)
    if sweep0:
        lib.hpmc_set_state(smp.ctx, s.pos, None, sweep0)
    smp.sweep(sweeps)
    pos, _, sweep, cnt = smp.state()
    smp.close()
    ref, _, rc, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, n_trial=n_trial, d_max=d_max,
                               seed=seed, n_cell=n_cell, n_sweeps=sweeps, sweep0=sweep0)
    assert sweep == sweep0 + sweeps
    for k in oracle.PARITY_COUNTERS:
        assert cnt[k] == rc[k], (k, cnt[k], rc[k])
    assert np.array_equal(pos, ref)
    return cnt


def test_cell_list_matches_oracle(oracle, lib):
    for s in (W.spheres_256(), W.spheres_16384(0.2)):
        nc = oracle.auto_cells(s.L, 0.5, s.q)
        pos = torch.tensor(s.pos, device="cuda")
        start = torch.empty(nc ** 3 + 1, dtype=torch.int32, device="cuda")
        idx = torch.empty(s.n, dtype=torch.int32, device="cuda")
        for sweep in (0, 7, 1234):
            lib.hpmc_cell_list(s.n, s.L, nc, pos, 1, 0, sweep, start, idx)
            torch.cuda.synchronize()
            rs, ri = oracle.cell_list(s.pos, s.L, nc, 1, 0, sweep)
            assert np.array_equal(start.cpu().numpy(), rs)
            assert np.array_equal(idx.cpu().numpy(), ri)


def test_cell_list_empty_and_single(oracle, lib):
    start = torch.empty(4 ** 3 + 1, dtype=torch.int32, device="cuda")
    idx = torch.empty(1, dtype=torch.int32, device="cuda")
    pos = torch.tensor([[0.3, 4.9, 2.0]], dtype=torch.float64, device="cuda")
    lib.hpmc_cell_list(1, 5.0, 4, pos, 3, 1, 9, start, idx)
    rs, ri = oracle.cell_list(pos.cpu().numpy(), 5.0, 4, 3, 1, 9)
    assert np.array_equal(start.cpu().numpy(), rs) and np.array_equal(idx.cpu().numpy(), ri)
    lib.hpmc_cell_list(0, 5.0, 4, pos, 3, 1, 9, start, idx)
    assert int(start.cpu().numpy().max()) == 0


@pytest.mark.parametrize("precision", PRECISIONS)
def test_spheres_256_plain_100_sweeps(oracle, lib, precision):
    """The 256-sphere system (phi .2, q .2, eta .2), max displacement 0.1, all
    100 sweeps, n_trial = 0: bit-identical trajectory."""
    cnt = _compare(oracle, lib, W.spheres_256(), 100, d_max=0.1, precision=precision)
    assert cnt["reject_depletant"] > 0 and cnt["accept"] > 0


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n_trial", [1, 4])
def test_spheres_256_configurational_bias(oracle, lib, n_trial, precision):
    cnt = _compare(oracle, lib, W.spheres_256(), 25, n_trial=n_trial, d_max=0.08,
                   precision=precision)
    assert cnt["reject_cb"] > 0 and cnt["reject_depletant"] == 0


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("warps", [1, 4])
def test_many_reinsertion_trials(oracle, lib, warps, precision):
    """n_trial = 40: a warp takes each CB factor's trial streams in several
    passes of 32 attempts (the first n_trial in-ball attempts by rank)."""
    cnt = _compare(oracle, lib, W.spheres_256(seed=6), 10, n_trial=40, d_max=0.08, warps=warps,
                   precision=precision)
    assert cnt["reject_cb"] > 0 and cnt["accept"] > 0


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("warps,schedule", [(1, 1), (1, 0), (3, 1), (8, 1), (8, 0)])
def test_launch_shape_does_not_change_results(oracle, lib, warps, schedule, precision):
    for n_trial in (0, 2):
        _compare(oracle, lib, W.spheres_256(), 10, warps=warps, schedule=schedule, n_trial=n_trial,
                 precision=precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_tiny_box_two_cells(oracle, lib, precision):
    """n_c = 2: the 27-cell stencil collapses to 8 distinct cells."""
    pos = W.tiny_spheres(8, 2.6)
    s = W.System("tiny", W.SPHERE, 8, 2.6, 0.2, 30.0, pos, None)
    _compare(oracle, lib, s, 40, d_max=0.08, precision=precision)
    _compare(oracle, lib, s, 20, d_max=0.08, n_trial=3, precision=precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_explicit_cell_count_and_resume_index(oracle, lib, precision):
    s = W.spheres_256()
    _compare(oracle, lib, s, 12, n_cell=4, d_max=0.1, precision=precision)
    _compare(oracle, lib, s, 12, d_max=0.1, sweep0=5000, precision=precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_zero_fugacity_and_zero_step(oracle, lib, precision):
    s = W.spheres_256()
    s0 = W.System("hs", W.SPHERE, s.n, s.L, s.q, 0.0, s.pos, None)
    _compare(oracle, lib, s0, 30, d_max=0.1, precision=precision)
    cnt = _compare(oracle, lib, s, 3, d_max=0.0, precision=precision)
    assert cnt["reject_cell"] == 0


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("eta", [0.1, 0.4])
def test_spheres_16384_first_sweeps(oracle, lib, eta, precision):
    """Full-size 16384-sphere system (phi .3, q .15): first sweeps bit-exact."""
    _compare(oracle, lib, W.spheres_16384(eta), 3, d_max=0.05, precision=precision)


@pytest.mark.parametrize("n_trial", [0, 3])
def test_fp32_recheck_path_is_exact(oracle, lib, n_trial):
    """With a margin of 1 nearly every FP32 decision is re-taken in FP64; the
    trajectory must not change, and the recheck counter shows the path ran."""
    cnt = _compare(oracle, lib, W.spheres_256(), 8, d_max=0.08, n_trial=n_trial,
                   precision=1, margin=1.0)
    assert cnt["rechecks"] > 10 * cnt["dep_evaluated"] // 20


def test_fp32_margin_below_bound_rejected(lib):
    s = W.spheres_256()
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, precision=1)
    lib.hpmc_set_fp32_margin(smp.ctx, 1e-9)
    with pytest.raises(lib.HPMCError):
        smp.sweep(1)
    smp.close()


@pytest.mark.parametrize("schedule,phase_launches", [(0, 8), (1, 1)])
def test_timing_mode_counts_launches(lib, schedule, phase_launches):
    """Eight colour-phase launches per sweep, or one persistent launch."""
    s = W.spheres_256()
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, precision=1, schedule=schedule)
    smp.sweep(1)
    lib.hpmc_set_timing(smp.ctx, True)
    smp.sweep(3)
    ms, n = lib.hpmc_get_timing(smp.ctx)
    smp.close()
    assert n == [3, 3 * phase_launches, 3] and ms[0] > 0 and ms[1] > 0 and ms[2] > 0


def test_resume_and_device_io(oracle, lib):
    s = W.spheres_256()
    a = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.05)
    a.sweep(10)
    pa, _, _, _ = a.state()
    a.close()
    b = lib.Sampler(torch.tensor(s.pos, device="cuda"), s.L, q=s.q, n_r=s.n_r, d_max=0.05)
    b.sweep(5)
    mid = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
    sweep, _ = lib.hpmc_get_state(b.ctx, mid)
    b.close()
    c = lib.Sampler(mid, s.L, q=s.q, n_r=s.n_r, d_max=0.05)
    lib.hpmc_set_state(c.ctx, mid, None, sweep)
    c.sweep(5)
    pc, _, sw, _ = c.state()
    c.close()
    assert sw == 10 and np.array_equal(pa, pc)


def test_errors_are_reported(lib):
    s = W.spheres_256()
    bad = s.pos.copy()
    bad[1] = bad[0] + np.array([0.3, 0.0, 0.0])
    bad[1] %= s.L
    smp = lib.Sampler(bad, s.L, q=s.q, n_r=s.n_r)
    with pytest.raises(lib.HPMCError) as e:
        smp.sweep(1)
    assert e.value.code == -2
    smp.close()
    with pytest.raises(lib.HPMCError):
        lib.Sampler(s.pos, s.L, q=s.q, n_r=1e7).sweep(1)  # lambda beyond the table
    with pytest.raises(lib.HPMCError):
        lib.Sampler(s.pos, 1.5, q=s.q, n_r=1.0).sweep(1)  # box smaller than two cells


@pytest.mark.parametrize("precision", PRECISIONS)
def test_configuration_check_finds_a_pair_in_any_direction(lib, precision):
    """The start check finds one overlapping pair wherever its partner sits
    relative to the colloid (the FP32 check tests each pair from one side:
    the own cell and the stencil cells after it), in a box of six cells per
    side and in one of two cells per side (the whole box is the stencil)."""
    rng = np.random.default_rng(21)
    for L, base in ((None, None), (2.6, W.tiny_spheres(8, 2.6))):
        if base is None:
            s = W.spheres_256(seed=5)
            base, L, q, n_r = s.pos, s.L, s.q, s.n_r
        else:
            q, n_r = 0.2, 30.0
        for trial in range(12):
            pos = base.copy()
            i, j = rng.choice(len(pos), size=2, replace=False)
            u = rng.normal(size=3)
            pos[j] = (pos[i] + 0.9 * u / np.linalg.norm(u)) % L
            smp = lib.Sampler(pos, L, q=q, n_r=n_r, d_max=0.05, precision=precision)
            with pytest.raises(lib.HPMCError) as e:
                smp.sweep(1)
            assert e.value.code == -2, (L, trial)
            smp.close()
        # and the unmodified configuration passes
        smp = lib.Sampler(base, L, q=q, n_r=n_r, d_max=0.05, precision=precision)
        smp.sweep(1)
        smp.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_configuration_check_at_contact(oracle, lib, precision):
    """The start check: a pair closer than contact (by 1e-12) is an overlap,
    one at contact (by 1e-12) is not; a position outside the box is an
    argument error.  The FP32 form decides such pairs in FP64."""
    s = W.spheres_256(seed=8)
    for gap, code in ((-1e-12, -2), (1e-12, 0)):
        pos = s.pos.copy()
        d = np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0)
        pos[1] = (pos[0] + (1.0 + gap) * d) % s.L
        # keep the pair clear of every other sphere
        far = np.linalg.norm(((pos[2:] - pos[0] + s.L / 2) % s.L) - s.L / 2, axis=1)
        keep = np.concatenate([[True, True], far > 2.2])
        pos = pos[keep]
        smp = lib.Sampler(pos, s.L, q=s.q, n_r=s.n_r, precision=precision)
        if code:
            with pytest.raises(lib.HPMCError) as e:
                smp.sweep(1)
            assert e.value.code == code
        else:
            smp.sweep(1)
            p, _, _, c = smp.state()
            ref, _, rc, _ = oracle.run(pos, s.L, q=s.q, n_r=s.n_r, n_sweeps=1)
            assert np.array_equal(p, ref)
        smp.close()
    pos = s.pos.copy()
    pos[3, 1] = s.L
    smp = lib.Sampler(pos, s.L, q=s.q, n_r=s.n_r, precision=precision)
    with pytest.raises(lib.HPMCError) as e:
        smp.sweep(1)
    assert e.value.code == -1
    smp.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_uploaded_state_is_checked(oracle, lib, precision):
    """hpmc_set_state checks the uploaded configuration in its own round trip:
    an overlap (or a position outside the box) is reported by every following
    sweep until a valid state replaces it; a valid upload continues the
    oracle's trajectory."""
    s = W.spheres_256(seed=9)
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.05, precision=precision)
    smp.sweep(2)
    good, _, sweep, _ = smp.state()
    bad = good.copy()
    bad[1] = (bad[0] + np.array([0.0, 0.4, 0.0])) % s.L
    outside = good.copy()
    outside[5, 2] = s.L
    for pos, code in ((bad, -2), (outside, -1)):
        lib.hpmc_set_state(smp.ctx, pos, None, sweep)
        for _ in range(2):
            with pytest.raises(lib.HPMCError) as e:
                smp.sweep(1)
            assert e.value.code == code
    lib.hpmc_set_state(smp.ctx, good, None, sweep)
    smp.sweep(3)
    p, _, sw, _ = smp.state()
    smp.close()
    ref, _, _, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.05, n_sweeps=5)
    assert sw == 5 and np.array_equal(p, ref)


def test_pinned_host_buffers_in_place(oracle, lib):
    """Pinned host buffers are read and written by the device in place (no
    staging copy): the same state and trajectory as through pageable ones;
    a buffer of the wrong length is refused before any device access."""
    s = W.spheres_256(seed=10)
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.05)
    smp.sweep(2)
    pageable = np.empty((s.n, 3))
    pinned = torch.empty((s.n, 3), dtype=torch.float64).pin_memory().numpy()
    sweep, _ = lib.hpmc_get_state(smp.ctx, pageable)
    lib.hpmc_get_state(smp.ctx, pinned)
    assert np.array_equal(pageable, pinned)
    lib.hpmc_set_state(smp.ctx, pinned, None, sweep)
    smp.sweep(3)
    p, _, sw, _ = smp.state()
    for bad in (np.zeros((s.n - 1, 3)), torch.zeros((s.n + 1, 3), dtype=torch.float64).pin_memory()):
        with pytest.raises(ValueError):
            lib.hpmc_set_state(smp.ctx, bad, None, sweep)
        with pytest.raises(ValueError):
            lib.hpmc_get_state(smp.ctx, bad)
    smp.close()
    ref, _, _, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.05, n_sweeps=5)
    assert sw == 5 and np.array_equal(p, ref)
