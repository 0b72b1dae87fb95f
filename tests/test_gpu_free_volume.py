"""GPU free-volume measurement (Sec. IV.A observable) against the oracle's
brute-force probe count: same probe stream, same FP64 tests, so the number
of free probes must be identical, for spheres, hemispheres and discoids, at
the start and after sweeps."""
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


@pytest.mark.parametrize("shape,phi,q,eta", [(W.SPHERE, 0.3, 0.15, 0.2),
                                             (W.HEMISPHERE, 0.25, 0.1, 0.3),
                                             (W.SPHEROID, 0.3, 0.1, 0.25)])
@pytest.mark.parametrize("precision", [0, 1])
def test_free_volume_equals_oracle(oracle, lib, shape, phi, q, eta, precision):
    s = W.make_system("fv", shape, 256, phi, q, eta, seed=2)
    smp = lib.Sampler(s.pos, s.L, quat=s.quat, shape=shape, shape_params=s.shape_params, q=q,
                      n_r=s.n_r, d_max=0.05, a_max=0.2 if shape != W.SPHERE else 0.0,
                      p_translate=0.5 if shape != W.SPHERE else 1.0, precision=precision)
    n_probe = 200000
    for k in range(2):
        pos, quat, _, _ = smp.state(with_quat=True)
        for qq in (q, 0.3):
            got, n = lib.hpmc_free_volume(smp.ctx, qq, seed=11, sample=k, n_probe=n_probe)
            ref = oracle.free_volume(pos, s.L, qq, shape=shape, shape_params=s.shape_params,
                                     quat=quat if shape != W.SPHERE else None, seed=11,
                                     sample=k, n_probe=n_probe)
            assert got / float(n) == ref
            assert 0.0 < ref < 1.0
        smp.sweep(3)
    smp.close()


def test_free_volume_many_probes_per_thread(oracle, lib):
    """More probes than resident threads: the grid-stride loop covers them all."""
    s = W.spheres_256()
    smp = lib.Sampler(s.pos, s.L, q=s.q, n_r=s.n_r)
    got, n = lib.hpmc_free_volume(smp.ctx, s.q, seed=3, n_probe=3000000)
    ref = oracle.free_volume(s.pos, s.L, s.q, seed=3, n_probe=3000000)
    assert got / float(n) == ref
    smp.close()
