"""Seeded synthetic inputs: initial colloid configurations and state points.

This module holds no step of the Monte Carlo method itself.  It is the one
module both the CUDA path and the CPU oracle draw their inputs from, so that
they start from identical configurations.

Workloads mirror the paper's systems (hard spheres in penetrable hard-sphere
depletants, Sec. IV; hemispheres, Sec. V.A; discoids, Sec. V.B) at the sizes
of the benchmark configurations:

* ``spheres_256``      N=256 spheres, phi_c=0.20, q=0.20, eta_r=0.20
* ``spheres_16384``    N=16384 spheres, phi_c=0.30, q=0.15, eta_r in {.1,.2,.3,.4}
* ``hemispheres_32768`` N=32768 hemispheres, phi_c=0.25, q=0.10, eta_r=0.30
* ``discoids_65536``   N=65536 oblate spheroids a=b=0.5, c=0.25, phi_c=0.30,
                       q=0.10, eta_r=0.25
* ``batched_128``      128 sphere replicas, N log-uniform in [500, 20000]

Initial configurations are an fcc lattice with a random subset of sites
occupied and a small random jitter, so they are free of overlaps by
construction at every packing fraction used here (up to 0.45); the sampler
then melts them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SPHERE, HEMISPHERE, SPHEROID = 0, 1, 2

# colloid volume per particle (unit diameter; spheroid a=b=0.5, c=0.25)
_VOLUME = {
    SPHERE: math.pi / 6.0,
    HEMISPHERE: math.pi / 12.0,
    SPHEROID: 4.0 / 3.0 * math.pi * 0.5 * 0.5 * 0.25,
}
# shape parameter vectors as passed to set_shape
SHAPE_PARAMS = {SPHERE: (1.0,), HEMISPHERE: (1.0,), SPHEROID: (0.5, 0.25)}


def box_length(n: int, phi_c: float, shape: int = SPHERE) -> float:
    """Cubic box side for n colloids at packing fraction phi_c."""
    return (n * _VOLUME[shape] / phi_c) ** (1.0 / 3.0)


def fugacity(eta_r: float, q: float) -> float:
    """Depletant fugacity z_p from the reservoir packing fraction
    eta_r = (pi/6) q^3 z_p (depletant diameter q, colloid diameter 1)."""
    return 6.0 * eta_r / (math.pi * q ** 3)


def fcc_positions(n: int, L: float, seed: int, contact: float = 1.0) -> np.ndarray:
    """n reference points on a random subset of an fcc lattice filling the box,
    jittered, all pairwise (minimum-image) distances >= contact."""
    rng = np.random.default_rng(seed)
    m = int(math.ceil((n / 4.0) ** (1.0 / 3.0)))
    while 4 * m ** 3 < n:
        m += 1
    a = L / m
    nn = a / math.sqrt(2.0)
    if nn < contact:
        raise ValueError("packing fraction too high for an fcc start")
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.arange(m)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    pick = rng.permutation(sites.shape[0])[:n]
    jitter = 0.45 * (nn - contact)
    pos = sites[pick] + rng.uniform(-jitter, jitter, size=(n, 3)) / math.sqrt(3.0)
    pos = np.mod(pos, L)
    pos[pos >= L] = 0.0
    return np.ascontiguousarray(pos, dtype=np.float64)


def random_quaternions(n: int, seed: int) -> np.ndarray:
    """Uniformly random unit quaternions (w, x, y, z) (normalised 4-D Gaussians)."""
    rng = np.random.default_rng(seed + 0x5151)
    qv = rng.normal(size=(n, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    return np.ascontiguousarray(qv, dtype=np.float64)


@dataclass
class System:
    """One replica's inputs."""
    name: str
    shape: int
    n: int
    L: float
    q: float
    n_r: float
    pos: np.ndarray
    quat: np.ndarray | None
    shape_params: tuple = (1.0,)
    d_max: float = 0.1
    a_max: float = 0.0
    p_translate: float = 1.0
    n_trial: int = 0
    seed: int = 1
    replica: int = 0
    extra: dict = field(default_factory=dict)


def make_system(name: str, shape: int, n: int, phi_c: float, q: float,
                eta_r: float, *, seed: int = 1, d_max: float = 0.1,
                a_max: float = 0.0, p_translate: float = 1.0, n_trial: int = 0,
                replica: int = 0) -> System:
    L = box_length(n, phi_c, shape)
    pos = fcc_positions(n, L, seed * 1000003 + replica)
    quat = random_quaternions(n, seed * 7919 + replica) if shape != SPHERE else None
    return System(name=name, shape=shape, n=n, L=L, q=q,
                  n_r=fugacity(eta_r, q) if eta_r > 0 else 0.0, pos=pos, quat=quat,
                  shape_params=SHAPE_PARAMS[shape], d_max=d_max, a_max=a_max,
                  p_translate=p_translate, n_trial=n_trial, seed=seed,
                  replica=replica, extra={"phi_c": phi_c, "eta_r": eta_r})


def spheres_256(seed: int = 1) -> System:
    return make_system("spheres_256", SPHERE, 256, 0.20, 0.20, 0.20, seed=seed,
                       d_max=0.1)


def spheres_16384(eta_r: float = 0.2, seed: int = 1, d_max: float = 0.1) -> System:
    return make_system("spheres_16384_eta%.1f" % eta_r, SPHERE, 16384, 0.30, 0.15,
                       eta_r, seed=seed, d_max=d_max)


def hemispheres_32768(seed: int = 1) -> System:
    return make_system("hemispheres_32768", HEMISPHERE, 32768, 0.25, 0.10, 0.30,
                       seed=seed, d_max=0.1, a_max=0.2, p_translate=0.5)


def discoids_65536(seed: int = 1) -> System:
    return make_system("discoids_65536", SPHEROID, 65536, 0.30, 0.10, 0.25,
                       seed=seed, d_max=0.1, a_max=0.2, p_translate=0.5)


def batched_replicas(count: int = 128, seed: int = 1, n_min: int = 500,
                     n_max: int = 20000) -> list[System]:
    """Independent sphere replicas with N log-uniform in [n_min, n_max],
    phi_c U[0.1,0.45], q in {0.1,0.15,0.2}, eta_r U[0.05,0.4], one seed."""
    rng = np.random.default_rng(seed * 31337)
    out = []
    for r in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        phi = float(rng.uniform(0.10, 0.45))
        q = float(rng.choice([0.10, 0.15, 0.20]))
        eta = float(rng.uniform(0.05, 0.40))
        out.append(make_system("replica%03d" % r, SPHERE, n, phi, q, eta,
                               seed=seed, d_max=0.1, replica=r))
    return out


def tiny_spheres(n: int = 8, L: float = 2.6, seed: int = 3) -> np.ndarray:
    """A handful of non-overlapping spheres in a small box (n_c = 2)."""
    rng = np.random.default_rng(seed)
    pts: list[np.ndarray] = []
    while len(pts) < n:
        p = rng.uniform(0.0, L, size=3)
        ok = True
        for o in pts:
            d = p - o
            d -= L * np.round(d / L)
            if float(d @ d) < 1.0:
                ok = False
                break
        if ok:
            pts.append(p)
    return np.ascontiguousarray(np.array(pts), dtype=np.float64)
