"""Seeded synthetic inputs for the nematic-isotropic interface runs.

This module is shared by the tests, the benchmark, the smoke check and the
oracle checks, and holds none of the method's arithmetic: it only builds
initial order-parameter fields Q = S (n n - I/3) (the uniaxial form of
Sec. 1.1) for the geometries of Sec. 2 (a nematic slab, disc or sphere in an
isotropic background, density 1 and velocity 0), plus seeded uniform noise.

All fields are float64 numpy arrays in the layout (5, nz, ny, nx) with the
components ordered (xx, xy, xz, yy, yz) and x fastest.
"""
from dataclasses import dataclass, field

import numpy as np

D2Q9 = 0
D3Q19 = 1

#: the parameter set used by the workloads (lattice units).  The paper's own
#: set (Sec. 2) is PAPER_PARAMS.
BASE_PARAMS = dict(A0=0.1, K=0.02, gamma=2.70, Gamma=0.3, xi=0.7, tau=1.0)
PAPER_PARAMS = dict(A0=0.1, K=0.04, gamma=2.70, Gamma=0.34, xi=0.7, tau=1.5)
PARAM_ORDER = ("A0", "K", "gamma", "Gamma", "xi", "tau")

S_COEX = 1.0 / 3.0  # nematic order at coexistence, gamma = 2.7 (Sec. 2.1)

Q_INDEX = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2))


def param_vector(params):
    return np.array([params[k] for k in PARAM_ORDER], dtype=np.float64)


def uniaxial_q5(S, director):
    """Q5 of Q = S (n n - I/3) for a scalar field S (nz, ny, nx), unit n."""
    n = np.asarray(director, dtype=np.float64)
    n = n / np.linalg.norm(n)
    S = np.asarray(S, dtype=np.float64)
    out = np.empty((5,) + S.shape)
    for k, (a, b) in enumerate(Q_INDEX):
        out[k] = S * (n[a] * n[b] - (1.0 / 3.0 if a == b else 0.0))
    return out


def add_noise(Q5, amplitude, seed):
    """i.i.d. uniform noise in [-amplitude, amplitude] on all five components,
    drawn from numpy's PCG64 generator with the given seed."""
    if amplitude == 0.0:
        return Q5
    rng = np.random.Generator(np.random.PCG64(seed))
    return Q5 + rng.uniform(-amplitude, amplitude, size=Q5.shape)


def slab_S(shape, x_split, S_in=S_COEX):
    """S = S_in for x < x_split, else 0 (sharp step; periodic in x)."""
    nz, ny, nx = shape
    S = np.where(np.arange(nx) < x_split, S_in, 0.0)
    return np.broadcast_to(S, shape).copy()


def ball_S(shape, radius, S_in=S_COEX):
    """S = S_in inside a disc (nz = 1) or sphere of the given radius centred
    at ((nx-1)/2, (ny-1)/2, (nz-1)/2), else 0."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                          indexing="ij")
    r2 = (x - (nx - 1) / 2.0) ** 2 + (y - (ny - 1) / 2.0) ** 2
    if nz > 1:
        r2 = r2 + (z - (nz - 1) / 2.0) ** 2
    return np.where(r2 < radius * radius, S_in, 0.0)


@dataclass
class Workload:
    """One lattice problem: geometry, parameters and initial Q."""
    name: str
    lattice: int
    shape: tuple  # (nz, ny, nx)
    params: dict
    steps: int
    geometry: str  # 'slab' | 'ball'
    size: float  # slab split position or ball radius
    director: tuple
    noise: float
    seed: int
    extra: dict = field(default_factory=dict)

    @property
    def n_cells(self):
        nz, ny, nx = self.shape
        return nx * ny * nz

    def initial_q5(self):
        if self.geometry == "slab":
            S = slab_S(self.shape, self.size)
        else:
            S = ball_S(self.shape, self.size)
        return add_noise(uniaxial_q5(S, self.director), self.noise, self.seed)

    def with_(self, **kw):
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


def flat_128x8():
    """Flat interface: 128x8 D2Q9, S = 1/3 for x < 64, n along y, noise 1e-6
    (seed 0), gamma = 2.70, 2000 steps, FP64."""
    return Workload("flat_128x8_d2q9", D2Q9, (1, 8, 128), dict(BASE_PARAMS),
                    2000, "slab", 64, (0, 1, 0), 1e-6, 0)


def disc_256(delta=0.0):
    """Circular droplet: 256x256 D2Q9, R = 32, n along x, gamma = 2.70 +
    delta, 20000 steps."""
    p = dict(BASE_PARAMS)
    p["gamma"] = 2.70 + delta
    return Workload(f"disc_r32_256x256_d2q9_delta{delta:g}", D2Q9,
                    (1, 256, 256), p, 20000, "ball", 32, (1, 0, 0), 0.0, 1,
                    extra=dict(delta=delta))


def sweep_64(n=64, seed=2):
    """Temperature sweep: n flat-interface instances, gamma evenly spaced over
    [2.60, 2.80], Lx from {256, 512, 1024, 2048} and Ly from {8, 16, 64}
    drawn by PCG64(seed); step at Lx/2, 50000 steps, FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lxs = rng.choice([256, 512, 1024, 2048], size=n)
    lys = rng.choice([8, 16, 64], size=n)
    gammas = np.linspace(2.60, 2.80, n)
    out = []
    for i in range(n):
        p = dict(BASE_PARAMS)
        p["gamma"] = float(gammas[i])
        lx, ly = int(lxs[i]), int(lys[i])
        out.append(Workload(f"sweep{i}_{lx}x{ly}", D2Q9, (1, ly, lx), p,
                            50000, "slab", lx // 2, (0, 1, 0), 1e-6,
                            seed + i))
    return out


def sphere_256():
    """Spherical droplet: 256^3 D3Q19, R = 48, n along z, noise 1e-4 (seed 3),
    gamma = 2.705, 5000 steps, FP32 (the bandwidth workload)."""
    p = dict(BASE_PARAMS)
    p["gamma"] = 2.705
    return Workload("sphere_r48_256cubed_d3q19", D3Q19, (256, 256, 256), p,
                    5000, "ball", 48, (0, 0, 1), 1e-4, 3)


def adjoint_disc_128():
    """Adjoint case: 128x128 D2Q9 disc of radius 24, gamma = 2.70, 2000 steps,
    checkpoints every 100 steps.  Noise 1e-6 (seed 4) keeps S > 0 in every
    cell, where the loss's dependence on S is differentiable."""
    return Workload("adjoint_disc_r24_128x128_d2q9", D2Q9, (1, 128, 128),
                    dict(BASE_PARAMS), 2000, "ball", 24, (1, 0, 0), 1e-6, 4,
                    extra=dict(ckpt_every=100, target_radius=24.0))


def scaled(w, shape, size=None, steps=None, name=None):
    """The same recipe on another lattice size (for parity-sized cases)."""
    return w.with_(shape=tuple(shape), size=w.size if size is None else size,
                   steps=w.steps if steps is None else steps,
                   name=name or f"{w.name}@{'x'.join(map(str, shape[::-1]))}")
