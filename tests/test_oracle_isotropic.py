"""Pins of the oracle's isotropic finite-difference stencils (the remedy the
paper points to for the spurious currents, Sec. 2.2: more isotropy).

The isotropic stencils use the lattice's own neighbour set.  Their defining
property, checked here against the standard stencils on the same fields: on
a plane wave cos(k.x) the Laplacian's eigenvalue is -|k|^2 + c4 |k|^4 + ...
with c4 the same in every direction (the standard 2d+1-point stencil's c4
varies by a factor of two), and likewise the first-derivative error.  On a
single plane the 19-point stencils reduce to the 9-point ones, so D3Q19 with
nz = 1 still equals D2Q9; the scheme keeps mass and momentum.  CPU only.
"""
import numpy as np
import pytest

from paper_1907_13415_gb300 import workloads as wl


def params(**kw):
    p = dict(wl.BASE_PARAMS)
    p.update(kw)
    return wl.param_vector(p)


@pytest.fixture
def iso(orc):
    yield orc
    orc.set_stencil(0)


def plane_wave(shape, kvec):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    L = np.array([nx, ny, nz], dtype=float)
    k = 2 * np.pi * np.asarray(kvec, dtype=float) / L
    return np.cos(k[0] * x + k[1] * y + k[2] * z), np.sin(k[0] * x + k[1] * y + k[2] * z), k


def laplacian_eigen(orc, lattice, shape, kvec):
    """lambda with lap cos(k.x) = lambda cos(k.x): H = K lap Q when A0 = 0."""
    c, s, k = plane_wave(shape, kvec)
    Q5 = np.zeros((5,) + shape)
    Q5[1] = 1e-3 * c
    p = params(A0=0.0, K=1.0)
    f = orc.init_equilibrium(lattice, shape)
    H = orc.fields(lattice, p, f, Q5)["H"][1]
    lam = np.sum(H * Q5[1]) / np.sum(Q5[1] ** 2)
    return lam, float(np.sum(k * k))


def gradient_eigen(orc, lattice, shape, kvec, axis):
    """mu with d_axis cos(k.x) = -mu sin(k.x): with Gamma = 0 and u = e_axis
    (uniform, no gradient, no co-rotation) R = -d_axis Q."""
    c, s, k = plane_wave(shape, kvec)
    Q5 = np.zeros((5,) + shape)
    Q5[1] = 1e-3 * c
    u = np.zeros((3,) + shape)
    u[axis] = 1.0
    R = orc.rhs(lattice, params(Gamma=0.0, xi=0.0), Q5, u)[1]
    return np.sum(R * 1e-3 * s) / np.sum((1e-3 * s) ** 2), k


@pytest.mark.parametrize("lattice,shape,kvecs", [
    (wl.D2Q9, (1, 64, 64), [(8, 0, 0), (6, 5, 0), (5, 6, 0)]),
    (wl.D3Q19, (32, 32, 32), [(4, 0, 0), (3, 2, 2), (2, 3, 3)]),
])
def test_laplacian_error_is_direction_free(iso, lattice, shape, kvecs):
    c4 = {}
    for kind in (0, 1):
        iso.set_stencil(kind)
        vals = []
        for kv in kvecs:
            lam, k2 = laplacian_eigen(iso, lattice, shape, kv)
            vals.append((lam + k2) / k2 ** 2)
        c4[kind] = np.array(vals)
    spread = lambda v: (v.max() - v.min()) / np.abs(v).mean()
    assert spread(c4[0]) > 0.4          # the 2d+1-point stencil is anisotropic
    assert spread(c4[1]) < 0.06         # the lattice stencil is not
    assert np.all(c4[1] > 0)            # and keeps the k^4 term of lap + k^2/12-like sign


@pytest.mark.parametrize("lattice,shape,kvecs", [
    (wl.D2Q9, (1, 64, 64), [(8, 0, 0), (6, 5, 0), (5, 6, 0)]),
    (wl.D3Q19, (32, 32, 32), [(4, 0, 0), (3, 2, 2), (2, 3, 3)]),
])
def test_gradient_error_is_direction_free(iso, lattice, shape, kvecs):
    e3 = {}
    for kind in (0, 1):
        iso.set_stencil(kind)
        vals = []
        for kv in kvecs:
            mu, k = gradient_eigen(iso, lattice, shape, kv, axis=0)
            if k[0] == 0:
                continue
            # mu = k_x (1 - e3 |k|^2 + ...): the relative error over |k|^2
            vals.append((1 - mu / k[0]) / np.sum(k * k))
        e3[kind] = np.array(vals)
    spread = lambda v: (v.max() - v.min()) / np.abs(v).mean()
    assert spread(e3[0]) > 0.3
    assert spread(e3[1]) < 0.06


def test_isotropic_d3q19_single_plane_equals_d2q9(iso):
    """With Qxz = Qyz = 0 (no out-of-plane force) the 19-point stencils one
    cell thick reduce to the 9-point ones."""
    iso.set_stencil(1)
    shape = (1, 11, 13)
    w = wl.flat_128x8().with_(shape=shape, geometry="ball", size=4, noise=0.0,
                              director=(0.6, 0.8, 0))
    Q0 = w.initial_q5() + np.random.default_rng(9).uniform(-1e-2, 1e-2, (5,) + shape) * \
        np.array([1, 1, 0, 1, 0])[:, None, None, None]
    p = wl.param_vector(w.params)
    out = []
    for lattice in (wl.D2Q9, wl.D3Q19):
        f = iso.init_equilibrium(lattice, shape)
        f, Q = iso.step(lattice, p, f, Q0, 40)
        out.append((Q, iso.fields(lattice, p, f, Q)["u"]))
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-13
    assert np.abs(out[0][1] - out[1][1]).max() < 1e-15


def test_isotropic_scheme_conserves_mass_and_momentum(iso):
    iso.set_stencil(1)
    rng = np.random.default_rng(13)
    for lattice, shape in ((wl.D2Q9, (1, 9, 10)), (wl.D3Q19, (5, 4, 6))):
        Q5 = rng.normal(scale=0.1, size=(5,) + shape)
        u = rng.normal(scale=0.01, size=(3,) + shape)
        f = iso.init_equilibrium(lattice, shape, u=u)
        p = params()
        o0 = iso.observables(lattice, p, f, Q5)
        f2, Q2 = iso.step(lattice, p, f, Q5, 40)
        o1 = iso.observables(lattice, p, f2, Q2)
        assert o1["mass"] == pytest.approx(o0["mass"], rel=1e-14)
        for key in ("mom_x", "mom_y", "mom_z"):
            assert abs(o1[key] - o0[key]) < 1e-13 * np.prod(shape)
