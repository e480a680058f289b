"""Pins of the oracle's observables (orc_observables) against values the
geometry and the lattice fix, not against the oracle's own formulas.

* droplet area and radius (Sec. 2.2; reading R11: A = sum S / S_n, R from
  the area of a disc or the volume of a sphere): a sharp uniaxial droplet
  with S = S_n in an exactly counted set of cells, each with its own random
  director, gives A = that count, and for a large droplet R is the radius it
  was drawn with, to the accuracy of the lattice count of a disc or ball;
* the interface position (Sec. 2.1; reading R10) and the y, z mean of S on
  a prescribed piecewise-linear profile;
* mass, the momentum sums and max |u| (Sec. 2.2, the spurious velocity) on
  equilibrium populations with a prescribed rho and u and Q = 0 (then F = 0
  and Eq. 6 returns u itself), and with Q != 0, where the total momentum is
  the lattice sum of sum_i c_i f_i because the force, a periodic divergence,
  sums to zero;
* the count of non-finite values planted in f and Q.

Runs on the CPU."""
import math

import numpy as np
import pytest

from paper_1907_13415_gb300 import workloads as wl

S_N = 1.0 / 3.0


def random_directors(rng, shape):
    n = rng.normal(size=shape + (3,))
    return n / np.linalg.norm(n, axis=-1, keepdims=True)


def uniaxial_cells(S, n):
    """Q5 of Q = S (n n - I/3) per cell, with a per-cell director n."""
    out = np.empty((5,) + S.shape)
    for k, (a, b) in enumerate(wl.Q_INDEX):
        out[k] = S * (n[..., a] * n[..., b] - (1.0 / 3.0 if a == b else 0.0))
    return out


def disc_mask(shape, centre, R):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2
    if nz > 1:
        r2 = r2 + (z - centre[2]) ** 2
    return r2 < R * R


def params():
    return wl.param_vector(wl.BASE_PARAMS)


@pytest.mark.parametrize("lattice,shape,R", [
    (wl.D2Q9, (1, 96, 96), 40.0),
    (wl.D3Q19, (1, 96, 96), 40.0),     # a single plane of D3Q19: the 2D form
    (wl.D3Q19, (48, 48, 48), 20.0),
])
def test_droplet_area_and_radius(orc, lattice, shape, R):
    rng = np.random.default_rng(31)
    centre = (shape[2] / 2 - 0.3, shape[1] / 2 + 0.2, shape[0] / 2 - 0.1)
    inside = disc_mask(shape, centre, R)
    count = int(inside.sum())
    Q5 = uniaxial_cells(np.where(inside, S_N, 0.0), random_directors(rng, shape))
    f = orc.init_equilibrium(lattice, shape)
    o = orc.observables(lattice, params(), f, Q5)
    # every nematic cell contributes S / S_n = 1 whatever its director
    assert o["s_area"] == pytest.approx(count, rel=1e-13)
    # the radius of the droplet it was drawn with: the lattice count of a
    # disc (ball) of radius R differs from pi R^2 (4 pi R^3 / 3) by a
    # boundary term of relative size O(1/R)
    assert o["radius"] == pytest.approx(R, rel=5e-3)
    if shape[0] == 1:
        assert o["radius"] == pytest.approx(math.sqrt(count / math.pi), rel=1e-13)
    else:
        assert o["radius"] == pytest.approx((count * 0.75 / math.pi) ** (1.0 / 3.0), rel=1e-13)


def test_radius_scales_with_the_droplet(orc):
    """Doubling R doubles the radius (2D) within the lattice count's error,
    and a sphere's radius is not a disc's: on 3D lattices the same cell
    count read with the 2D formula would be far off."""
    lattice = wl.D3Q19
    shape = (40, 40, 40)
    out = []
    for R in (8.0, 16.0):
        inside = disc_mask(shape, (19.5, 19.5, 19.5), R)
        Q5 = wl.uniaxial_q5(np.where(inside, S_N, 0.0), (0, 0, 1))
        f = orc.init_equilibrium(lattice, shape)
        out.append(orc.observables(lattice, params(), f, Q5)["radius"])
    assert out[0] == pytest.approx(8.0, rel=2e-2)
    assert out[1] == pytest.approx(16.0, rel=1e-2)


@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 6, 40)),
                                           (wl.D3Q19, (4, 5, 40))])
def test_interface_position_and_profile(orc, lattice, shape):
    """S falls linearly from S_n at x = 10 to 0 at x = 20 along every (y, z)
    column, with a y, z dependent offset of zero mean: the mean profile is
    the line, and it crosses S_n / 2 at x = 15.  A rising edge at x = 30 must
    not count (the first descending crossing)."""
    nz, ny, nx = shape
    x = np.arange(nx, dtype=float)
    line = np.clip((20.0 - x) / 10.0, 0.0, 1.0) * S_N
    line = np.where(x >= 30, S_N, line)
    rng = np.random.default_rng(5)
    off = rng.uniform(-0.02, 0.02, size=(nz, ny, 1))
    off -= off.mean()
    S = np.broadcast_to(line, shape) + np.where(line > 0.05, off, 0.0)
    # each cell's own director: S is invariant under rotations of n
    Q5 = uniaxial_cells(S, random_directors(rng, shape))
    f = orc.init_equilibrium(lattice, shape)
    o = orc.observables(lattice, params(), f, Q5)
    assert np.allclose(o["s_profile"], line, rtol=0, atol=1e-14)
    assert o["x_iface"] == pytest.approx(15.0, abs=1e-12)


@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 7, 9)),
                                           (wl.D3Q19, (3, 4, 5))])
def test_mass_momentum_and_max_speed_at_rest_force(orc, lattice, shape):
    """Q = 0 gives F = 0, and equilibrium populations of a prescribed rho, u
    return that u (Eq. 6): mass = sum rho, momentum = sum rho u, and max |u|
    is the largest speed, placed at a cell whose components are each
    smaller than another cell's largest component."""
    d = 2 if lattice == wl.D2Q9 else 3
    rng = np.random.default_rng(8)
    nz, ny, nx = shape
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, size=shape)
    u = np.zeros((3,) + shape)
    u[:d] = rng.uniform(-0.02, 0.02, size=(d,) + shape)
    u[:, 0, 0, 0] = 0.0
    u[0, 0, 0, 0], u[1, 0, 0, 0] = 0.03, 0.04           # |u| = 0.05
    u[:, 0, 1, 1] = 0.0
    u[0, 0, 1, 1] = 0.045                               # largest component
    f = orc.init_equilibrium(lattice, shape, rho=rho, u=u)
    o = orc.observables(lattice, params(), f, np.zeros((5,) + shape))
    assert o["mass"] == pytest.approx(rho.sum(), rel=1e-14)
    for a, name in enumerate(("mom_x", "mom_y", "mom_z")):
        assert o[name] == pytest.approx((rho * u[a]).sum(), abs=1e-14)
    assert o["max_u"] == pytest.approx(0.05, rel=1e-12)
    assert o["nonfinite"] == 0


@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 10, 12)),
                                           (wl.D3Q19, (6, 6, 8))])
def test_momentum_sum_with_force(orc, lattice, shape):
    """With Q != 0 the momentum is sum_i c_i f_i + F/2 per cell, and F, the
    divergence of a periodic stress, sums to zero over the lattice: the
    totals equal sum over cells and velocities of c_i f_i, formed here from
    the oracle's own lattice vectors."""
    rng = np.random.default_rng(9)
    w = wl.Workload("t", lattice, shape, dict(wl.BASE_PARAMS), 0, "ball", 3.0,
                    (1, 1, 0), 0.02, 3)
    Q5 = w.initial_q5()
    u = np.zeros((3,) + shape)
    d = 2 if lattice == wl.D2Q9 else 3
    u[:d] = rng.uniform(-0.01, 0.01, size=(d,) + shape)
    f = orc.init_equilibrium(lattice, shape, u=u)
    p = params()
    fl = orc.fields(lattice, p, f, Q5)
    assert np.abs(fl["F"]).max() > 1e-6          # the force is not trivially zero
    c, _ = orc.lattice(lattice)
    J = np.einsum("ia,izyx->a", c.astype(float), f)
    o = orc.observables(lattice, p, f, Q5)
    for a, name in enumerate(("mom_x", "mom_y", "mom_z")):
        assert o[name] == pytest.approx(J[a], abs=1e-13)
    # and max |u| is the largest speed of the physical velocity of Eq. 6
    sp = np.sqrt((fl["u"] ** 2).sum(axis=0)).max()
    assert o["max_u"] == pytest.approx(sp, rel=1e-14)


def test_nonfinite_count(orc):
    lattice, shape = wl.D2Q9, (1, 6, 7)
    f = orc.init_equilibrium(lattice, shape)
    Q5 = wl.uniaxial_q5(np.full(shape, S_N), (0, 1, 0))
    f[3, 0, 2, 2] = np.nan
    f[5, 0, 4, 1] = np.inf
    f[5, 0, 4, 2] = -np.inf
    Q5[1, 0, 0, 6] = np.nan
    Q5[4, 0, 5, 0] = np.inf
    o = orc.observables(lattice, params(), f, Q5)
    assert o["nonfinite"] == 5
