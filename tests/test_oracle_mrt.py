"""Pins of the oracle's multiple-relaxation-time collision (Sec. 1.2.1 names
MRT as the operator the paper uses but gives neither its matrices nor its
rates; the rates are the caller's).

The pins: with every rate equal to 1/tau it is the BGK step with its source
term (pinned separately); the shear viscosity follows only the rate of the
second-order traceless moments, nu = (1/s_nu - 1/2)/3, whatever the other
rates; mass and momentum are conserved for any rates; and a disturbance
along one non-conserved moment relaxes by the factor 1 - s_k of that moment
alone.  CPU only.
"""
import numpy as np
import pytest

from paper_1907_13415_gb300 import workloads as wl

# moments of the oracle's basis that carry the viscous stress
SHEAR = {wl.D2Q9: (7, 8), wl.D3Q19: (9, 11, 13, 14, 15)}
CONSERVED = {wl.D2Q9: (0, 3, 5), wl.D3Q19: (0, 3, 5, 7)}


def params(**kw):
    p = dict(wl.BASE_PARAMS)
    p.update(kw)
    return wl.param_vector(p)


@pytest.fixture
def mrt(orc):
    yield orc
    orc.set_mrt(wl.D2Q9, None)


def random_rates(q, lattice, s_nu, seed):
    rng = np.random.default_rng(seed)
    s = rng.uniform(1.05, 1.85, size=q)
    for k in SHEAR[lattice]:
        s[k] = s_nu
    return s


@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 12, 13)),
                                           (wl.D3Q19, (5, 6, 7))])
def test_equal_rates_give_bgk(mrt, lattice, shape):
    w = wl.sphere_256().with_(lattice=lattice, shape=shape, geometry="ball",
                              size=0.35 * min(shape[1:]), noise=1e-2, seed=5)
    tau = 0.9
    p = params(tau=tau)
    q = 9 if lattice == wl.D2Q9 else 19
    f0 = mrt.init_equilibrium(lattice, shape)
    fb, Qb = mrt.step(lattice, p, f0, w.initial_q5(), 30)
    mrt.set_mrt(lattice, np.full(q, 1.0 / tau))
    fm, Qm = mrt.step(lattice, p, f0, w.initial_q5(), 30)
    assert np.abs(fm - fb).max() < 1e-13
    assert np.abs(Qm - Qb).max() < 1e-13 * np.abs(Qb).max()


@pytest.mark.parametrize("lattice", [wl.D2Q9, wl.D3Q19])
def test_shear_viscosity_follows_its_own_rate(mrt, lattice):
    """A shear wave u_x = U sin(k y) with Q = 0, xi = 0 decays as
    exp(-nu k^2 t), nu = (1/s_nu - 1/2)/3; the other rates (random) and tau
    (unused by MRT) do not enter."""
    L, U, T = 64, 1e-4, 600
    nz = 1 if lattice == wl.D2Q9 else 2
    shape = (nz, L, 4)
    q = 9 if lattice == wl.D2Q9 else 19
    tau_nu = 0.8
    mrt.set_mrt(lattice, random_rates(q, lattice, 1.0 / tau_nu, seed=3))
    y = np.arange(L)[None, :, None] * np.ones(shape)
    k = 2 * np.pi / L
    u = np.zeros((3,) + shape)
    u[0] = U * np.sin(k * y)
    f = mrt.init_equilibrium(lattice, shape, u=u)
    Q5 = np.zeros((5,) + shape)
    p = params(tau=1.7, xi=0.0)
    f, Q5 = mrt.step(lattice, p, f, Q5, T)
    ux = mrt.fields(lattice, p, f, Q5)["u"][0]
    amp = 2 * np.mean(ux * np.sin(k * y))
    nu = (tau_nu - 0.5) / 3
    assert amp / U == pytest.approx(np.exp(-nu * k * k * T), rel=3e-3)


def test_conservation_with_arbitrary_rates(mrt):
    rng = np.random.default_rng(9)
    for lattice, shape in ((wl.D2Q9, (1, 9, 10)), (wl.D3Q19, (5, 4, 6))):
        q = 9 if lattice == wl.D2Q9 else 19
        mrt.set_mrt(lattice, rng.uniform(0.6, 1.9, size=q))
        Q5 = rng.normal(scale=0.1, size=(5,) + shape)
        u = rng.normal(scale=0.01, size=(3,) + shape)
        rho = 1 + 0.01 * rng.normal(size=shape)
        f = mrt.init_equilibrium(lattice, shape, rho=rho, u=u)
        p = params()
        o0 = mrt.observables(lattice, p, f, Q5)
        f2, Q2 = mrt.step(lattice, p, f, Q5, 40)
        o1 = mrt.observables(lattice, p, f2, Q2)
        assert o1["mass"] == pytest.approx(o0["mass"], rel=1e-14)
        for key in ("mom_x", "mom_y", "mom_z"):
            assert abs(o1[key] - o0[key]) < 1e-13 * np.prod(shape)


@pytest.mark.parametrize("lattice", [wl.D2Q9, wl.D3Q19])
def test_each_moment_relaxes_with_its_rate(mrt, lattice):
    """At rest (u = 0, F = 0) a disturbance eps v_k of the equilibrium along
    one non-conserved moment row comes out as (1 - s_k) eps v_k: the moment
    rows are orthogonal and each carries exactly its own rate."""
    q = 9 if lattice == wl.D2Q9 else 19
    rates = np.linspace(0.55, 1.95, q)
    mrt.set_mrt(lattice, rates)
    V = mrt.mrt_basis(lattice)
    c, _ = mrt.lattice(lattice)
    # the rows span, in order, the listed polynomials: row 1 is c^2 minus
    # its mean, row 3 is c_x itself
    c2 = (c ** 2).sum(1)
    assert np.allclose(V[0], 1.0)
    assert np.allclose(V[1], c2 - c2.mean())
    assert np.allclose(V[3], c[:, 0])
    feq = mrt.equilibrium_point(lattice, 1.0, np.zeros(3))
    for k in range(q):
        if k in CONSERVED[lattice]:
            continue
        post = mrt.mrt_point(lattice, feq + 1e-3 * V[k], 1.0, np.zeros(3),
                             np.zeros(3))
        assert np.allclose(post - feq, (1 - rates[k]) * 1e-3 * V[k], atol=1e-16)
