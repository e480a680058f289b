"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle through a route other than its own formulas:
closed forms derived from the free energy (Eq. 2), identities that hold for
any field, textbook lattice-Boltzmann results, convergence orders, and the
values the paper prints (tests/golden/paper_values.json).  None of these needs
a GPU.
"""
import json
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.linalg import expm
from scipy.optimize import least_squares

from paper_1907_13415_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden",
                      "paper_values.json")
IDX5 = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2))


def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def rand_sym_traceless(rng, scale=0.3):
    A = rng.normal(size=(3, 3)) * scale
    A = (A + A.T) / 2
    return A - np.trace(A) / 3 * np.eye(3)


def full_from5(Q5):
    """(5, ...) -> (3, 3, ...) with Qzz = -Qxx - Qyy."""
    xx, xy, xz, yy, yz = Q5
    zz = -xx - yy
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def params(**kw):
    p = dict(wl.BASE_PARAMS)
    p.update(kw)
    return wl.param_vector(p)


# ---------------------------------------------------------------------------
# Free energy (Eq. 2) and molecular field (Eq. 3)
# ---------------------------------------------------------------------------

def free_energy_np(Q5, p):
    """Discrete Eq. 2 written independently in numpy: bulk terms plus the
    gradient term with forward differences, K/2 sum_g (Q(x+e_g) - Q(x))^2.
    Works for complex Q5 (complex-step differentiation)."""
    A0, K, gam = p[0], p[1], p[2]
    Q = full_from5(Q5)
    tr2 = np.einsum("ab...,ab...->...", Q, Q)
    tr3 = np.einsum("ab...,bc...,ca...->...", Q, Q, Q)
    bulk = (A0 / 2 * (1 - gam / 3) * tr2 - A0 * gam / 3 * tr3
            + A0 * gam / 4 * tr2 ** 2)
    grad = 0
    for axis in (-1, -2, -3):  # x, y, z
        d = np.roll(Q, -1, axis=axis) - Q
        grad = grad + np.einsum("ab...,ab...->...", d, d)
    return np.sum(bulk) + K / 2 * np.sum(grad)


@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 12, 14)),
                                           (wl.D3Q19, (6, 7, 8))])
def test_free_energy_decreases_without_flow(orc, lattice, shape):
    """With u = 0, Eq. 1 is the gradient flow dQ/dt = Gamma H = -Gamma dF/dQ
    of the discrete free energy, so F (Eq. 2, written independently above)
    never increases under the predictor-corrector steps of the oracle's
    right-hand side (small steps: Gamma K 4d << 1).  Also pins the oracle's
    free-energy observable to that independent F."""
    w = wl.sphere_256().with_(lattice=lattice, shape=shape, geometry="ball",
                              size=0.35 * min(shape[1:]), noise=2e-2, seed=11)
    p = params(gamma=2.7)
    Q = w.initial_q5()
    u0 = np.zeros((3,) + shape)
    f = orc.init_equilibrium(lattice, shape)
    F = [free_energy_np(Q, p)]
    assert orc.observables(lattice, p, f, Q)["free_energy"] == pytest.approx(
        F[0], rel=1e-12)
    for _ in range(60):
        R1 = orc.rhs(lattice, p, Q, u0)
        R2 = orc.rhs(lattice, p, Q + R1, u0)
        Q = Q + 0.5 * (R1 + R2)
        F.append(free_energy_np(Q, p))
    F = np.array(F)
    assert np.all(np.diff(F) <= 1e-14 * np.abs(F[:-1]))
    assert F[-1] < F[0]


@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 5, 6)),
                                           (wl.D3Q19, (3, 4, 5))])
def test_H_is_minus_gradient_of_free_energy(orc, lattice, shape):
    """Eq. 3 is -dF/dQ (made traceless) of Eq. 2.  With the 2d+1-point
    Laplacian the discrete identity is exact: the derivative of the discrete
    energy with respect to the five stored components equals
    -(Hxx - Hzz), -2Hxy, -2Hxz, -(Hyy - Hzz), -2Hyz."""
    rng = np.random.default_rng(11)
    p = params(K=0.07, gamma=2.9)
    Q5 = rng.normal(scale=0.2, size=(5,) + shape)
    f = orc.init_equilibrium(lattice, shape)
    H5 = orc.fields(lattice, p, f, Q5)["H"]
    H = full_from5(H5)
    expect = -np.array([H[0, 0] - H[2, 2], 2 * H[0, 1], 2 * H[0, 2],
                        H[1, 1] - H[2, 2], 2 * H[1, 2]])
    h = 1e-30
    got = np.zeros_like(Q5)
    for k in range(5):
        for cell in [(0, 0, 0), (shape[0] - 1, 1, 2), (0, shape[1] - 1, 3)]:
            Qc = Q5.astype(np.complex128)
            Qc[(k,) + cell] += 1j * h
            got[(k,) + cell] = free_energy_np(Qc, p).imag / h
            assert got[(k,) + cell] == pytest.approx(
                expect[(k,) + cell], rel=1e-11, abs=1e-14)


def test_H_symmetric_traceless(orc):
    rng = np.random.default_rng(1)
    for _ in range(20):
        Q = rand_sym_traceless(rng)
        L = rand_sym_traceless(rng)
        H = orc.molecular_field_point(Q, L, params(gamma=3.3 * rng.random()))
        assert np.allclose(H, H.T, atol=1e-16)
        assert abs(np.trace(H)) < 1e-16


def s_nematic(gamma):
    """Bulk nematic order of the free energy of Eq. 2 (uniaxial reduction
    f(S) = A0/3 (1-g/3) S^2 - 2 A0 g/27 S^3 + A0 g/9 S^4, nonzero root of
    f'(S) = 0 with f'' > 0)."""
    return 0.25 + 0.75 * np.sqrt(1 - 8 / (3 * gamma))


@pytest.mark.parametrize("gamma", [2.7, 2.72, 2.9, 3.2])
def test_uniform_nematic_minimum_has_zero_field(orc, gamma):
    rng = np.random.default_rng(int(gamma * 100))
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    S = s_nematic(gamma)
    Q = S * (np.outer(n, n) - np.eye(3) / 3)
    H = orc.molecular_field_point(Q, np.zeros((3, 3)), params(gamma=gamma))
    assert np.abs(H).max() < 1e-16


def test_coexistence_at_gamma_2p7(orc):
    """The paper's gamma_NI = 2.7 with S_n = 1/3 (Sec. 2.1): uniform nematic
    and isotropic states have equal free energy there; the nematic wins
    above it and loses below it."""
    g = golden()
    assert g["gamma_NI"]["value"] == 2.7 and g["S_n"]["value"] == pytest.approx(1 / 3)
    shape = (1, 2, 3)
    f = orc.init_equilibrium(wl.D2Q9, shape)

    def energy(S, gamma):
        Q5 = wl.uniaxial_q5(np.full(shape, S), (0, 1, 0))
        return orc.observables(wl.D2Q9, params(gamma=gamma), f, Q5)["free_energy"]

    assert abs(energy(1 / 3, 2.7)) < 1e-18
    assert energy(0.0, 2.7) == 0.0
    assert energy(1 / 6, 2.7) > 0  # barrier between the two minima
    assert energy(s_nematic(2.71), 2.71) < 0
    assert energy(1 / 3, 2.69) > 0
    assert s_nematic(g["gamma_NI"]["value"]) == pytest.approx(1 / 3, abs=1e-15)


def test_correlation_length_value(orc):
    """lambda = sqrt(27 K / (A0 gamma)) = 2 for the paper's K = 0.04,
    A0 = 0.1, gamma = 2.7 (Eq. 7 and the text after it)."""
    g = golden()
    p = wl.PAPER_PARAMS
    lam = np.sqrt(27 * p["K"] / (p["A0"] * 2.7))
    assert lam == pytest.approx(g["lambda"]["value"], abs=1e-12)


def test_stability_limits_bracket_spinodals(orc):
    """Sec. 2.1: below gamma = 2.65 everything becomes isotropic and above
    3.1 everything becomes nematic.  The uniform nematic exists only above
    the spinodal 8/3 and the isotropic state is locally stable only below 3,
    so 2.65 < 8/3 and 3.1 > 3.  In the oracle a uniform nematic at 2.65
    melts and a uniform small-S seed at 3.1 orders."""
    g = golden()
    lo, hi = g["gamma_low"]["value"], g["gamma_high"]["value"]
    assert lo < 8 / 3 < 3 < hi
    shape = (1, 2, 2)
    f = orc.init_equilibrium(wl.D2Q9, shape)
    Q5 = wl.uniaxial_q5(np.full(shape, 1 / 3), (0, 1, 0))
    _, Qa = orc.step(wl.D2Q9, params(gamma=lo), f, Q5, 20000)
    assert np.abs(Qa).max() < 1e-3
    Q5 = wl.uniaxial_q5(np.full(shape, 0.01), (0, 1, 0))
    _, Qb = orc.step(wl.D2Q9, params(gamma=hi), f, Q5, 20000)
    S = np.sqrt(1.5 * np.einsum("ab...,ab...->...", full_from5(Qb),
                                full_from5(Qb)))
    assert S.min() == pytest.approx(s_nematic(hi), rel=1e-6)


# ---------------------------------------------------------------------------
# Co-rotational term (Eq. 1's S) and stress (Eq. 5)
# ---------------------------------------------------------------------------

def test_corotation_symmetric_with_trace_identity(orc):
    """S(W, D, Q) is symmetric and Tr S = 2 xi (div u)/3 for traceless Q."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        G = rng.normal(size=(3, 3))
        Q = rand_sym_traceless(rng)
        xi = rng.random()
        S = orc.corotation_point(G, Q, xi)
        assert np.allclose(S, S.T, atol=1e-15)
        assert np.trace(S) == pytest.approx(2 * xi * np.trace(G) / 3,
                                            abs=1e-15)


def test_corotation_rigid_rotation(orc):
    """In a rigid rotation u = w x r (D = 0) the co-rotational term is the
    rate of change of the rotated tensor, d/dt [R(t) (Q+I/3) R(t)^T] at
    t = 0, whatever xi is."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        w = rng.normal(size=3)
        Om = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
        # u = w x r  =>  d_b u_a = Om[a, b]
        Q = rand_sym_traceless(rng)
        Qt = Q + np.eye(3) / 3
        h = 1e-5
        Rp, Rm = expm(Om * h), expm(-Om * h)
        dQ = (Rp @ Qt @ Rp.T - Rm @ Qt @ Rm.T) / (2 * h)
        S = orc.corotation_point(Om, Q, rng.random())
        assert np.allclose(S, dQ, atol=1e-9)


@pytest.mark.parametrize("traceless_G", [True, False])
def test_reactive_stress_conserves_energy(orc, traceless_G):
    """The reactive part of Eq. 5 and the co-rotational term of Eq. 1 are an
    energy-conserving pair: for any velocity gradient G (G_ab = d_b u_a) and
    symmetric traceless Q, H,  G:Pi(Q, H) + H:S(G, Q) = 2 xi (Tr G/3)(Q:H)
    (zero for incompressible flow).  Elastic term off (dQ = 0)."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        G = rng.normal(size=(3, 3))
        if traceless_G:
            G -= np.trace(G) / 3 * np.eye(3)
        Q = rand_sym_traceless(rng)
        H = rand_sym_traceless(rng)
        xi = rng.random()
        Pi = orc.stress_point(Q, H, np.zeros((3, 3, 3)), 0.05, xi)
        S = orc.corotation_point(G, Q, xi)
        lhs = np.sum(G * Pi) + np.sum(H * S)
        rhs = 2 * xi * np.trace(G) / 3 * np.sum(Q * H)
        assert lhs == pytest.approx(rhs, abs=1e-14)


def test_elastic_stress_divergence_converges(orc):
    """For xi = 0 and a uniaxial field with a fixed director (Q and H commute,
    so only the elastic term of Eq. 5 is left) the continuum force is
    F_a = -(K/2) d_a |grad Q|^2 - K d_a Q : lap Q.  The oracle's discrete
    force converges to it at second order."""
    K = 0.05
    n = np.array([np.cos(0.3), np.sin(0.3), 0.0])
    N = np.outer(n, n) - np.eye(3) / 3
    errs = []
    for L in (24, 48):
        kx = 2 * np.pi / L
        y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
        S = 0.2 + 0.1 * np.sin(kx * x) * np.cos(kx * y)
        Sx = 0.1 * kx * np.cos(kx * x) * np.cos(kx * y)
        Sy = -0.1 * kx * np.sin(kx * x) * np.sin(kx * y)
        Sxx = -0.1 * kx ** 2 * np.sin(kx * x) * np.cos(kx * y)
        Syy = Sxx
        Sxy = -0.1 * kx ** 2 * np.cos(kx * x) * np.sin(kx * y)
        lapS = Sxx + Syy
        nn = np.sum(N * N)  # |grad Q|^2 = nn |grad S|^2 ; d_a Q:lap Q = nn d_aS lapS
        Fx = -(K / 2) * nn * 2 * (Sx * Sxx + Sy * Sxy) - K * nn * Sx * lapS
        Fy = -(K / 2) * nn * 2 * (Sx * Sxy + Sy * Syy) - K * nn * Sy * lapS
        Q5 = wl.uniaxial_q5(S[None], n)
        p = params(K=K, xi=0.0)
        f = orc.init_equilibrium(wl.D2Q9, (1, L, L))
        F = orc.fields(wl.D2Q9, p, f, Q5)["F"]
        errs.append(max(np.abs(F[0, 0] - Fx).max(), np.abs(F[1, 0] - Fy).max())
                    / np.abs(Fx).max())
    assert errs[1] < 0.02
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)


@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 7, 6)),
                                           (wl.D3Q19, (4, 3, 5))])
def test_force_is_divergence_of_stress(orc, lattice, shape):
    """F_a = d_b Pi_ab with central differences: summation by parts on the
    periodic lattice gives sum_x u.F = -sum_x G:Pi for any field u, with
    G_ab = d_b u_a by the same differences (Pi is not symmetric here).
    Also sum_x F = 0."""
    rng = np.random.default_rng(5)
    p = params()
    Q5 = rng.normal(scale=0.2, size=(5,) + shape)
    f = orc.init_equilibrium(lattice, shape)
    out = orc.fields(lattice, p, f, Q5)
    Pi, F = out["Pi"], out["F"]
    assert np.abs(Pi - np.swapaxes(Pi, 0, 1)).max() > 1e-3
    u = rng.normal(size=(3,) + shape)
    if lattice == wl.D2Q9:
        u[2] = 0
    G = np.zeros((3, 3) + shape)
    for b, axis in enumerate((-1, -2, -3)):
        G[:, b] = (np.roll(u, -1, axis=axis) - np.roll(u, 1, axis=axis)) / 2
    dims = 2 if lattice == wl.D2Q9 else 3
    lhs = np.sum(u[:dims] * F[:dims])
    rhs = -np.sum(G[:dims] * Pi[:dims])
    assert lhs == pytest.approx(rhs, rel=1e-12)
    assert np.abs(F.sum(axis=(1, 2, 3))).max() < 1e-13


def test_advection_term_converges(orc):
    """With Gamma = 0 and a uniform velocity the right-hand side of Eq. 1 is
    -u.grad Q; compared against the exact derivative of a smooth field."""
    errs = []
    u0 = np.array([0.03, -0.02, 0.01])
    for L in (16, 32):
        k = 2 * np.pi / L
        z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L),
                              indexing="ij")
        ph = k * (x + 2 * y - z)
        amp = np.array([0.1, 0.02, -0.03, 0.05, 0.04])
        Q5 = amp[:, None, None, None] * np.sin(ph)[None]
        dQ = amp[:, None, None, None] * np.cos(ph)[None] * k
        exact = -(u0[0] * dQ + u0[1] * 2 * dQ - u0[2] * dQ)
        u = np.broadcast_to(u0[:, None, None, None], (3, L, L, L)).copy()
        R = orc.rhs(wl.D3Q19, params(Gamma=0.0), Q5, u)
        errs.append(np.abs(R - exact).max() / np.abs(exact).max())
    assert errs[1] < 0.06
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)


def test_rhs_assembles_eq1(orc):
    """R = proj(-u.grad Q + S(W, D, Q) + Gamma H): the oracle's whole-lattice
    right-hand side against its separately pinned pointwise pieces, with a
    compressible u so that the traceless projection is exercised."""
    rng = np.random.default_rng(6)
    shape = (3, 4, 5)
    p = params(Gamma=0.37, xi=0.6)
    Q5 = rng.normal(scale=0.2, size=(5,) + shape)
    u = rng.normal(scale=0.05, size=(3,) + shape)
    R5 = orc.rhs(wl.D3Q19, p, Q5, u)
    Q = full_from5(Q5)
    for cell in [(0, 0, 0), (1, 2, 3), (2, 3, 4)]:
        z, y, x = cell
        nb = lambda a, d: tuple(((c + (d if i == a else 0)) % s)
                                for i, (c, s) in enumerate(zip(cell, shape)))
        axes = {0: 2, 1: 1, 2: 0}  # x, y, z -> array axis of (z, y, x)
        dQ = np.zeros((3, 3, 3))
        lap = np.zeros((3, 3))
        G = np.zeros((3, 3))
        for g in range(3):
            ip, im = nb(axes[g], 1), nb(axes[g], -1)
            dQ[g] = (Q[(..., *ip)] - Q[(..., *im)]) / 2
            lap += Q[(..., *ip)] + Q[(..., *im)] - 2 * Q[(..., *cell)]
            G[:, g] = (u[(..., *ip)] - u[(..., *im)]) / 2
        Qc = Q[(..., *cell)]
        H = orc.molecular_field_point(Qc, lap, p)
        S = orc.corotation_point(G, Qc, p[4])
        R = -np.einsum("g,gab->ab", u[(..., *cell)], dQ) + S + p[3] * H
        R -= np.trace(R) / 3 * np.eye(3)
        got = full_from5(R5[(..., *cell)])
        assert np.allclose(got, R, atol=1e-15)


# ---------------------------------------------------------------------------
# Lattice Boltzmann (Sec. 1.2.1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("lattice", [wl.D2Q9, wl.D3Q19])
def test_lattice_isotropy(orc, lattice):
    c, w = orc.lattice(lattice)
    d = 2 if lattice == wl.D2Q9 else 3
    c = c[:, :d].astype(float)
    assert w.sum() == pytest.approx(1, abs=1e-15)
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(d) / 3,
                       atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    I = np.eye(d)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
           + np.einsum("ad,bc->abcd", I, I)) / 9
    assert np.allclose(m4, iso, atol=1e-16)


@pytest.mark.parametrize("lattice", [wl.D2Q9, wl.D3Q19])
def test_equilibrium_and_source_moments(orc, lattice):
    """sum feq = rho, sum c feq = rho u, sum cc feq = rho/3 I + rho uu;
    sum S_i = 0, sum c S_i = (1 - 1/2tau) F, sum cc S_i = (1-1/2tau)(uF+Fu)."""
    c, _ = orc.lattice(lattice)
    d = 2 if lattice == wl.D2Q9 else 3
    rng = np.random.default_rng(7)
    for _ in range(10):
        rho = 0.8 + 0.4 * rng.random()
        u = np.zeros(3)
        u[:d] = rng.normal(scale=0.05, size=d)
        F = np.zeros(3)
        F[:d] = rng.normal(scale=1e-3, size=d)
        tau = 0.6 + rng.random()
        feq = orc.equilibrium_point(lattice, rho, u)
        src = orc.guo_point(lattice, tau, u, F)
        cc = c.astype(float)
        assert feq.sum() == pytest.approx(rho, rel=1e-14)
        assert np.allclose(cc.T @ feq, rho * u, atol=1e-15)
        assert np.allclose(np.einsum("i,ia,ib->ab", feq, cc, cc)[:d, :d],
                           (rho / 3 * np.eye(3) + rho * np.outer(u, u))[:d, :d],
                           atol=1e-15)
        k = 1 - 1 / (2 * tau)
        assert abs(src.sum()) < 1e-17
        assert np.allclose(cc.T @ src, k * F, atol=1e-17)
        assert np.allclose(np.einsum("i,ia,ib->ab", src, cc, cc)[:d, :d],
                           (k * (np.outer(u, F) + np.outer(F, u)))[:d, :d],
                           atol=1e-17)


def test_velocity_includes_half_force(orc):
    """Eq. 6: from populations at rest (f = w_i) the velocity is F/(2 rho)."""
    w = wl.flat_128x8().with_(shape=(1, 4, 32), size=16, noise=0)
    p = params()
    f = orc.init_equilibrium(wl.D2Q9, w.shape)
    out = orc.fields(wl.D2Q9, p, f, w.initial_q5())
    assert np.abs(out["F"]).max() > 1e-6
    assert np.allclose(out["u"], out["F"] / (2 * out["rho"]), atol=1e-20)


@pytest.mark.parametrize("lattice,tau", [(wl.D2Q9, 1.0), (wl.D2Q9, 0.8),
                                         (wl.D3Q19, 0.9)])
def test_shear_wave_decay(orc, lattice, tau):
    """With Q = 0 and xi = 0 the scheme is plain BGK (for xi != 0 a shear
    flow would induce order through the (2 xi/3) D part of S): a shear wave
    u_x = U sin(k y) decays as exp(-nu k^2 t) with nu = (tau - 1/2)/3."""
    L, U, T = 64, 1e-4, 600
    nz = 1 if lattice == wl.D2Q9 else 2
    shape = (nz, L, 4)
    y = np.arange(L)[None, :, None] * np.ones(shape)
    k = 2 * np.pi / L
    u = np.zeros((3,) + shape)
    u[0] = U * np.sin(k * y)
    f = orc.init_equilibrium(lattice, shape, u=u)
    Q5 = np.zeros((5,) + shape)
    p = params(tau=tau, xi=0.0)
    f, Q5 = orc.step(lattice, p, f, Q5, T)
    assert np.abs(Q5).max() == 0.0
    ux = orc.fields(lattice, p, f, Q5)["u"][0]
    amp = 2 * np.mean(ux * np.sin(k * y))
    nu = (tau - 0.5) / 3
    # the lattice's own O(k^2) correction to nu is ~1e-3 at this k
    assert amp / U == pytest.approx(np.exp(-nu * k * k * T), rel=3e-3)


def test_mass_and_momentum_conserved(orc):
    """Streaming permutes populations and collision keeps sum f; the force is
    a central-difference divergence, so sum_x F = 0 and the total momentum
    sum_x rho u stays constant."""
    rng = np.random.default_rng(8)
    for lattice, shape in ((wl.D2Q9, (1, 9, 10)), (wl.D3Q19, (5, 4, 6))):
        Q5 = rng.normal(scale=0.1, size=(5,) + shape)
        u = rng.normal(scale=0.01, size=(3,) + shape)
        rho = 1 + 0.01 * rng.normal(size=shape)
        f = orc.init_equilibrium(lattice, shape, rho=rho, u=u)
        p = params()
        o0 = orc.observables(lattice, p, f, Q5)
        f2, Q2 = orc.step(lattice, p, f, Q5, 50)
        o1 = orc.observables(lattice, p, f2, Q2)
        assert o1["mass"] == pytest.approx(o0["mass"], rel=1e-14)
        for k in ("mom_x", "mom_y", "mom_z"):
            assert abs(o1[k] - o0[k]) < 1e-13 * np.prod(shape)


def test_d3q19_single_plane_equals_d2q9(orc):
    """With Qxz = Qyz = 0 the D3Q19 lattice one cell thick reproduces D2Q9
    (its out-of-plane populations lump into the D2Q9 weights)."""
    w = wl.flat_128x8().with_(shape=(1, 6, 40), size=20, noise=0)
    Q5 = wl.uniaxial_q5(wl.ball_S((1, 6, 40), 5), (np.cos(0.4), np.sin(0.4), 0))
    Q5 = Q5 + np.random.default_rng(9).uniform(-1e-3, 1e-3, Q5.shape) * \
        np.array([1, 1, 0, 1, 0])[:, None, None, None]
    p = params()
    out = []
    for lattice in (wl.D2Q9, wl.D3Q19):
        f = orc.init_equilibrium(lattice, w.shape)
        f, Q = orc.step(lattice, p, f, Q5, 100)
        fl = orc.fields(lattice, p, f, Q)
        out.append((Q, fl["rho"], fl["u"]))
    for a, b in zip(out[0], out[1]):
        assert np.allclose(a, b, atol=1e-15, rtol=0)


# ---------------------------------------------------------------------------
# Predictor-corrector (Sec. 1.2.2)
# ---------------------------------------------------------------------------

def test_uniform_relaxation_is_second_order_in_time(orc):
    """A uniform uniaxial Q stays uniaxial, the flow stays at rest, and S
    obeys dS/dt = -(3 Gamma/2) f'(S) with f the uniaxial reduction of Eq. 2.
    Refining the time step (Gamma/m over m*n steps) the oracle's error
    against the exact ODE solution falls as 1/m^2 (Heun is second order)."""
    A0, gam, Gam = 0.1, 2.75, 0.3
    S0, n_steps = 0.2, 400

    def rhs(_, S):
        fp = (2 * A0 / 3 * (1 - gam / 3) * S - 2 * A0 * gam / 9 * S ** 2
              + 4 * A0 * gam / 9 * S ** 3)
        return -1.5 * Gam * fp

    exact = solve_ivp(rhs, (0, n_steps), [S0], rtol=1e-13, atol=1e-15).y[0, -1]
    shape = (1, 2, 2)
    f = orc.init_equilibrium(wl.D2Q9, shape)
    Q5 = wl.uniaxial_q5(np.full(shape, S0), (0, 1, 0))
    errs = []
    for m in (1, 2, 4):
        p = params(A0=A0, gamma=gam, Gamma=Gam / m)
        _, Q = orc.step(wl.D2Q9, p, f, Q5, n_steps * m)
        S = np.sqrt(1.5 * np.einsum("ab...,ab...->...", full_from5(Q),
                                    full_from5(Q)))
        errs.append(abs(S.mean() - exact))
        assert np.ptp(S) == 0.0
    assert errs[0] / errs[1] == pytest.approx(4, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(4, rel=0.05)
    assert errs[0] < 1e-4


def test_uniform_nematic_is_a_fixed_point(orc):
    shape = (1, 3, 3)
    g = 2.8
    Q5 = wl.uniaxial_q5(np.full(shape, s_nematic(g)), (0.6, 0.8, 0))
    f = orc.init_equilibrium(wl.D2Q9, shape)
    f2, Q2 = orc.step(wl.D2Q9, params(gamma=g), f, Q5, 100)
    assert np.abs(Q2 - Q5).max() < 1e-15
    assert np.abs(f2 - f).max() < 1e-15


# ---------------------------------------------------------------------------
# Whole runs: the flat interface of Sec. 2.1
# ---------------------------------------------------------------------------

def tanh_profile(x, xi, lam, Sn=1 / 3):
    return Sn / 2 * (1 - np.tanh((x - xi) / (2 * lam)))


def equilibrium_profile(orc, K, steps=3000):
    w = wl.flat_128x8().with_(shape=(1, 4, 128), noise=0.0)
    p = params(K=K)
    f = orc.init_equilibrium(wl.D2Q9, w.shape)
    f, Q = orc.step(wl.D2Q9, p, f, w.initial_q5(), steps)
    return orc.observables(wl.D2Q9, p, f, Q)


def test_flat_interface_static_at_coexistence(orc):
    """Sec. 2.1: at gamma_NI = 2.7 the flat interface does not move.  From
    the centred step the right interface stays at x = 63.5 (to within the
    1e-4-cell sloshing of the start-up sound waves, which die out)."""
    w = wl.flat_128x8()
    p = wl.param_vector(w.params)
    f = orc.init_equilibrium(w.lattice, w.shape)
    f, Q = orc.step(w.lattice, p, f, w.initial_q5(), 3500)
    x1 = orc.observables(w.lattice, p, f, Q)["x_iface"]
    f, Q = orc.step(w.lattice, p, f, Q, 500)
    x2 = orc.observables(w.lattice, p, f, Q)["x_iface"]
    assert abs(x1 - 63.5) < 1e-3 and abs(x2 - 63.5) < 1e-3
    assert abs(x2 - x1) / 500 < 1e-8
    # the out-of-plane components stay at the noise level
    assert np.abs(Q[[2, 4]]).max() < 2e-6


def test_tanh_profile_second_order(orc):
    """Eq. 7: the relaxed profile is S_n/2 [1 - tanh((x - x_i)/2 lambda)]
    with lambda = sqrt(27K/(A0 gamma)).  The discrete profile deviates by an
    O(h^2/lambda^2) amount: quadrupling K (doubling lambda) cuts the largest
    deviation about four times."""
    devs = []
    x = np.arange(32, 96)
    for K in (0.02, 0.08):
        prof = equilibrium_profile(orc, K)["s_profile"][32:96]
        lam = np.sqrt(27 * K / (0.1 * 2.7))
        fit = least_squares(lambda a: tanh_profile(x, a[0], lam) - prof,
                            [63.5])
        devs.append(np.abs(tanh_profile(x, fit.x[0], lam) - prof).max())
        assert abs(fit.x[0] - 63.5) < 5e-3
    assert devs[0] < 3e-3
    assert devs[1] / devs[0] == pytest.approx(0.25, abs=0.06)


@pytest.mark.parametrize("delta", [-0.01, 0.01])
def test_interface_velocity_near_coexistence(orc, delta):
    """Sec. 2.1: off coexistence the interface moves at constant speed, the
    nematic growing for gamma > gamma_NI.  Allen-Cahn travelling-wave
    estimate from Eqs. 2 and 7: v = (3 Gamma/2) df / int S'^2 with
    df = 10 A0 delta/729 and int S'^2 = S_n^2/(6 lambda), i.e.
    v = (10/9) Gamma A0 lambda delta."""
    g = 2.7 + delta
    w = wl.flat_128x8().with_(shape=(1, 4, 256), size=128, noise=0.0)
    p = params(gamma=g)
    f = orc.init_equilibrium(wl.D2Q9, w.shape)
    f, Q = orc.step(wl.D2Q9, p, f, w.initial_q5(), 2000)
    x1 = orc.observables(wl.D2Q9, p, f, Q)["x_iface"]
    f, Q = orc.step(wl.D2Q9, p, f, Q, 2000)
    x2 = orc.observables(wl.D2Q9, p, f, Q)["x_iface"]
    v = (x2 - x1) / 2000
    lam = np.sqrt(27 * 0.02 / (0.1 * g))
    v_est = 10 / 9 * 0.3 * 0.1 * lam * delta
    assert np.sign(v) == np.sign(delta)
    assert v == pytest.approx(v_est, rel=0.15)


# ---------------------------------------------------------------------------
# The complex-step twin of the oracle (used as the reference gradient)
# ---------------------------------------------------------------------------

def test_complex_step_twin_matches_real_oracle_and_differences(orc, orc_cs):
    """The complex build with zero imaginary parts reproduces the real
    oracle bit for bit, and its derivatives agree with FP64 central
    differences of the real oracle (h = 1e-6)."""
    w = wl.disc_256().with_(shape=(1, 20, 22), size=5, noise=1e-4, seed=3)
    p = wl.param_vector(w.params)
    Q0 = w.initial_q5()
    f0 = orc.init_equilibrium(w.lattice, w.shape)
    f_r, Q_r = orc.step(w.lattice, p, f0, Q0, 25)
    f_c, Q_c = orc_cs.step(w.lattice, p.astype(complex), f0.astype(complex),
                           Q0.astype(complex), 25)
    assert np.array_equal(Q_r, Q_c.real) and np.array_equal(f_r, f_c.real)

    def L(pv, Q, cs):
        o = orc_cs if cs else orc
        f, Qe = o.step(w.lattice, pv, o.init_equilibrium(w.lattice, w.shape), Q, 25)
        R = o.observables(w.lattice, pv, f, Qe)["radius"]
        u = o.fields(w.lattice, pv, f, Qe)["u"]
        return (R - 5.0) ** 2 + 10 * np.sqrt(np.sum(u * u))

    h = 1e-6
    for k in (1, 2, 3):  # K, gamma, Gamma
        pc = p.astype(complex)
        pc[k] += 1e-30j
        d_cs = L(pc, Q0.astype(complex), True).imag / 1e-30
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        d_fd = (L(pp, Q0, False) - L(pm, Q0, False)) / (2 * h)
        assert d_cs == pytest.approx(d_fd, rel=1e-5)
