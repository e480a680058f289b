"""The library's pointwise physics (csrc/physics.cuh, compiled for the host)
against the oracle's pointwise functions: H (Eq. 3), the stress (Eq. 5),
the co-rotational term and the right-hand side of Eq. 1.  Runs on the CPU."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
IDX5 = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2))


@pytest.fixture(scope="module")
def hp(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("hp") / "libhp.so"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr",
                           "-Xcompiler", "-fPIC", "-shared", "-x", "cu",
                           os.path.join(HERE, "host_physics.cu"), "-o", str(out)])
    lib = ctypes.CDLL(str(out))
    for name in ("hp_molecular_field", "hp_stress3", "hp_corotation", "hp_be_rhs3",
                 "hp_lattice"):
        getattr(lib, name).restype = None
    lib.hp_collide.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_double,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.hp_collide_mrt.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_double,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]
    lib.hp_lb_pairs_f32.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]
    lib.hp_corotation.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                  ctypes.c_void_p]
    return lib


def P(a):
    return ctypes.c_void_p(a.ctypes.data)


def sym5(rng, s=0.3):
    A = rng.normal(size=(3, 3)) * s
    A = (A + A.T) / 2
    A -= np.trace(A) / 3 * np.eye(3)
    return A, np.array([A[a, b] for a, b in IDX5])


def params(rng):
    return np.array([0.05 + 0.1 * rng.random(), 0.01 + 0.05 * rng.random(),
                     2.6 + 0.5 * rng.random(), 0.2 + 0.3 * rng.random(),
                     rng.random(), 0.8 + rng.random()])


def test_molecular_field(hp, orc):
    rng = np.random.default_rng(0)
    for _ in range(50):
        Q, q = sym5(rng)
        L, l = sym5(rng)
        p = params(rng)
        h = np.zeros(5)
        hp.hp_molecular_field(P(q), P(l), P(p), P(h))
        H = orc.molecular_field_point(Q, L, p)
        assert np.allclose(h, [H[a, b] for a, b in IDX5], rtol=1e-13, atol=1e-16)


def test_stress(hp, orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        Q, q = sym5(rng)
        H, h = sym5(rng)
        dQ = np.zeros((3, 3, 3))
        dq = np.zeros((3, 5))
        for g in range(3):
            dQ[g], dq[g] = sym5(rng)
        p = params(rng)
        pi = np.zeros(9)
        hp.hp_stress3(P(q), P(h), P(np.ascontiguousarray(dq)), P(p), P(pi))
        ref = orc.stress_point(Q, H, dQ, p[1], p[4])
        assert np.allclose(pi.reshape(3, 3), ref, rtol=1e-13, atol=1e-16)


def test_corotation(hp, orc):
    rng = np.random.default_rng(2)
    for _ in range(50):
        Q, q = sym5(rng)
        G = rng.normal(size=(3, 3))
        xi = rng.random()
        s = np.zeros(5)
        hp.hp_corotation(P(np.ascontiguousarray(G)), P(q), xi, P(s))
        ref = orc.corotation_point(G, Q, xi)
        assert np.allclose(s, [ref[a, b] for a, b in IDX5], rtol=1e-13, atol=1e-16)


def test_rhs_traceless_projection(hp, orc):
    """be_rhs against Eq. 1 assembled from the oracle's pieces, with the
    orthogonal traceless projection (compressible G)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        Q, q = sym5(rng)
        L, l = sym5(rng)
        dQ = np.zeros((3, 3, 3))
        dq = np.zeros((3, 5))
        for g in range(3):
            dQ[g], dq[g] = sym5(rng)
        u = rng.normal(scale=0.05, size=3)
        G = rng.normal(scale=0.05, size=(3, 3))
        p = params(rng)
        r = np.zeros(5)
        hp.hp_be_rhs3(P(q), P(np.ascontiguousarray(dq)), P(l), P(u),
                      P(np.ascontiguousarray(G)), P(p), P(r))
        H = orc.molecular_field_point(Q, L, p)
        S = orc.corotation_point(G, Q, p[4])
        R = -np.einsum("g,gab->ab", u, dQ) + S + p[3] * H
        R -= np.trace(R) / 3 * np.eye(3)
        assert np.allclose(r, [R[a, b] for a, b in IDX5], rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("lattice", [0, 1])
def test_collision_with_source(hp, orc, lattice):
    """The pairwise BGK + source update against f - (f - feq)/tau + S_i from
    the oracle's equilibrium and source term (same velocity matched up)."""
    q = 9 if lattice == 0 else 19
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    hp.hp_lattice(lattice, P(c), P(w))
    co, wo = orc.lattice(lattice)
    perm = [int(np.where((co == cv).all(axis=1))[0][0]) for cv in c]
    rng = np.random.default_rng(4)
    d = 2 if lattice == 0 else 3
    for _ in range(30):
        p = params(rng)
        rho = 1 + 0.05 * rng.normal()
        u = np.zeros(3)
        u[:d] = rng.normal(scale=0.05, size=d)
        F = np.zeros(3)
        F[:d] = rng.normal(scale=1e-3, size=d)
        f = orc.equilibrium_point(lattice, rho, u) + rng.normal(scale=1e-3, size=q)
        g = f[perm] - w
        hp.hp_collide(lattice, P(g), rho, P(u), P(F), P(p))
        feq = orc.equilibrium_point(lattice, rho, u)
        S = orc.guo_point(lattice, p[5], u, F)
        ref = f - (f - feq) / p[5] + S
        assert np.allclose(g + w, ref[perm], rtol=0, atol=1e-15)


@pytest.mark.parametrize("lattice", [0, 1])
@pytest.mark.parametrize("tau", [0.8, 1.5, "random"])
def test_packed_fp32_collision_matches_oracle(hp, orc, lattice, tau):
    """The FP32 kernels' moments and collision on packed opposite pairs
    (packed.cuh: moments_pairs, collide_bgk_pairs) against the oracle's
    equilibrium and source term, f* = f - (f - feq)/tau + S_i with rho and u
    of Eq. 6 (u with F/2), at tau != 1, where the (1 - 1/tau) f part of the
    collision is not zero (tau = 1.5 is the paper's value, Sec. 2)."""
    q = 9 if lattice == 0 else 19
    d = 2 if lattice == 0 else 3
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    hp.hp_lattice(lattice, P(c), P(w))
    rng = np.random.default_rng(21 + lattice)
    worst = 0.0
    for _ in range(40):
        p = params(rng)
        p[5] = rng.uniform(0.6, 2.0) if tau == "random" else tau
        rho = 1 + 0.05 * rng.normal()
        u0 = np.zeros(3)
        u0[:d] = rng.normal(scale=0.05, size=d)
        F = np.zeros(3)
        F[:d] = rng.normal(scale=1e-3, size=d)
        co, _ = orc.lattice(lattice)
        perm = [int(np.where((co == cv).all(axis=1))[0][0]) for cv in c]
        f = orc.equilibrium_point(lattice, rho, u0)[perm] + rng.normal(scale=2e-3, size=q)
        g32 = (f - w).astype(np.float32)
        f = g32.astype(np.float64) + w          # the FP32 input, exactly
        F32 = F.astype(np.float32)
        Fd = F32.astype(np.float64)
        ru = np.zeros(4, dtype=np.float32)
        hp.hp_lb_pairs_f32(lattice, P(g32), P(F32), P(p), P(ru))
        rho_ref = f.sum()
        u_ref = (c.T.astype(np.float64) @ f + Fd / 2) / rho_ref
        feq = orc.equilibrium_point(lattice, rho_ref, u_ref)[perm]
        S = orc.guo_point(lattice, p[5], u_ref, Fd)[perm]
        ref = f - (f - feq) / p[5] + S
        gref = ref - w
        assert ru[0] == pytest.approx(rho_ref, rel=1e-6)
        assert np.allclose(ru[1:], u_ref, rtol=0, atol=1e-6 * np.abs(u_ref).max())
        err = np.abs(g32 - gref).max() / np.abs(gref).max()
        worst = max(worst, err)
    # a few float32 roundings of terms of the size of the deviations
    assert worst < 2e-6


@pytest.mark.parametrize("lattice", [0, 1])
def test_mrt_collision_matches_oracle(hp, orc, lattice):
    """The library's MRT collision (its own moment rows, its own velocity
    order) against the oracle's, for random rates; the two moment bases are
    the same rows up to the velocity order."""
    q = 9 if lattice == 0 else 19
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    hp.hp_lattice(lattice, P(c), P(w))
    co, wo = orc.lattice(lattice)
    perm = [int(np.where((co == cv).all(axis=1))[0][0]) for cv in c]
    rng = np.random.default_rng(12)
    rates = rng.uniform(0.6, 1.9, size=q)
    orc.set_mrt(lattice, rates)
    try:
        v = np.zeros(q * q)
        hp.hp_moment_basis(lattice, P(v))
        assert np.allclose(v.reshape(q, q), orc.mrt_basis(lattice)[:, perm], atol=1e-13)
        d = 2 if lattice == 0 else 3
        for _ in range(30):
            p = params(rng)
            rho = 1 + 0.05 * rng.normal()
            u = np.zeros(3)
            u[:d] = rng.normal(scale=0.05, size=d)
            F = np.zeros(3)
            F[:d] = rng.normal(scale=1e-3, size=d)
            f = orc.equilibrium_point(lattice, rho, u) + rng.normal(scale=1e-3, size=q)
            # rho and u of Eq. 6 from f itself: then the mass and momentum
            # rows of f - feq + Ft/2 vanish, as in every step
            rho = f.sum()
            u = (co.T @ f + F / 2) / rho
            g = f[perm] - w
            hp.hp_collide_mrt(lattice, P(g), rho, P(u), P(F), P(p), P(rates))
            ref = orc.mrt_point(lattice, f, rho, u, F)
            assert np.allclose(g + w, ref[perm], rtol=0, atol=2e-15)
    finally:
        orc.set_mrt(lattice, None)


# piece id: (inputs, outputs)
PIECES = {0: (10, 5), 1: (25, 9), 2: (14, 5), 3: (37, 5), 4: (11, 12), 5: (22, 22)}


def piece_input(k, rng):
    if k == 0:
        return np.concatenate([sym5(rng)[1], sym5(rng)[1]])
    if k == 1:
        return np.concatenate([sym5(rng)[1], sym5(rng)[1]] + [sym5(rng)[1] for _ in range(3)])
    if k == 2:
        return np.concatenate([rng.normal(size=9), sym5(rng)[1]])
    if k == 3:
        return np.concatenate([sym5(rng)[1]] + [sym5(rng)[1] for _ in range(3)]
                              + [sym5(rng)[1], rng.normal(scale=0.05, size=3),
                                 rng.normal(scale=0.05, size=9)])
    q = 9 if k == 4 else 19
    g = rng.normal(scale=0.01, size=q)
    F = rng.normal(scale=1e-3, size=2 if k == 4 else 3)
    return np.concatenate([g, F])


@pytest.mark.parametrize("k", sorted(PIECES))
def test_pointwise_adjoints_dot_product(hp, k):
    """<ob, J v> (complex step) == <J^T ob, v> + <pb, vp> (hand adjoint) for
    H, the stress, the co-rotation, Eq. 1's right-hand side and the LB cell
    update (moments + collision), including the gamma, K, Gamma adjoints."""
    nin, nout = PIECES[k]
    rng = np.random.default_rng(100 + k)
    hp.hp_piece_jvp.restype = None
    hp.hp_piece_vjp.restype = None
    for _ in range(20):
        x = piece_input(k, rng)
        assert x.size == nin
        p = params(rng)
        v = rng.normal(size=nin)
        vp = np.zeros(6)
        vp[[1, 2, 3]] = rng.normal(size=3)  # K, gamma, Gamma
        jv = np.zeros(nout)
        hp.hp_piece_jvp(ctypes.c_int(k), P(x), ctypes.c_int(nin), P(p), P(v), P(vp),
                        ctypes.c_int(nout), P(jv))
        ob = rng.normal(size=nout)
        ib = np.zeros(nin)
        pb = np.zeros(3)
        hp.hp_piece_vjp(ctypes.c_int(k), P(x), P(p), P(ob), P(ib), P(pb))
        lhs = ob @ jv
        rhs = ib @ v + pb[0] * vp[2] + pb[1] * vp[1] + pb[2] * vp[3]
        assert lhs == pytest.approx(rhs, rel=1e-11, abs=1e-13)


def test_float_float_sums_of_the_observables_are_nearly_exact(hp):
    """The observables' per-thread running sums (AccFF: Knuth's TwoSum on
    float32, read out in float64) against the exact sum (math.fsum) of the
    same float32 terms: within 2^-40 of the sum of magnitudes over a
    million terms of mixed sign and magnitude (a thread of the observables
    kernels sums tens of terms), where a plain float32 sum is off by three
    orders more; products by add_prod likewise (exact float32 products in
    float64)."""
    import math
    rng = np.random.default_rng(71)
    n = 1 << 20
    v = (rng.standard_normal(n) * 10.0 ** rng.integers(-4, 3, n)).astype(np.float32)
    w = (1.0 + 1e-3 * rng.standard_normal(n)).astype(np.float32)
    hp.hp_accff_sum.restype = ctypes.c_double
    hp.hp_accff_sum.argtypes = [ctypes.c_void_p, ctypes.c_int]
    hp.hp_accff_dot.restype = ctypes.c_double
    hp.hp_accff_dot.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    exact = math.fsum(v.astype(np.float64))
    mag = float(np.abs(v.astype(np.float64)).sum())
    got = hp.hp_accff_sum(P(v), n)
    assert abs(got - exact) < 2.0 ** -40 * mag
    naive = np.float32(0)
    for x in v[:65536]:
        naive += x
    ex16 = math.fsum(v[:65536].astype(np.float64))
    assert abs(float(naive) - ex16) > 1e3 * abs(hp.hp_accff_sum(P(v), 65536) - ex16)
    prods = v.astype(np.float64) * w.astype(np.float64)  # exact in float64
    exact_dot = math.fsum(prods)
    got_dot = hp.hp_accff_dot(P(v), P(w), n)
    assert abs(got_dot - exact_dot) < 2.0 ** -40 * float(np.abs(prods).sum())


def test_fp32_gradient_contraction_is_the_full_tensor_contraction(hp):
    """grad_dot in float32 (packed pairs) against d_a Q : d_b Q summed over
    all nine entries of the full tensors in float64 (Qzz = -Qxx - Qyy)."""
    hp.hp_grad_dot_f32.restype = ctypes.c_float
    hp.hp_grad_dot_f32.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    rng = np.random.default_rng(73)

    def full(q):
        return np.array([[q[0], q[1], q[2]], [q[1], q[3], q[4]],
                         [q[2], q[4], -q[0] - q[3]]])

    for _ in range(200):
        A = rng.standard_normal(5).astype(np.float32)
        B = rng.standard_normal(5).astype(np.float32)
        ref = float(np.sum(full(A.astype(np.float64)) * full(B.astype(np.float64))))
        got = hp.hp_grad_dot_f32(P(A), P(B))
        scale = float(np.sum(np.abs(full(A.astype(np.float64)) * full(B.astype(np.float64)))))
        assert abs(got - ref) < 1e-6 * scale
