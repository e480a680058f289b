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
    for name in ("hp_molecular_field", "hp_stress3", "hp_corotation", "hp_be_rhs3"):
        getattr(lib, name).restype = None
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
