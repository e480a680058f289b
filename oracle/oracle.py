"""ctypes wrapper over liboracle.so (test infrastructure only)."""
import ctypes
import os

import numpy as np

from . import build as _build

D2Q9 = 0
D3Q19 = 1
PARAM_NAMES = ("A0", "K", "gamma", "Gamma", "xi", "tau")
OBS_NAMES = ("mass", "mom_x", "mom_y", "mom_z", "s_area", "radius",
             "x_iface", "max_u", "free_energy", "nonfinite")


def nvel(lattice):
    return 9 if lattice == D2Q9 else 19


_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_long
_D = ctypes.c_double


class Oracle:
    """FP64 oracle (complex=False) or its complex-step twin (complex=True)."""

    def __init__(self, lib, complex_step=False):
        self.cs = complex_step
        self._lib = lib
        self.dtype = np.complex128 if complex_step else np.float64
        sfx = "_cs" if complex_step else ""
        self._f = {}
        sigs = {
            "orc_lattice": [_I, _P, _P],
            "orc_molecular_field_point": [_P, _P, _P, _P],
            "orc_stress_point": [_P, _P, _P, None, None, _P],
            "orc_corotation_point": [_P, _P, None, _P],
            "orc_equilibrium_point": [_I, None, _P, _P],
            "orc_guo_point": [_I, None, _P, _P, _P],
            "orc_init_equilibrium": [_I, _I, _I, _I, _P, _P, _P],
            "orc_fields": [_I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P],
            "orc_rhs": [_I, _I, _I, _I, _P, _P, _P, _P],
            "orc_step": [_I, _I, _I, _I, _P, _P, _P, _L],
            "orc_observables": [_I, _I, _I, _I, _P, _P, _P, _D, _P, _P],
        }
        for name, args in sigs.items():
            fn = getattr(lib, name + sfx)
            # scalar `rt` arguments: double, or a complex passed by value
            # (two doubles in registers on both x86-64 and AArch64)
            fn.argtypes = None
            self._f[name] = (fn, args)
            fn.restype = _I if name not in ("orc_molecular_field_point",
                                            "orc_stress_point",
                                            "orc_corotation_point",
                                            "orc_equilibrium_point",
                                            "orc_guo_point") else None

    # -- helpers -------------------------------------------------------
    def _arr(self, a, shape=None):
        a = np.ascontiguousarray(a, dtype=self.dtype)
        if shape is not None:
            a = a.reshape(shape)
        return a

    def _scalar(self, v):
        if self.cs:
            return _Complex(complex(v))
        return _D(float(v))

    def _call(self, name, *args):
        fn, _ = self._f[name]
        conv = []
        for a in args:
            if isinstance(a, np.ndarray):
                conv.append(_P(a.ctypes.data))
            elif a is None:
                conv.append(_P(None))
            else:
                conv.append(a)
        return fn(*conv)

    def set_mrt(self, lattice, rates=None):
        """MRT collision with q rates in the oracle's moment order (see
        nlc_oracle.c), or BGK again with rates=None."""
        fn = getattr(self._lib, "orc_set_mrt" + ("_cs" if self.cs else ""))
        fn.restype = _I
        r = None if rates is None else np.ascontiguousarray(rates, dtype=np.float64)
        rc = fn(_I(lattice), _P(None) if r is None else _P(r.ctypes.data))
        assert rc == 0
        self._mrt_rates = r  # keep alive

    def mrt_point(self, lattice, f, rho, u, F):
        fn = getattr(self._lib, "orc_mrt_point" + ("_cs" if self.cs else ""))
        fn.restype = _I
        f = self._arr(f)
        u = self._arr(u, (3,))
        F = self._arr(F, (3,))
        post = np.zeros_like(f)
        rc = fn(_I(lattice), _P(f.ctypes.data), self._scalar(rho), _P(u.ctypes.data),
                _P(F.ctypes.data), _P(post.ctypes.data))
        assert rc == 0
        return post

    def mrt_basis(self, lattice):
        fn = getattr(self._lib, "orc_mrt_basis" + ("_cs" if self.cs else ""))
        fn.restype = _I
        q = nvel(lattice)
        v = np.zeros((q, q))
        rc = fn(_I(lattice), _P(v.ctypes.data))
        assert rc == q
        return v

    def set_stencil(self, kind):
        """0: standard stencils (2d+1-point Laplacian, central first
        derivatives); 1: the isotropic stencils of the lattice's neighbour
        set.  Applies to every later call of this oracle (real or complex)."""
        fn = getattr(self._lib, "orc_set_stencil" + ("_cs" if self.cs else ""))
        fn.argtypes = [_I]
        fn.restype = _I
        assert fn(int(kind)) == 0

    def set_threads(self, n=0):
        """OpenMP threads of the cell loops (n <= 0: unchanged); returns the
        count in effect."""
        fn = self._lib.orc_set_threads
        fn.argtypes = [_I]
        fn.restype = _I
        return int(fn(int(n)))

    # -- lattice -------------------------------------------------------
    def lattice(self, lattice):
        q = nvel(lattice)
        c = np.zeros((q, 3), dtype=np.int32)
        w = np.zeros(q, dtype=np.float64)
        rc = self._call("orc_lattice", _I(lattice), c, w)
        assert rc == q
        return c, w

    # -- pointwise -----------------------------------------------------
    def molecular_field_point(self, Q, lapQ, params):
        Q = self._arr(Q, (9,))
        L = self._arr(lapQ, (9,))
        p = self._arr(params, (6,))
        H = np.zeros(9, dtype=self.dtype)
        self._call("orc_molecular_field_point", Q, L, p, H)
        return H.reshape(3, 3)

    def stress_point(self, Q, H, dQ, K, xi):
        Q = self._arr(Q, (9,))
        H = self._arr(H, (9,))
        dQ = self._arr(dQ, (27,))
        Pi = np.zeros(9, dtype=self.dtype)
        self._call("orc_stress_point", Q, H, dQ, self._scalar(K),
                   self._scalar(xi), Pi)
        return Pi.reshape(3, 3)

    def corotation_point(self, Gu, Q, xi):
        G = self._arr(Gu, (9,))
        Q = self._arr(Q, (9,))
        S = np.zeros(9, dtype=self.dtype)
        self._call("orc_corotation_point", G, Q, self._scalar(xi), S)
        return S.reshape(3, 3)

    def equilibrium_point(self, lattice, rho, u):
        u = self._arr(u, (3,))
        feq = np.zeros(nvel(lattice), dtype=self.dtype)
        self._call("orc_equilibrium_point", _I(lattice), self._scalar(rho), u,
                   feq)
        return feq

    def guo_point(self, lattice, tau, u, F):
        u = self._arr(u, (3,))
        F = self._arr(F, (3,))
        s = np.zeros(nvel(lattice), dtype=self.dtype)
        self._call("orc_guo_point", _I(lattice), self._scalar(tau), u, F, s)
        return s

    # -- grids ---------------------------------------------------------
    @staticmethod
    def _dims(Q5):
        _, nz, ny, nx = Q5.shape
        return nx, ny, nz

    def init_equilibrium(self, lattice, shape, rho=None, u=None):
        nz, ny, nx = shape
        f = np.zeros((nvel(lattice), nz, ny, nx), dtype=self.dtype)
        r = None if rho is None else self._arr(rho, (nz, ny, nx))
        uu = None if u is None else self._arr(u, (3, nz, ny, nx))
        rc = self._call("orc_init_equilibrium", _I(lattice), _I(nx), _I(ny),
                        _I(nz), r, uu, f)
        assert rc == 0
        return f

    def fields(self, lattice, params, f, Q5):
        f = self._arr(f)
        Q5 = self._arr(Q5)
        nx, ny, nz = self._dims(Q5)
        p = self._arr(params, (6,))
        sh = (nz, ny, nx)
        out = {
            "H": np.zeros((5,) + sh, dtype=self.dtype),
            "Pi": np.zeros((3, 3) + sh, dtype=self.dtype),
            "F": np.zeros((3,) + sh, dtype=self.dtype),
            "rho": np.zeros(sh, dtype=self.dtype),
            "u": np.zeros((3,) + sh, dtype=self.dtype),
        }
        rc = self._call("orc_fields", _I(lattice), _I(nx), _I(ny), _I(nz), p,
                        f, Q5, out["H"], out["Pi"], out["F"], out["rho"],
                        out["u"])
        assert rc == 0
        return out

    def rhs(self, lattice, params, Q5, u):
        Q5 = self._arr(Q5)
        nx, ny, nz = self._dims(Q5)
        u = self._arr(u, (3, nz, ny, nx))
        p = self._arr(params, (6,))
        R = np.zeros_like(Q5)
        rc = self._call("orc_rhs", _I(lattice), _I(nx), _I(ny), _I(nz), p, Q5,
                        u, R)
        assert rc == 0
        return R

    def step(self, lattice, params, f, Q5, nsteps):
        """Advance copies of (f, Q5) by nsteps; returns the new pair."""
        f = self._arr(f).copy()
        Q5 = self._arr(Q5).copy()
        nx, ny, nz = self._dims(Q5)
        p = self._arr(params, (6,))
        rc = self._call("orc_step", _I(lattice), _I(nx), _I(ny), _I(nz), p, f,
                        Q5, _L(int(nsteps)))
        if rc != 0:
            raise RuntimeError(f"orc_step failed: {rc}")
        return f, Q5

    def observables(self, lattice, params, f, Q5, s_ref=1.0 / 3.0):
        f = self._arr(f)
        Q5 = self._arr(Q5)
        nx, ny, nz = self._dims(Q5)
        p = self._arr(params, (6,))
        out = np.zeros(10, dtype=self.dtype)
        prof = np.zeros(nx, dtype=self.dtype)
        rc = self._call("orc_observables", _I(lattice), _I(nx), _I(ny), _I(nz),
                        p, f, Q5, _D(s_ref), out, prof)
        assert rc == 0
        d = dict(zip(OBS_NAMES, out))
        d["s_profile"] = prof
        return d


class _Complex(ctypes.Structure):
    """C `double _Complex` passed by value: laid out as two doubles."""
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]

    def __init__(self, z):
        super().__init__(z.real, z.imag)


_cache = {}


def get(complex_step=False):
    """The oracle (built on first use)."""
    key = bool(complex_step)
    if key not in _cache:
        path = _build.build()
        lib = _cache.get("lib")
        if lib is None:
            lib = ctypes.CDLL(path)
            _cache["lib"] = lib
        _cache[key] = Oracle(lib, complex_step=key)
    return _cache[key]
