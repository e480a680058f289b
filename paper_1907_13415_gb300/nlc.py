"""Python binding of libnlc's C ABI (include/nlc.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Function names match the C entry points; `Simulation` is a
small convenience wrapper over them.  There is no fallback: if libnlc.so
cannot be loaded, every call raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

NLC_OK = 0
STATUS = {0: "NLC_OK", -1: "NLC_EINVAL", -2: "NLC_ENOMEM", -3: "NLC_ECUDA",
          -4: "NLC_EUNSTABLE", -5: "NLC_ETIMEOUT", -6: "NLC_ECORRUPT",
          -7: "NLC_EUNSUPPORTED"}
NLC_D2Q9, NLC_D3Q19 = 0, 1
NLC_FP64, NLC_FP32, NLC_FP32_QF64 = 0, 1, 2
NLC_SCHED_FUSED, NLC_SCHED_UNFUSED = 0, 1
NLC_STATIC_MAX_CELLS, NLC_STATIC_MAX_NX = 65536, 4096


class NlcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class nlc_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("lattice", ctypes.c_int32),
                ("precision", ctypes.c_int32)]


class nlc_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("A0", "K", "gamma", "Gamma", "xi", "tau", "rho0")]


class nlc_obs(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("mom", ctypes.c_double * 3),
                ("s_area", ctypes.c_double), ("radius", ctypes.c_double),
                ("x_iface", ctypes.c_double), ("max_u", ctypes.c_double),
                ("free_energy", ctypes.c_double), ("u_l2", ctypes.c_double),
                ("nonfinite", ctypes.c_int64), ("step", ctypes.c_int64)]

    def as_dict(self):
        return dict(mass=self.mass, mom_x=self.mom[0], mom_y=self.mom[1],
                    mom_z=self.mom[2], s_area=self.s_area, radius=self.radius,
                    x_iface=self.x_iface, max_u=self.max_u,
                    free_energy=self.free_energy, u_l2=self.u_l2,
                    nonfinite=self.nonfinite, step=self.step)


class nlc_loss(ctypes.Structure):
    _fields_ = [("target_radius", ctypes.c_double), ("w_radius", ctypes.c_double),
                ("w_velocity", ctypes.c_double)]


class nlc_tune(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int32), ("taper", ctypes.c_int32),
                ("from_cache", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("trial_steps", ctypes.c_int32),
                ("best_ms", ctypes.c_double), ("default_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class nlc_grad(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("loss", "radius", "u_l2", "dgamma", "dK", "dGamma")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libnlc.so (compiling it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise OSError(f"libnlc.so not found at {path}; run build()")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                      ctypes.c_double)
    sig = {
        "nlc_create": ([ctypes.POINTER(nlc_grid), ctypes.POINTER(nlc_params),
                        P, ctypes.POINTER(P)], I32),
        "nlc_create_batch": ([I32, P, P, P, ctypes.POINTER(P)], I32),
        "nlc_count": ([P], I32),
        "nlc_set_graph": ([P, I32], I32),
        "nlc_set_check": ([P, I32], I32),
        "nlc_set_wait_budget": ([P, I64], I32),
        "nlc_set_persistent": ([P, I32], I32),
        "nlc_set_params": ([P, I32, ctypes.POINTER(nlc_params)], I32),
        "nlc_set_mrt": ([P, I32, P, I32], I32),
        "nlc_set_stencil": ([P, I32], I32),
        "nlc_set_schedule": ([P, I32], I32),
        "nlc_set_chunk": ([P, I32, I32], I32),
        "nlc_get_chunk": ([P, I32, P], I32),
        "nlc_autotune": ([P, I32, ctypes.POINTER(nlc_tune)], I32),
        "nlc_set_fields": ([P, I32, P, P, P], I32),
        "nlc_set_fields_f32": ([P, I32, P], I32),
        "nlc_get_fields": ([P, I32, P, P, P], I32),
        "nlc_get_populations": ([P, I32, P], I32),
        "nlc_step": ([P, I64], I32),
        "nlc_observables": ([P, I32, ctypes.POINTER(nlc_obs), P], I32),
        "nlc_last_error": ([P], ctypes.c_char_p),
        "nlc_destroy": ([P], None),
        "nlc_lattice_velocities": ([I32, P, P], I32),
        "nlc_set_timing": ([P, I32], I32),
        "nlc_save": ([P, P, ctypes.POINTER(ctypes.c_size_t)], I32),
        "nlc_adjoint": ([P, P, I64, I32, P, P], I32),
        "nlc_observables_static": ([ctypes.POINTER(nlc_grid), ctypes.POINTER(nlc_params),
                                    P, P, P, ctypes.POINTER(nlc_obs)], I32),
        "nlc_load": ([P, P, ctypes.c_size_t], I32),
        "nlc_get_timing": ([P, I32, P, P, P], I32),
        "nlc_timing_name": ([I32], ctypes.c_char_p),
        "nlc_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return ["nlc_create", "nlc_create_batch", "nlc_count", "nlc_set_graph", "nlc_set_check",
            "nlc_set_params", "nlc_set_mrt", "nlc_set_stencil",
            "nlc_set_schedule", "nlc_set_fields", "nlc_set_fields_f32",
            "nlc_get_fields", "nlc_get_populations", "nlc_step",
            "nlc_observables", "nlc_last_error", "nlc_destroy",
            "nlc_lattice_velocities", "nlc_version", "nlc_set_timing",
            "nlc_get_timing", "nlc_timing_name", "nlc_save", "nlc_load",
            "nlc_adjoint", "nlc_observables_static", "nlc_set_chunk",
            "nlc_get_chunk", "nlc_autotune", "nlc_set_wait_budget",
            "nlc_set_persistent"]


def _check(ctx, status):
    if status != NLC_OK:
        msg = load().nlc_last_error(ctx).decode() if ctx else ""
        raise NlcError(status, msg)


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _f32(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != int(np.prod(shape)):
        raise ValueError(f"expected {shape}, got {a.shape}")
    return a


def _f64(a, shape):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != int(np.prod(shape)):
        raise ValueError(f"expected {shape}, got {a.shape}")
    return a


# -- thin wrappers with the C names ------------------------------------------

def nlc_create(grid, params, stream=None):
    lib = load()
    ctx = ctypes.c_void_p()
    st = lib.nlc_create(ctypes.byref(grid), ctypes.byref(params),
                        ctypes.c_void_p(stream or 0), ctypes.byref(ctx))
    _check(None, st)
    return ctx


def nlc_create_batch(grids, params, stream=None):
    lib = load()
    n = len(grids)
    G = (nlc_grid * n)(*grids)
    Pm = (nlc_params * n)(*params)
    ctx = ctypes.c_void_p()
    st = lib.nlc_create_batch(n, ctypes.cast(G, ctypes.c_void_p),
                              ctypes.cast(Pm, ctypes.c_void_p),
                              ctypes.c_void_p(stream or 0), ctypes.byref(ctx))
    _check(None, st)
    return ctx


def nlc_count(ctx):
    return load().nlc_count(ctx)


def nlc_set_params(ctx, inst, params):
    P = params if isinstance(params, nlc_params) else _params(params)
    _check(ctx, load().nlc_set_params(ctx, inst, ctypes.byref(P)))


def nlc_set_mrt(ctx, inst, rates=None):
    """MRT collision with q rates in the library's moment order (nlc.h), or
    BGK again with rates=None."""
    if rates is None:
        _check(ctx, load().nlc_set_mrt(ctx, inst, None, 0))
        return
    r = np.ascontiguousarray(rates, dtype=np.float64)
    _check(ctx, load().nlc_set_mrt(ctx, inst, _ptr(r), int(r.size)))


NLC_STENCIL_STANDARD = 0
NLC_STENCIL_ISOTROPIC = 1


def nlc_set_stencil(ctx, kind):
    _check(ctx, load().nlc_set_stencil(ctx, int(kind)))


def nlc_set_check(ctx, every):
    _check(ctx, load().nlc_set_check(ctx, int(every)))


def nlc_set_wait_budget(ctx, ns):
    _check(ctx, load().nlc_set_wait_budget(ctx, int(ns)))


def nlc_set_persistent(ctx, steps):
    _check(ctx, load().nlc_set_persistent(ctx, int(steps)))


def nlc_set_graph(ctx, steps):
    _check(ctx, load().nlc_set_graph(ctx, int(steps)))


def nlc_set_schedule(ctx, schedule):
    _check(ctx, load().nlc_set_schedule(ctx, schedule))


def nlc_set_chunk(ctx, chunk, taper=False):
    _check(ctx, load().nlc_set_chunk(ctx, int(chunk), 1 if taper else 0))


def nlc_get_chunk(ctx, inst=0):
    """(chunk depth, tapered) of lattice inst."""
    t = ctypes.c_int32(0)
    c = int(load().nlc_get_chunk(ctx, int(inst), ctypes.byref(t)))
    return c, bool(t.value)


def nlc_autotune(ctx, trial_steps):
    out = nlc_tune()
    _check(ctx, load().nlc_autotune(ctx, int(trial_steps), ctypes.byref(out)))
    return out.as_dict()


def nlc_set_fields(ctx, inst, Q5, rho=None, u=None):
    _check(ctx, load().nlc_set_fields(ctx, inst, _ptr(Q5), _ptr(rho), _ptr(u)))


def nlc_set_fields_f32(ctx, inst, Q5):
    """Q5: a float32 numpy array (host), or the integer address of a float32
    device array of the same layout (read in place)."""
    ptr = ctypes.c_void_p(Q5) if isinstance(Q5, int) else _ptr(Q5)
    _check(ctx, load().nlc_set_fields_f32(ctx, inst, ptr))


def nlc_get_fields(ctx, inst, Q5=None, rho=None, u=None):
    _check(ctx, load().nlc_get_fields(ctx, inst, _ptr(Q5), _ptr(rho), _ptr(u)))


def nlc_get_populations(ctx, inst, f):
    _check(ctx, load().nlc_get_populations(ctx, inst, _ptr(f)))


def nlc_step(ctx, n):
    _check(ctx, load().nlc_step(ctx, int(n)))


def nlc_observables(ctx, inst, s_profile=None):
    out = nlc_obs()
    _check(ctx, load().nlc_observables(ctx, inst, ctypes.byref(out),
                                       _ptr(s_profile)))
    return out


def nlc_last_error(ctx):
    return load().nlc_last_error(ctx).decode()


def nlc_destroy(ctx):
    load().nlc_destroy(ctx)


def nlc_lattice_velocities(lattice):
    q = 9 if lattice == NLC_D2Q9 else 19
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    r = load().nlc_lattice_velocities(lattice, _ptr(c), _ptr(w))
    if r != q:
        raise NlcError(-1, "bad lattice")
    return c, w


def nlc_set_timing(ctx, enable):
    _check(ctx, load().nlc_set_timing(ctx, int(bool(enable))))


def nlc_get_timing(ctx):
    """{kernel name: (total ms, launches)} since timing was enabled."""
    ms = np.zeros(16)
    cnt = np.zeros(16, dtype=np.int64)
    n = ctypes.c_int32()
    _check(ctx, load().nlc_get_timing(ctx, 16, _ptr(ms), _ptr(cnt),
                                      ctypes.byref(n)))
    lib = load()
    return {lib.nlc_timing_name(k).decode(): (float(ms[k]), int(cnt[k]))
            for k in range(n.value)}


def nlc_save(ctx):
    """The context's checkpoint as bytes."""
    lib = load()
    n = ctypes.c_size_t(0)
    _check(ctx, lib.nlc_save(ctx, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(ctx, lib.nlc_save(ctx, buf, ctypes.byref(n)))
    return buf.raw[:n.value]


def nlc_load(ctx, data):
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(ctx, load().nlc_load(ctx, buf, len(data)))


def nlc_adjoint(ctx, loss, nsteps, ckpt_every, dQ0=None):
    """Runs nsteps with checkpoints every ckpt_every steps and returns the
    loss and its gradients (dict); fills dQ0 (float64 [5][nz][ny][nx]) if
    given."""
    out = nlc_grad()
    L = nlc_loss(*loss) if not isinstance(loss, nlc_loss) else loss
    _check(ctx, load().nlc_adjoint(ctx, ctypes.cast(ctypes.pointer(L), ctypes.c_void_p),
                                   int(nsteps), int(ckpt_every),
                                   ctypes.cast(ctypes.pointer(out), ctypes.c_void_p),
                                   _ptr(dQ0)))
    return out.as_dict()


def nlc_observables_static(grid, params, f_dev, Q5_dev, stream=None):
    """Observables of a state in caller-owned device memory (f_dev and
    Q5_dev are device addresses of float64 arrays); allocates no device
    memory (see include/nlc.h)."""
    out = nlc_obs()
    P = params if isinstance(params, nlc_params) else _params(params)
    st = load().nlc_observables_static(ctypes.byref(grid), ctypes.byref(P),
                                       ctypes.c_void_p(f_dev), ctypes.c_void_p(Q5_dev),
                                       ctypes.c_void_p(stream or 0), ctypes.byref(out))
    if st != NLC_OK:
        raise NlcError(st, "nlc_observables_static failed")
    return out.as_dict()


def nlc_version():
    return load().nlc_version().decode()


# -- convenience wrappers ----------------------------------------------------

def _params(d):
    return nlc_params(d["A0"], d["K"], d["gamma"], d["Gamma"], d["xi"],
                      d["tau"], d.get("rho0", 1.0))


class Batch:
    """Several lattices (same lattice type and precision) advanced together.

    shapes: list of (nz, ny, nx); params: list of parameter dicts."""

    def __init__(self, lattice, shapes, params, precision=NLC_FP32,
                 stream=None, graph_steps=0, persistent_steps=0):
        self.lattice = lattice
        self.q = 9 if lattice == NLC_D2Q9 else 19
        self.shapes = [tuple(s) for s in shapes]
        grids = [nlc_grid(s[2], s[1], s[0], lattice, precision)
                 for s in self.shapes]
        self.ctx = nlc_create_batch(grids, [_params(p) for p in params],
                                    stream)
        if graph_steps:
            nlc_set_graph(self.ctx, graph_steps)
        if persistent_steps:
            nlc_set_persistent(self.ctx, persistent_steps)

    def __len__(self):
        return len(self.shapes)

    def set_mrt(self, i, rates=None):
        nlc_set_mrt(self.ctx, i, rates)

    def set_stencil(self, kind):
        nlc_set_stencil(self.ctx, kind)

    def set_fields(self, i, Q5, rho=None, u=None):
        sh = self.shapes[i]
        nlc_set_fields(self.ctx, i, _f64(Q5, (5,) + sh), _f64(rho, sh),
                       _f64(u, (3,) + sh))

    def set_fields_f32(self, i, Q5):
        nlc_set_fields_f32(self.ctx, i, _f32(Q5, (5,) + self.shapes[i]))

    def get_fields(self, i):
        sh = self.shapes[i]
        Q5, rho, u = np.empty((5,) + sh), np.empty(sh), np.empty((3,) + sh)
        nlc_get_fields(self.ctx, i, Q5, rho, u)
        return Q5, rho, u

    def get_populations(self, i):
        f = np.empty((self.q,) + self.shapes[i])
        nlc_get_populations(self.ctx, i, f)
        return f

    def step(self, n=1):
        nlc_step(self.ctx, n)

    def set_persistent(self, steps):
        nlc_set_persistent(self.ctx, steps)

    def set_chunk(self, chunk, taper=False):
        nlc_set_chunk(self.ctx, chunk, taper)

    def chunk(self, i=0):
        """(chunk depth, tapered) of lattice i."""
        return nlc_get_chunk(self.ctx, i)

    def autotune(self, trial_steps=10):
        return nlc_autotune(self.ctx, trial_steps)

    def observables(self, i, profile=False):
        prof = np.empty(self.shapes[i][2]) if profile else None
        d = nlc_observables(self.ctx, i, prof).as_dict()
        if profile:
            d["s_profile"] = prof
        return d

    def close(self):
        if self.ctx:
            nlc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """One lattice on the current CUDA device.

    shape is (nz, ny, nx); params a dict with A0, K, gamma, Gamma, xi, tau
    (and optionally rho0).  stream: a cudaStream_t as an int (for example
    torch.cuda.current_stream().cuda_stream), or None.
    """

    def __init__(self, lattice, shape, params, precision=NLC_FP64,
                 stream=None, schedule=NLC_SCHED_FUSED):
        nz, ny, nx = shape
        self.shape = (nz, ny, nx)
        self.lattice = lattice
        self.q = 9 if lattice == NLC_D2Q9 else 19
        g = nlc_grid(nx, ny, nz, lattice, precision)
        p = nlc_params(params["A0"], params["K"], params["gamma"],
                       params["Gamma"], params["xi"], params["tau"],
                       params.get("rho0", 1.0))
        self.ctx = nlc_create(g, p, stream)
        if schedule != NLC_SCHED_FUSED:
            nlc_set_schedule(self.ctx, schedule)

    @property
    def n_cells(self):
        nz, ny, nx = self.shape
        return nx * ny * nz

    def set_fields(self, Q5, rho=None, u=None):
        sh = self.shape
        nlc_set_fields(self.ctx, 0, _f64(Q5, (5,) + sh), _f64(rho, sh),
                       _f64(u, (3,) + sh))

    def set_fields_f32(self, Q5):
        """Q in float32 (a float32 array is passed as is, pinned memory
        included; an integer is the address of a float32 device array), the
        fluid at rest with rho = rho0."""
        if isinstance(Q5, int):
            nlc_set_fields_f32(self.ctx, 0, Q5)
        else:
            nlc_set_fields_f32(self.ctx, 0, _f32(Q5, (5,) + self.shape))

    def get_fields(self):
        sh = self.shape
        Q5 = np.empty((5,) + sh)
        rho = np.empty(sh)
        u = np.empty((3,) + sh)
        nlc_get_fields(self.ctx, 0, Q5, rho, u)
        return Q5, rho, u

    def get_populations(self):
        f = np.empty((self.q,) + self.shape)
        nlc_get_populations(self.ctx, 0, f)
        return f

    def step(self, n=1):
        nlc_step(self.ctx, n)

    def set_chunk(self, chunk, taper=False):
        nlc_set_chunk(self.ctx, chunk, taper)

    def chunk(self):
        """(chunk depth, tapered)."""
        return nlc_get_chunk(self.ctx, 0)

    def autotune(self, trial_steps=10):
        return nlc_autotune(self.ctx, trial_steps)

    def observables(self, profile=False):
        prof = np.empty(self.shape[2]) if profile else None
        d = nlc_observables(self.ctx, 0, prof).as_dict()
        if profile:
            d["s_profile"] = prof
        return d

    def save(self):
        return nlc_save(self.ctx)

    def load_state(self, data):
        nlc_load(self.ctx, data)

    def set_mrt(self, rates=None):
        nlc_set_mrt(self.ctx, 0, rates)

    def set_stencil(self, kind):
        nlc_set_stencil(self.ctx, kind)

    def set_graph(self, steps):
        nlc_set_graph(self.ctx, steps)

    def set_persistent(self, steps):
        nlc_set_persistent(self.ctx, steps)

    def set_params(self, params):
        nlc_set_params(self.ctx, 0, params)

    def set_wait_budget(self, ns):
        nlc_set_wait_budget(self.ctx, ns)

    def adjoint(self, target_radius, w_radius, w_velocity, nsteps, ckpt_every,
                want_dQ0=True):
        dQ0 = np.empty((5,) + self.shape) if want_dQ0 else None
        g = nlc_adjoint(self.ctx, (target_radius, w_radius, w_velocity), nsteps,
                        ckpt_every, dQ0)
        if want_dQ0:
            g["dQ0"] = dQ0
        return g

    def close(self):
        if self.ctx:
            nlc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
