"""Shared test helpers: run a workload on the GPU library and on the oracle."""
import numpy as np

from paper_1907_13415_gb300 import workloads as wl

EPS32 = np.finfo(np.float32).eps  # 1.19e-7

#: parameter sets of the parity tests.  At tau = 1 the BGK collision keeps
#: nothing of the incoming populations ((1 - 1/tau) f = 0); tau = 0.8 and the
#: paper's own set (Sec. 2: tau = 1.5, K = 0.04, Gamma = 0.34) exercise that
#: part of the collision and of its adjoint.
PARAM_SETS = {
    "tau1": dict(wl.BASE_PARAMS),
    "tau0.8": dict(wl.BASE_PARAMS, tau=0.8),
    "paper": dict(wl.PAPER_PARAMS),
}


def fp32_tolerance(steps):
    """Normwise relative bound for FP32 storage and arithmetic against the
    FP64 oracle after `steps` steps: each step rounds every stored value once
    (relative eps/2) and carries about ten rounded operations into it, and the
    relaxational dynamics do not amplify earlier errors, so the error grows at
    most linearly: 8 eps per step plus a 1e-6 floor for the first steps."""
    return max(1e-6, 8 * EPS32 * steps)


def perm_to_oracle(orc, lattice):
    """Index map from the library's velocity order to the oracle's."""
    from paper_1907_13415_gb300 import nlc
    c_g, w_g = nlc.nlc_lattice_velocities(lattice)
    c_o, w_o = orc.lattice(lattice)
    perm = []
    for cv in c_g:
        j = int(np.where((c_o == cv).all(axis=1))[0][0])
        perm.append(j)
    assert np.allclose(w_o[perm], w_g, rtol=0, atol=1e-16)
    return perm


def rel(a, b):
    """max |a - b| / max |b| (normwise relative difference)."""
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def run_gpu(w, steps, precision, schedule=0, rho=None, u=None, Q0=None):
    import torch
    from paper_1907_13415_gb300 import nlc
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=precision,
                         stream=torch.cuda.current_stream().cuda_stream,
                         schedule=schedule)
    sim.set_fields(w.initial_q5() if Q0 is None else Q0, rho, u)
    sim.step(steps)
    Q, r, uu = sim.get_fields()
    f = sim.get_populations()
    obs = sim.observables(profile=True)
    sim.close()
    return dict(Q=Q, rho=r, u=uu, f=f, obs=obs)


def run_oracle(orc, w, steps, rho=None, u=None, Q0=None):
    p = wl.param_vector(w.params)
    f0 = orc.init_equilibrium(w.lattice, w.shape, rho=rho, u=u)
    f, Q = orc.step(w.lattice, p, f0, w.initial_q5() if Q0 is None else Q0,
                    steps)
    fl = orc.fields(w.lattice, p, f, Q)
    obs = orc.observables(w.lattice, p, f, Q)
    return dict(Q=Q, rho=fl["rho"], u=fl["u"], f=f, obs=obs)
