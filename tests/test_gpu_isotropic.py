"""The isotropic stencils (nlc_set_stencil) against the oracle's, in both
schedules, alone and with the MRT collision; the adjoint refuses them."""
import numpy as np
import pytest

from helpers import fp32_tolerance, perm_to_oracle, rel
from paper_1907_13415_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def droplet(lattice, shape, pset="tau1"):
    from helpers import PARAM_SETS
    base = wl.flat_128x8() if lattice == wl.D2Q9 else wl.sphere_256()
    return base.with_(lattice=lattice, shape=shape, geometry="ball",
                      size=0.3 * min(s for s in shape if s > 1), noise=1e-3, seed=23,
                      director=(0.6, 0.8, 0.0),
                      params=dict(PARAM_SETS[pset], gamma=base.params["gamma"]))


def run_gpu(w, steps, precision, schedule, rates=None):
    from paper_1907_13415_gb300 import nlc
    s = nlc.Simulation(w.lattice, w.shape, w.params, precision=precision, stream=stream())
    nlc.nlc_set_schedule(s.ctx, schedule)
    s.set_stencil(nlc.NLC_STENCIL_ISOTROPIC)
    if rates is not None:
        s.set_mrt(rates)
    s.set_fields(w.initial_q5())
    s.step(steps)
    f = s.get_populations()
    Q, _, u = s.get_fields()
    o = s.observables()
    s.close()
    return f, Q, u, o


def run_oracle(orc, w, steps, rates=None):
    orc.set_stencil(1)
    if rates is not None:
        orc.set_mrt(w.lattice, rates)
    try:
        f0 = orc.init_equilibrium(w.lattice, w.shape)
        p = wl.param_vector(w.params)
        f, Q = orc.step(w.lattice, p, f0, w.initial_q5(), steps)
        u = orc.fields(w.lattice, p, f, Q)["u"]
    finally:
        orc.set_stencil(0)
        orc.set_mrt(w.lattice, None)
    return f, Q, u


@pytest.mark.parametrize("pset", ["tau1", "paper"])
@pytest.mark.parametrize("schedule", [0, 1], ids=["fused", "unfused"])
@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 19, 43)), (wl.D2Q9, (1, 3, 5)),
                                           (wl.D3Q19, (9, 10, 37)), (wl.D3Q19, (3, 3, 3))])
def test_isotropic_fp64_matches_oracle(orc, lattice, shape, schedule, pset):
    w = droplet(lattice, shape, pset)
    f, Q, u, _ = run_gpu(w, 40, 0, schedule)
    fo, Qo, uo = run_oracle(orc, w, 40)
    perm = perm_to_oracle(orc, lattice)
    assert rel(Q, Qo) < 1e-12
    assert rel(f, fo[perm]) < 1e-12
    d = 2 if lattice == wl.D2Q9 else 3
    assert rel(u[:d], uo[:d]) < 1e-10


@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 24, 64)), (wl.D3Q19, (8, 12, 40))])
def test_isotropic_with_mrt_fp64_and_fp32(orc, lattice, shape):
    w = droplet(lattice, shape)
    q = 9 if lattice == wl.D2Q9 else 19
    r = np.random.default_rng(5).uniform(0.7, 1.8, size=q)
    f, Q, _, _ = run_gpu(w, 30, 0, 0, r)
    fo, Qo, _ = run_oracle(orc, w, 30, r)
    assert rel(Q, Qo) < 1e-12
    assert rel(f, fo[perm_to_oracle(orc, lattice)]) < 1e-12
    _, Q32, _, _ = run_gpu(w, 30, 1, 0, r)
    assert rel(Q32, Qo) < fp32_tolerance(30)


def test_adjoint_refuses_isotropic_stencils():
    from paper_1907_13415_gb300 import nlc
    w = droplet(wl.D2Q9, (1, 16, 16))
    s = nlc.Simulation(w.lattice, w.shape, w.params, precision=0, stream=stream())
    s.set_stencil(nlc.NLC_STENCIL_ISOTROPIC)
    s.set_fields(w.initial_q5())
    with pytest.raises(nlc.NlcError) as ei:
        s.adjoint(4.0, 1.0, 1.0, nsteps=4, ckpt_every=2)
    assert ei.value.status == -7
    with pytest.raises(nlc.NlcError):
        s.set_stencil(2)
    s.close()
