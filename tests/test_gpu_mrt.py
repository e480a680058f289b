"""The MRT collision (nlc_set_mrt) against the oracle's, in both schedules,
and its boundaries: equal rates give the BGK step, the adjoint refuses it,
bad rates are rejected."""
import numpy as np
import pytest

from helpers import PARAM_SETS, perm_to_oracle, rel
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


def rates_for(lattice, seed):
    q = 9 if lattice == wl.D2Q9 else 19
    return np.random.default_rng(seed).uniform(0.7, 1.8, size=q)


def droplet(lattice, shape, pset="tau1"):
    base = wl.flat_128x8() if lattice == wl.D2Q9 else wl.sphere_256()
    return base.with_(lattice=lattice, shape=shape, geometry="ball",
                      size=0.3 * min(s for s in shape if s > 1), noise=1e-3, seed=21,
                      director=(0.6, 0.8, 0.0),
                      params=dict(PARAM_SETS[pset], gamma=base.params["gamma"]))


def run_gpu(w, steps, precision, schedule, rates):
    from paper_1907_13415_gb300 import nlc
    s = nlc.Simulation(w.lattice, w.shape, w.params, precision=precision, stream=stream())
    nlc.nlc_set_schedule(s.ctx, schedule)
    if rates is not None:
        s.set_mrt(rates)
    s.set_fields(w.initial_q5())
    s.step(steps)
    f = s.get_populations()
    Q, _, _ = s.get_fields()
    s.close()
    return f, Q


@pytest.mark.parametrize("pset", ["tau1", "paper"])
@pytest.mark.parametrize("schedule", [0, 1], ids=["fused", "unfused"])
@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 19, 43)),
                                           (wl.D3Q19, (9, 10, 37))])
def test_mrt_fp64_matches_oracle(orc, lattice, shape, schedule, pset):
    w = droplet(lattice, shape, pset)
    r = rates_for(lattice, 3)
    steps = 40
    f, Q = run_gpu(w, steps, 0, schedule, r)
    orc.set_mrt(lattice, r)
    try:
        f0 = orc.init_equilibrium(lattice, shape)
        fo, Qo = orc.step(lattice, wl.param_vector(w.params), f0, w.initial_q5(), steps)
    finally:
        orc.set_mrt(lattice, None)
    perm = perm_to_oracle(orc, lattice)
    assert rel(Q, Qo) < 1e-12
    assert rel(f, fo[perm]) < 1e-12


@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 24, 64)),
                                           (wl.D3Q19, (8, 12, 40))])
def test_mrt_fp32_within_bound(orc, lattice, shape):
    from helpers import fp32_tolerance
    w = droplet(lattice, shape)
    r = rates_for(lattice, 4)
    steps = 60
    _, Q = run_gpu(w, steps, 1, 0, r)
    orc.set_mrt(lattice, r)
    try:
        f0 = orc.init_equilibrium(lattice, shape)
        _, Qo = orc.step(lattice, wl.param_vector(w.params), f0, w.initial_q5(), steps)
    finally:
        orc.set_mrt(lattice, None)
    assert rel(Q, Qo) < fp32_tolerance(steps)


@pytest.mark.parametrize("pset", ["tau1", "tau0.8", "paper"])
def test_equal_rates_reproduce_bgk_and_reset(pset):
    # at tau = 1 the rates 1/tau relax every moment fully; tau = 0.8 and the
    # paper's 1.5 keep part of the incoming populations
    w = droplet(wl.D3Q19, (6, 9, 33), pset)
    tau = w.params["tau"]
    f_b, Q_b = run_gpu(w, 25, 0, 0, None)
    f_m, Q_m = run_gpu(w, 25, 0, 0, np.full(19, 1.0 / tau))
    assert rel(Q_m, Q_b) < 1e-13 and rel(f_m, f_b) < 1e-13
    # back to BGK: bitwise the BGK run
    from paper_1907_13415_gb300 import nlc
    s = nlc.Simulation(w.lattice, w.shape, w.params, precision=0, stream=stream())
    s.set_mrt(np.full(19, 1.3))
    s.set_mrt(None)
    s.set_fields(w.initial_q5())
    s.step(25)
    assert np.array_equal(s.get_populations(), f_b)
    s.close()


def test_rates_checked_and_adjoint_refused():
    from paper_1907_13415_gb300 import nlc
    w = droplet(wl.D2Q9, (1, 16, 16))
    s = nlc.Simulation(w.lattice, w.shape, w.params, precision=0, stream=stream())
    for bad in (np.full(8, 1.0), np.r_[np.full(8, 1.0), 2.0], np.r_[np.full(8, 1.0), 0.0]):
        with pytest.raises(nlc.NlcError) as ei:
            s.set_mrt(bad)
        assert ei.value.status == -1
    s.set_mrt(np.full(9, 1.2))
    s.set_fields(w.initial_q5())
    with pytest.raises(nlc.NlcError) as ei:
        s.adjoint(4.0, 1.0, 1.0, nsteps=4, ckpt_every=2)
    assert ei.value.status == -7
    s.close()
