"""NLC_FP32_QF64: populations stored in float, Q, u and all arithmetic in
double.  Against the FP64 oracle it sits within the FP32 bound, and its Q is
much closer to the oracle's than the all-FP32 run's (the FP32 rounding is
confined to the stored populations); checkpoints round-trip exactly; the
adjoint refuses it."""
import numpy as np
import pytest

from helpers import PARAM_SETS, fp32_tolerance, perm_to_oracle, rel
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
    base = wl.flat_128x8() if lattice == wl.D2Q9 else wl.sphere_256()
    return base.with_(lattice=lattice, shape=shape, geometry="ball",
                      size=0.3 * min(s for s in shape if s > 1), noise=1e-3, seed=29,
                      director=(0.6, 0.8, 0.0),
                      params=dict(PARAM_SETS[pset], gamma=base.params["gamma"]))


def run(w, steps, precision, schedule=0):
    from paper_1907_13415_gb300 import nlc
    s = nlc.Simulation(w.lattice, w.shape, w.params, precision=precision, stream=stream())
    nlc.nlc_set_schedule(s.ctx, schedule)
    s.set_fields(w.initial_q5())
    s.step(steps)
    f = s.get_populations()
    Q, _, _ = s.get_fields()
    s.close()
    return f, Q


@pytest.mark.parametrize("pset", ["tau1", "paper"])
@pytest.mark.parametrize("schedule", [0, 1], ids=["fused", "unfused"])
@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 24, 64)), (wl.D3Q19, (8, 12, 40))])
def test_mixed_precision_against_oracle(orc, lattice, shape, schedule, pset):
    from paper_1907_13415_gb300 import nlc
    w = droplet(lattice, shape, pset)
    steps = 60
    f0 = orc.init_equilibrium(lattice, shape)
    fo, Qo = orc.step(lattice, wl.param_vector(w.params), f0, w.initial_q5(), steps)
    fm, Qm = run(w, steps, nlc.NLC_FP32_QF64, schedule)
    _, Q32 = run(w, steps, nlc.NLC_FP32, schedule)
    em, e32 = rel(Qm, Qo), rel(Q32, Qo)
    assert em < fp32_tolerance(steps)
    assert em < 0.1 * e32, (em, e32)
    assert rel(fm, fo[perm_to_oracle(orc, lattice)]) < fp32_tolerance(steps)


def test_mixed_checkpoint_round_trip_and_adjoint_refused():
    from paper_1907_13415_gb300 import nlc
    w = droplet(wl.D3Q19, (6, 8, 20))
    a = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32_QF64,
                       stream=stream())
    a.set_fields(w.initial_q5())
    a.step(5)
    blob = a.save()
    # float populations and double Q: (19 * 4 + 5 * 8) bytes per cell of payload
    assert len(blob) >= (19 * 4 + 5 * 8) * np.prod(w.shape)
    a.step(7)
    b = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32_QF64,
                       stream=stream())
    b.load_state(blob)
    b.step(7)
    assert np.array_equal(a.get_populations(), b.get_populations())
    assert np.array_equal(a.get_fields()[0], b.get_fields()[0])
    with pytest.raises(nlc.NlcError) as ei:
        a.adjoint(4.0, 1.0, 1.0, nsteps=4, ckpt_every=2)
    assert ei.value.status == -7
    a.close()
    b.close()
