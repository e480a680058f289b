"""The step kernels are launched with programmatic dependent launch: each may
be scheduled while the kernel before it in the stream is finishing and waits
on the device for it before touching memory.  Whatever precedes a step on
the stream (the library's own kernels, a caller's kernels, a host
synchronisation, a graph replay), the state after n steps is the same bit
for bit."""
import numpy as np
import pytest

from paper_1907_13415_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def workload(lattice, shape):
    base = wl.disc_256(0.005) if lattice == wl.D2Q9 else wl.sphere_256()
    return base.with_(shape=shape, size=min(s for s in shape if s > 1) / 4)


def run(w, steps, mode):
    """steps steps of w in FP32: 'sync' synchronises the host after every
    step, 'caller' puts a caller's kernels on the stream between steps,
    'graph' replays graphs of 10 steps."""
    import torch
    from paper_1907_13415_gb300 import nlc
    stream = torch.cuda.current_stream()
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32,
                         stream=stream.cuda_stream)
    sim.set_graph(10 if mode == "graph" else 0)
    sim.set_fields(w.initial_q5())
    scratch = torch.ones(1 << 24, device="cuda")
    if mode == "graph":
        sim.step(steps)
    else:
        for _ in range(steps):
            sim.step(1)
            if mode == "sync":
                torch.cuda.synchronize()
            else:
                scratch.mul_(1.0000001).add_(1e-7)
    Q, rho, u = sim.get_fields()
    f = sim.get_populations()
    sim.close()
    return Q, rho, u, f


# one-wave grids (the next kernel is released at once) and a multi-wave grid
@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 128, 128)),
                                           (wl.D3Q19, (32, 32, 32)),
                                           (wl.D3Q19, (64, 256, 256))])
def test_state_does_not_depend_on_what_precedes_a_step(lattice, shape):
    w = workload(lattice, shape)
    ref = run(w, 30, "sync")
    for mode in ("caller", "graph"):
        got = run(w, 30, mode)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), mode
