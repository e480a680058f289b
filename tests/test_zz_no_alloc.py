"""nlc_observables_static, the observables entry point that allocates no
device memory (for callers that may not call cudaMalloc: code inside an
application that owns all device memory through its own pool, or
monitoring code that must not trigger an allocation's device-wide
synchronisation).  Its results must equal those of nlc_observables on a
context holding the same state, on two calls in a row (the second call
reuses the library's fixed scratch block left over from the first).

This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_1907_13415_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 parity tolerance of the other GPU tests


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 40, 64)),
                                           (wl.D3Q19, (10, 12, 14))])
def test_static_observables_equal_context_observables(orc, lattice, shape):
    import torch
    from paper_1907_13415_gb300 import nlc
    base = wl.disc_256() if lattice == wl.D2Q9 else wl.sphere_256()
    w = base.with_(lattice=lattice, shape=shape, size=0.3 * min(shape[1:]),
                   noise=1e-4, seed=17)
    stream = torch.cuda.current_stream().cuda_stream
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP64,
                         stream=stream)
    sim.set_fields(w.initial_q5())
    sim.step(25)
    ref = sim.observables()
    f = sim.get_populations()
    Q, _, _ = sim.get_fields()
    sim.close()
    f_d = torch.tensor(f, dtype=torch.float64, device="cuda")
    Q_d = torch.tensor(Q, dtype=torch.float64, device="cuda")
    nz, ny, nx = shape
    grid = nlc.nlc_grid(nx, ny, nz, lattice, nlc.NLC_FP64)
    for _ in range(2):
        got = nlc.nlc_observables_static(grid, w.params, f_d.data_ptr(),
                                         Q_d.data_ptr(), stream)
        for k in ("mass", "s_area", "radius", "free_energy", "u_l2", "max_u"):
            assert got[k] == pytest.approx(ref[k], rel=TOL), k
        for k in ("mom_x", "mom_y", "mom_z"):
            assert abs(got[k] - ref[k]) < TOL * np.prod(shape), k
        assert abs(got["x_iface"] - ref["x_iface"]) < 1e-9
        assert got["nonfinite"] == 0
    # and, independently of the library's other entry point, against the
    # oracle's observables of the same populations and Q
    from helpers import perm_to_oracle
    perm = perm_to_oracle(orc, lattice)
    fo = np.empty_like(f)
    fo[perm] = f
    oo = orc.observables(lattice, wl.param_vector(w.params), fo, Q)
    for k in ("mass", "s_area", "radius", "free_energy", "max_u"):
        assert got[k] == pytest.approx(float(oo[k]), rel=TOL), k
    assert abs(got["x_iface"] - float(oo["x_iface"])) < 1e-9


def test_static_observables_refuse_lattices_beyond_the_scratch():
    import torch
    from paper_1907_13415_gb300 import nlc
    stream = torch.cuda.current_stream().cuda_stream
    f_d = torch.zeros(9, dtype=torch.float64, device="cuda")
    grid = nlc.nlc_grid(nlc.NLC_STATIC_MAX_NX + 1, 1, 1, nlc.NLC_D2Q9, nlc.NLC_FP64)
    with pytest.raises(nlc.NlcError) as ei:
        nlc.nlc_observables_static(grid, wl.BASE_PARAMS, f_d.data_ptr(),
                                   f_d.data_ptr(), stream)
    assert ei.value.status == -1
    grid = nlc.nlc_grid(256, 257, 1, nlc.NLC_D2Q9, nlc.NLC_FP64)  # > max cells
    with pytest.raises(nlc.NlcError):
        nlc.nlc_observables_static(grid, wl.BASE_PARAMS, f_d.data_ptr(),
                                   f_d.data_ptr(), stream)


def test_static_observables_refuse_a_capturing_stream():
    """The call ends with a copy to the host and a stream synchronisation,
    which no stream capture can hold: a capturing stream is refused before
    any work is queued."""
    import torch
    from paper_1907_13415_gb300 import nlc
    f_d = torch.zeros(9 * 64, dtype=torch.float64, device="cuda")
    q_d = torch.zeros(5 * 64, dtype=torch.float64, device="cuda")
    grid = nlc.nlc_grid(8, 8, 1, nlc.NLC_D2Q9, nlc.NLC_FP64)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.graph(g, stream=s):
        q_d.add_(0.0)  # the capture holds one kernel
        status = nlc.load().nlc_observables_static(
            grid, nlc._params(wl.BASE_PARAMS), f_d.data_ptr(), q_d.data_ptr(),
            s.cuda_stream, nlc.nlc_obs())
    assert status == -1
