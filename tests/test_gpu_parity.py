"""Parity of the CUDA step (through the C ABI) with the FP64 CPU oracle.

FP64 builds must agree to 1e-12 normwise relative; FP32 builds to the bound
of helpers.fp32_tolerance.  Sizes span several tiles of the fused kernels
(32 x 8 in x, y; z chunks on D3Q19) with ragged edges, plus lattices smaller
than one tile and single-cell extents.
"""
import numpy as np
import pytest

from paper_1907_13415_gb300 import workloads as wl

from helpers import PARAM_SETS, fp32_tolerance, perm_to_oracle, rel, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12

D2_SHAPES = [(1, 8, 128), (1, 11, 37), (1, 3, 5), (1, 1, 1), (1, 17, 70),
             (1, 24, 64)]
D3_SHAPES = [(3, 3, 3), (5, 7, 9), (20, 10, 40), (1, 9, 33), (37, 9, 35)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_13415_gb300 import nlc
    nlc.load()
    torch.cuda.set_device(0)


def workload(lattice, shape, kind="slab", pset="tau1"):
    base = wl.flat_128x8() if lattice == wl.D2Q9 else wl.sphere_256()
    nz, ny, nx = shape
    p = dict(PARAM_SETS[pset], gamma=base.params["gamma"])
    if kind == "slab":
        w = base.with_(lattice=lattice, shape=shape, geometry="slab",
                       size=max(1, nx // 2), director=(0.3, 0.9, 0.3),
                       noise=1e-3, seed=7, params=p)
    else:
        r = 0.3 * min(s for s in shape if s > 1) if max(shape) > 1 else 1
        w = base.with_(lattice=lattice, shape=shape, geometry="ball", size=r,
                       director=(0.6, 0.0, 0.8), noise=1e-3, seed=8, params=p)
    return w


PSETS = list(PARAM_SETS)


def compare(orc, g, o, lattice, tol):
    perm = perm_to_oracle(orc, lattice)
    assert rel(g["Q"], o["Q"]) < tol
    assert rel(g["f"], o["f"][perm]) < tol
    assert rel(g["rho"], o["rho"]) < tol
    # u is a small difference of O(1) population sums: compare absolutely,
    # on the scale of the populations
    assert np.abs(g["u"] - o["u"]).max() < tol


@pytest.mark.parametrize("pset", PSETS)
@pytest.mark.parametrize("schedule", [0, 1], ids=["fused", "unfused"])
@pytest.mark.parametrize("shape", D2_SHAPES, ids=lambda s: "x".join(map(str, s[::-1])))
def test_d2q9_fp64_matches_oracle(orc, shape, schedule, pset):
    w = workload(wl.D2Q9, shape, pset=pset)
    steps = 60
    g = run_gpu(w, steps, precision=0, schedule=schedule)
    o = run_oracle(orc, w, steps)
    compare(orc, g, o, wl.D2Q9, FP64_TOL)


@pytest.mark.parametrize("pset", PSETS)
@pytest.mark.parametrize("schedule", [0, 1], ids=["fused", "unfused"])
@pytest.mark.parametrize("shape", D3_SHAPES, ids=lambda s: "x".join(map(str, s[::-1])))
def test_d3q19_fp64_matches_oracle(orc, shape, schedule, pset):
    w = workload(wl.D3Q19, shape, kind="ball", pset=pset)
    steps = 12
    g = run_gpu(w, steps, precision=0, schedule=schedule)
    o = run_oracle(orc, w, steps)
    compare(orc, g, o, wl.D3Q19, FP64_TOL)


@pytest.mark.parametrize("pset", PSETS)
@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 24, 64)),
                                           (wl.D2Q9, (1, 11, 37)),
                                           (wl.D3Q19, (20, 10, 40))])
def test_fp32_matches_oracle_within_bound(orc, lattice, shape, pset):
    w = workload(lattice, shape, kind="ball", pset=pset)
    steps = 40
    g = run_gpu(w, steps, precision=1)
    o = run_oracle(orc, w, steps)
    tol = fp32_tolerance(steps)
    perm = perm_to_oracle(orc, lattice)
    assert rel(g["Q"], o["Q"]) < tol
    assert rel(g["f"], o["f"][perm]) < tol


@pytest.mark.parametrize("pset", ["tau1", "paper"])
def test_flat_interface_2000_steps_fp64(orc, pset):
    """The flat-interface workload (128x8 D2Q9, 2000 steps, FP64) in full,
    with its own parameters and with the paper's (Sec. 2)."""
    w = wl.flat_128x8()
    w = w.with_(params=dict(PARAM_SETS[pset], gamma=w.params["gamma"]))
    g = run_gpu(w, w.steps, precision=0)
    o = run_oracle(orc, w, w.steps)
    compare(orc, g, o, wl.D2Q9, FP64_TOL)
    assert abs(g["obs"]["x_iface"] - o["obs"]["x_iface"]) < 1e-9
    assert rel(g["obs"]["s_profile"], o["obs"]["s_profile"]) < FP64_TOL


@pytest.mark.parametrize("pset", ["tau1", "paper"])
@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 40, 50)),
                                           (wl.D3Q19, (9, 10, 12))])
def test_observables_match_oracle(orc, lattice, shape, pset):
    w = workload(lattice, shape, kind="ball", pset=pset)
    g = run_gpu(w, 30, precision=0)
    o = run_oracle(orc, w, 30)
    go, oo = g["obs"], o["obs"]
    for k in ("mass", "s_area", "radius", "free_energy"):
        assert go[k] == pytest.approx(float(oo[k]), rel=1e-12), k
    for k in ("mom_x", "mom_y", "mom_z"):
        assert abs(go[k] - float(oo[k])) < 1e-12 * np.prod(shape), k
    assert go["max_u"] == pytest.approx(float(oo["max_u"]), rel=1e-10)
    assert go["nonfinite"] == 0
    assert go["step"] == 30
    assert rel(go["s_profile"], oo["s_profile"]) < FP64_TOL


def test_initial_flow_and_density(orc):
    """nlc_set_fields with rho and u: populations start at f^eq(rho, u)."""
    w = workload(wl.D3Q19, (6, 5, 7), kind="ball")
    rng = np.random.default_rng(3)
    rho = 1 + 0.01 * rng.normal(size=w.shape)
    u = 0.02 * rng.normal(size=(3,) + w.shape)
    g = run_gpu(w, 0, precision=0, rho=rho, u=u)
    f0 = orc.init_equilibrium(w.lattice, w.shape, rho=rho, u=u)
    perm = perm_to_oracle(orc, w.lattice)
    assert rel(g["f"], f0[perm]) < 1e-15
    g5 = run_gpu(w, 5, precision=0, rho=rho, u=u)
    o5 = run_oracle(orc, w, 5, rho=rho, u=u)
    compare(orc, g5, o5, w.lattice, FP64_TOL)


def test_nonfinite_input_is_rejected():
    import torch
    from paper_1907_13415_gb300 import nlc
    w = workload(wl.D2Q9, (1, 8, 16))
    sim = nlc.Simulation(w.lattice, w.shape, w.params,
                         stream=torch.cuda.current_stream().cuda_stream)
    Q = w.initial_q5()
    Q[2, 0, 3, 4] = np.nan
    with pytest.raises(nlc.NlcError) as ei:
        sim.set_fields(Q)
    assert ei.value.status == -4
    assert "non-finite" in nlc.nlc_last_error(sim.ctx)
    sim.close()


@pytest.mark.parametrize("pset", ["tau1", "paper"])
def test_fused_and_unfused_agree_fp32(pset):
    w = workload(wl.D3Q19, (20, 17, 45), kind="ball", pset=pset)
    a = run_gpu(w, 10, precision=1, schedule=0)
    b = run_gpu(w, 10, precision=1, schedule=1)
    assert rel(a["Q"], b["Q"]) < 1e-6
    assert rel(a["f"], b["f"]) < 1e-6
