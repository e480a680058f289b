"""The observables computed by the fused lb kernel in its observing form
(the default with the standard stencils and 32-bit population offsets)
against the one-cell-per-thread kernels (stress, then rho, u and the
observables), which NLC_POP_INDEX64=1 selects: the same sums up to the
order of summation and the reciprocal of rho, on ragged lattices whose
tiles and z-chunks end part-way, single lattices and a batch."""
import numpy as np
import pytest

from paper_1907_13415_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

KEYS_REL = ("mass", "s_area", "free_energy", "radius", "u_l2", "max_u")
KEYS_ABS = ("mom_x", "mom_y", "mom_z")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def cases():
    sphere = wl.sphere_256().with_(shape=(21, 19, 45), size=6.0, noise=1e-3, seed=51)
    disc = wl.disc_256().with_(shape=(1, 61, 70), size=14.0, noise=1e-3, seed=53)
    return {"D3Q19": sphere, "D2Q9": disc}


def observe(w, precision, wide, steps, monkeypatch):
    from paper_1907_13415_gb300 import nlc
    monkeypatch.setenv("NLC_POP_INDEX64", "1" if wide else "0")
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=precision,
                         stream=stream())
    sim.set_fields(w.initial_q5())
    sim.step(steps)
    o = sim.observables(profile=True)
    sim.close()
    return o


def compare(a, b, rel, mass):
    for k in KEYS_REL:
        assert a[k] == pytest.approx(b[k], rel=rel, abs=1e-300), k
    for k in KEYS_ABS:
        assert abs(a[k] - b[k]) < rel * mass, k
    assert a["nonfinite"] == b["nonfinite"] == 0
    assert a["x_iface"] == b["x_iface"]
    assert np.array_equal(a["s_profile"], b["s_profile"])


@pytest.mark.parametrize("lattice", ["D3Q19", "D2Q9"])
@pytest.mark.parametrize("precision,rel", [("NLC_FP32", 2e-6), ("NLC_FP64", 1e-12),
                                           ("NLC_FP32_QF64", 1e-12)])
@pytest.mark.parametrize("steps", [0, 5])
def test_fused_observables_match_per_cell_kernels(lattice, precision, rel, steps,
                                                  monkeypatch):
    from paper_1907_13415_gb300 import nlc
    w = cases()[lattice]
    prec = getattr(nlc, precision)
    fused = observe(w, prec, False, steps, monkeypatch)
    ref = observe(w, prec, True, steps, monkeypatch)
    compare(fused, ref, rel, ref["mass"])


def test_fused_observables_of_each_lattice_in_a_batch(monkeypatch):
    """Every lattice of a batch observed on its own tiles, against the same
    lattice stepped alone through the per-cell kernels."""
    from paper_1907_13415_gb300 import nlc
    base = wl.sphere_256()
    ws = [base.with_(shape=s, size=0.3 * min(s), noise=1e-3, seed=60 + k)
          for k, s in enumerate([(18, 17, 40), (9, 30, 33), (24, 8, 64)])]
    monkeypatch.setenv("NLC_POP_INDEX64", "0")
    b = nlc.Batch(wl.D3Q19, [w.shape for w in ws], [w.params for w in ws],
                  precision=nlc.NLC_FP32, stream=stream())
    for i, w in enumerate(ws):
        b.set_fields(i, w.initial_q5())
    b.step(4)
    got = [b.observables(i, profile=True) for i in range(len(ws))]
    b.close()
    for w, g in zip(ws, got):
        ref = observe(w, nlc.NLC_FP32, True, 4, monkeypatch)
        compare(g, ref, 2e-6, ref["mass"])
