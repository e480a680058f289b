"""The experiments module at reduced sizes: FP32 against FP64 drift is
reported and small, and the physics goes the way Sec. 2 says."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_flat_interface_static_and_drift_small():
    from paper_1907_13415_gb300 import experiments as ex
    r = ex.flat(2.7, steps=1500, lx=128, ly=8, every=100)
    assert abs(r["x_iface_fp64"] - 63.5) < 1e-3
    assert r["fp32_vs_fp64"]["max_dQ_rel"] < 1e-3
    assert abs(r["fp32_vs_fp64"]["x_iface_drift_max"]) < 1e-2


@pytest.mark.parametrize("delta,sign", [(-0.03, -1), (0.03, 1)])
def test_disc_grows_above_and_shrinks_below_the_shift(delta, sign):
    """Sec. 2.2: a circular nematic domain shrinks at coexistence and needs a
    positive temperature shift to stand still; well above it grows."""
    from paper_1907_13415_gb300 import experiments as ex
    r = ex.disc(delta, steps=3000, n=64, radius=14, every=250)
    assert r["dRdt_fp64"] * sign > 0
    assert r["fp32_vs_fp64"]["max_dQ_rel"] < 1e-2


def test_flat_interface_with_paper_parameters_follows_eq7():
    """Sec. 2.1 with the paper's parameters (lambda = 2 at gamma = 2.7): the
    relaxed right interface is the tanh of Eq. 7 to within the
    discretisation (lambda is only two cells), it does not move, and the
    flow stays at the rounding level."""
    from paper_1907_13415_gb300 import experiments as ex
    r = ex.flat_paper(2.7, steps=20000, lx=120, ly=4, every=2000)
    assert abs(r["x_iface"] - 89.5) < 1e-3
    assert r["eq7_max_deviation"] < 5e-3
    assert abs(r["velocity"]) < 1e-9
    assert r["max_u"] < 1e-12
    lo = ex.flat_paper(2.69, steps=6000, lx=120, ly=4, every=1000)["velocity"]
    hi = ex.flat_paper(2.71, steps=6000, lx=120, ly=4, every=1000)["velocity"]
    assert lo < 0 < hi


def test_paper_circle_on_single_plane_d3q19_matches_d2q9(tmp_path):
    """The paper runs its circle on D3Q19; on one plane D3Q19 gives the same
    fields as D2Q9 (pinned on the oracle).  The dump holds the vorticity
    field d_x u_y - d_y u_x of the final velocity."""
    import numpy as np
    from paper_1907_13415_gb300 import experiments as ex
    from paper_1907_13415_gb300 import workloads as wl
    a = ex.paper_circle(20.0, steps=400, every=200, lattice=wl.D2Q9,
                        dump=str(tmp_path / "a.npz"))
    b = ex.paper_circle(20.0, steps=400, every=200, lattice=wl.D3Q19,
                        dump=str(tmp_path / "b.npz"))
    A, B = np.load(tmp_path / "a.npz"), np.load(tmp_path / "b.npz")
    assert np.abs(A["Q"] - B["Q"]).max() < 1e-12 * np.abs(A["Q"]).max()
    assert np.abs(A["u"] - B["u"]).max() < 1e-12 * np.abs(A["u"]).max() + 1e-20
    u = A["u"]
    om = (np.roll(u[1], -1, axis=-1) - np.roll(u[1], 1, axis=-1)
          - np.roll(u[0], -1, axis=-2) + np.roll(u[0], 1, axis=-2)) / 2
    assert np.allclose(A["vorticity"], om)
    assert a["max_u_final"] == pytest.approx(b["max_u_final"], rel=1e-9)


def test_free_energy_decreases_during_relaxation():
    """A relaxing droplet loses free energy (Eq. 2, the FP64 observable):
    the flow it drives is damped by viscosity and carries almost no kinetic
    energy, so the free energy never rises between samples."""
    import numpy as np
    from paper_1907_13415_gb300 import nlc
    from paper_1907_13415_gb300 import workloads as wl
    import torch
    w = wl.disc_256(0.0).with_(shape=(1, 48, 48), size=11, noise=2e-3, seed=7)
    s = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP64,
                       stream=torch.cuda.current_stream().cuda_stream)
    s.set_fields(w.initial_q5())
    F = [s.observables()["free_energy"]]
    for _ in range(30):
        s.step(40)
        F.append(s.observables()["free_energy"])
    s.close()
    F = np.array(F)
    assert np.all(np.diff(F) <= 1e-12 * np.abs(F[:-1]))
    assert F[-1] < F[0]
