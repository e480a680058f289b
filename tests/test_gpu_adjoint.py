"""The hand-written adjoint (nlc_adjoint) against derivatives of the oracle.

The oracle's complex-step twin gives the exact (to rounding) derivative of
the droplet loss L = w_R (R - R_target)^2 + w_u |u|_2 after T steps with
respect to gamma, K, Gamma and any direction of the initial Q field.  The
FP64 adjoint must agree to 1e-8 relative; the FP32 adjoint to 1e-4 (the
loss gradient is accumulated over T steps in single precision; measured
errors are below 2e-6 here).  FP64 central finite differences of the GPU forward run
(h = 1e-6) are checked as well.
"""
import numpy as np
import pytest

from paper_1907_13415_gb300 import workloads as wl

from helpers import PARAM_SETS

pytestmark = pytest.mark.gpu

LOSS = (7.5, 1.0, 50.0)  # target radius, w_radius, w_velocity


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
    base = wl.adjoint_disc_128() if lattice == wl.D2Q9 else wl.sphere_256()
    r = 0.25 * min(s for s in shape if s > 1)
    p = dict(PARAM_SETS[pset], gamma=2.70)
    return base.with_(shape=shape, size=r, noise=1e-4, seed=41, params=p,
                      director=(0.8, 0.6, 0.0))


def oracle_loss_derivative(orc_cs, w, steps, dparam=None, dQ=None, h=1e-30):
    """Im L(x + i h v) / h for a parameter index or a Q0 direction."""
    p = wl.param_vector(w.params).astype(np.complex128)
    Q0 = w.initial_q5().astype(np.complex128)
    if dparam is not None:
        p[dparam] += 1j * h
    if dQ is not None:
        Q0 = Q0 + 1j * h * dQ
    f0 = orc_cs.init_equilibrium(w.lattice, w.shape)
    f, Q = orc_cs.step(w.lattice, p, f0, Q0, steps)
    R = orc_cs.observables(w.lattice, p, f, Q)["radius"]
    u = orc_cs.fields(w.lattice, p, f, Q)["u"]
    L = LOSS[1] * (R - LOSS[0]) ** 2 + LOSS[2] * np.sqrt(np.sum(u * u))
    return L.real, L.imag / h


def gpu_adjoint(w, steps, ckpt, precision):
    from paper_1907_13415_gb300 import nlc
    s = nlc.Simulation(w.lattice, w.shape, w.params, precision=precision,
                       stream=stream())
    s.set_fields(w.initial_q5())
    g = s.adjoint(*LOSS, nsteps=steps, ckpt_every=ckpt)
    obs = s.observables()
    s.close()
    return g, obs


@pytest.mark.parametrize("pset", ["tau1", "tau0.8", "paper"])
@pytest.mark.parametrize("lattice,shape,steps,ckpt",
                         [(wl.D2Q9, (1, 32, 32), 60, 16),
                          (wl.D3Q19, (10, 12, 14), 20, 7)])
def test_fp64_adjoint_matches_complex_step_oracle(orc_cs, lattice, shape, steps, ckpt, pset):
    w = droplet(lattice, shape, pset)
    g, obs = gpu_adjoint(w, steps, ckpt, precision=0)
    L, dg = oracle_loss_derivative(orc_cs, w, steps, dparam=2)
    assert g["loss"] == pytest.approx(L, rel=1e-10)
    assert obs["step"] == steps
    assert g["dgamma"] == pytest.approx(dg, rel=1e-8)
    _, dK = oracle_loss_derivative(orc_cs, w, steps, dparam=1)
    assert g["dK"] == pytest.approx(dK, rel=1e-8)
    _, dG = oracle_loss_derivative(orc_cs, w, steps, dparam=3)
    assert g["dGamma"] == pytest.approx(dG, rel=1e-8)
    rng = np.random.default_rng(5)
    for _ in range(3):
        v = rng.normal(size=(5,) + w.shape)
        _, dv = oracle_loss_derivative(orc_cs, w, steps, dQ=v)
        assert np.sum(g["dQ0"] * v) == pytest.approx(dv, rel=1e-8)


@pytest.mark.parametrize("pset", ["tau1", "paper"])
def test_fp32_adjoint_matches_oracle_within_bound(orc_cs, pset):
    w = droplet(wl.D2Q9, (1, 32, 32), pset)
    g, _ = gpu_adjoint(w, 60, 16, precision=1)
    for idx, key in ((2, "dgamma"), (1, "dK"), (3, "dGamma")):
        _, d = oracle_loss_derivative(orc_cs, w, 60, dparam=idx)
        assert g[key] == pytest.approx(d, rel=1e-4), key
    v = np.random.default_rng(6).normal(size=(5,) + w.shape)
    _, dv = oracle_loss_derivative(orc_cs, w, 60, dQ=v)
    assert np.sum(g["dQ0"] * v) == pytest.approx(dv, rel=1e-4)


def test_fp64_adjoint_matches_central_differences():
    """dL/dgamma against (L(gamma + h) - L(gamma - h)) / 2h of the GPU's own
    FP64 forward run, h = 1e-6."""
    from paper_1907_13415_gb300 import nlc
    w = droplet(wl.D2Q9, (1, 24, 24))
    g, _ = gpu_adjoint(w, 40, 10, precision=0)
    h = 1e-6
    Ls = []
    for sgn in (1, -1):
        p = dict(w.params, gamma=w.params["gamma"] + sgn * h)
        s = nlc.Simulation(w.lattice, w.shape, p, precision=0, stream=stream())
        s.set_fields(w.initial_q5())
        s.step(40)
        o = s.observables()
        Ls.append(LOSS[1] * (o["radius"] - LOSS[0]) ** 2 + LOSS[2] * o["u_l2"])
        s.close()
    fd = (Ls[0] - Ls[1]) / (2 * h)
    assert g["dgamma"] == pytest.approx(fd, rel=1e-5)


def test_adjoint_leaves_final_state_and_rejects_batches():
    from paper_1907_13415_gb300 import nlc
    w = droplet(wl.D2Q9, (1, 16, 20))
    a = nlc.Simulation(w.lattice, w.shape, w.params, precision=0, stream=stream())
    a.set_fields(w.initial_q5())
    a.adjoint(*LOSS, nsteps=13, ckpt_every=5, want_dQ0=False)
    b = nlc.Simulation(w.lattice, w.shape, w.params, precision=0, stream=stream())
    b.set_fields(w.initial_q5())
    b.step(13)
    assert np.array_equal(a.get_populations(), b.get_populations())
    assert np.array_equal(a.get_fields()[0], b.get_fields()[0])
    a.close()
    b.close()
    bt = nlc.Batch(wl.D2Q9, [w.shape, w.shape], [w.params, w.params], stream=stream())
    with pytest.raises(nlc.NlcError):
        nlc.nlc_adjoint(bt.ctx, LOSS, 5, 5)
    bt.close()


def test_torch_autograd_function(orc_cs):
    """loss.backward() through the autograd bridge gives the adjoint's
    gradients, which match the oracle's complex-step derivative."""
    import torch
    from paper_1907_13415_gb300 import nlc
    from paper_1907_13415_gb300.autograd import droplet_loss
    w = droplet(wl.D2Q9, (1, 24, 26))
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=0, stream=stream())
    Q0 = torch.tensor(w.initial_q5(), dtype=torch.float64, requires_grad=True)
    theta = torch.tensor([w.params["gamma"], w.params["K"], w.params["Gamma"]],
                         dtype=torch.float64, requires_grad=True)
    L = droplet_loss(Q0, theta, sim, w.params, 30, 8, *LOSS)
    L.backward()
    _, dg = oracle_loss_derivative(orc_cs, w, 30, dparam=2)
    _, dK = oracle_loss_derivative(orc_cs, w, 30, dparam=1)
    assert theta.grad[0].item() == pytest.approx(dg, rel=1e-8)
    assert theta.grad[1].item() == pytest.approx(dK, rel=1e-8)
    v = np.random.default_rng(9).normal(size=Q0.shape)
    _, dv = oracle_loss_derivative(orc_cs, w, 30, dQ=v)
    assert float((Q0.grad.numpy() * v).sum()) == pytest.approx(dv, rel=1e-8)
    # a second evaluation at shifted gamma through set_params
    theta2 = torch.tensor([w.params["gamma"] + 0.01, w.params["K"], w.params["Gamma"]],
                          dtype=torch.float64, requires_grad=True)
    L2 = droplet_loss(Q0.detach(), theta2, sim, w.params, 30, 8, *LOSS)
    w2 = w.with_(params=dict(w.params, gamma=w.params["gamma"] + 0.01))
    L2_ref, _ = oracle_loss_derivative(orc_cs, w2, 30, dparam=2)
    assert L2.item() == pytest.approx(L2_ref, rel=1e-10)
    sim.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(1, 40, 36), (1, 128, 128), (1, 3, 7)])
def test_tiled_reverse_equals_cell_reverse(monkeypatch, precision, shape):
    """On single-plane lattices the reverse sweep runs as owned tiles with
    recomputed halos (one grid barrier per reverse step); it forms every
    state adjoint with the same functions as the one-cell-per-thread
    segment kernel (NLC_ADJ_TILED=0), so dL/dQ0 and the parameter adjoints
    agree to rounding (the compiler may fuse multiply-adds differently in
    the two kernels, and the parameter adjoints are summed in another
    grouping).  40 x 36 leaves partial tiles on both axes; on 7 x 3 one
    tile's box wraps around the lattice several times."""
    w = droplet(wl.D2Q9, shape, "paper")
    g_tiled, _ = gpu_adjoint(w, 30, 8, precision)
    monkeypatch.setenv("NLC_ADJ_TILED", "0")
    g_cell, _ = gpu_adjoint(w, 30, 8, precision)
    tol = 1e-12 if precision == 0 else 1e-5
    dq = np.abs(g_tiled["dQ0"] - g_cell["dQ0"]).max() / np.abs(g_cell["dQ0"]).max()
    assert dq < tol
    assert g_tiled["loss"] == g_cell["loss"]
    for k in ("dgamma", "dK", "dGamma"):
        assert g_tiled[k] == pytest.approx(g_cell[k], rel=tol), k


def test_adjoint_with_persistent_forward_sweep():
    """With the persistent form of the step switched on, the adjoint's forward
    sweep (graphs of the checkpoint segments) runs the cooperative kernel;
    the gradients equal those of the two-kernel form to rounding."""
    from paper_1907_13415_gb300 import nlc
    w = droplet(wl.D2Q9, (1, 24, 32))
    out = []
    for k in (0, 7):
        s = nlc.Simulation(w.lattice, w.shape, w.params, precision=0, stream=stream())
        s.set_persistent(k)
        s.set_fields(w.initial_q5())
        out.append(s.adjoint(*LOSS, nsteps=30, ckpt_every=10))
        s.close()
    for key in ("loss", "dgamma", "dK", "dGamma"):
        assert out[1][key] == pytest.approx(out[0][key], rel=1e-12), key
    assert np.abs(out[1]["dQ0"] - out[0]["dQ0"]).max() <= 1e-12 * np.abs(out[0]["dQ0"]).max()
