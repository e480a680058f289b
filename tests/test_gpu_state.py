"""Checkpoints (nlc_save / nlc_load) and the device-side error paths."""
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


def make(w, precision):
    import torch
    from paper_1907_13415_gb300 import nlc
    return nlc.Simulation(w.lattice, w.shape, w.params, precision=precision,
                          stream=torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("lattice,shape", [(wl.D2Q9, (1, 20, 45)),
                                           (wl.D3Q19, (10, 12, 34))])
def test_resume_is_bitwise_identical(lattice, shape, precision):
    base = wl.flat_128x8() if lattice == wl.D2Q9 else wl.sphere_256()
    w = base.with_(lattice=lattice, shape=shape, geometry="ball",
                   size=0.3 * min(shape[1:]), noise=1e-3)
    a = make(w, precision)
    a.set_fields(w.initial_q5())
    a.step(7)
    blob = a.save()
    a.step(9)
    fa = a.get_populations()
    Qa, _, _ = a.get_fields()
    b = make(w, precision)
    b.load_state(blob)
    b.step(9)
    fb = b.get_populations()
    Qb, _, _ = b.get_fields()
    assert np.array_equal(fa, fb) and np.array_equal(Qa, Qb)
    assert b.observables()["step"] == 16
    a.close()
    b.close()


def test_corrupt_or_mismatched_checkpoint_is_rejected():
    from paper_1907_13415_gb300 import nlc
    w = wl.flat_128x8().with_(shape=(1, 8, 40), size=20)
    a = make(w, 0)
    a.set_fields(w.initial_q5())
    a.step(3)
    blob = bytearray(a.save())
    Q0, _, _ = a.get_fields()
    bad = bytearray(blob)
    bad[-5] ^= 0x40
    with pytest.raises(nlc.NlcError) as ei:
        a.load_state(bytes(bad))
    assert ei.value.status == -6
    Q1, _, _ = a.get_fields()
    assert np.array_equal(Q0, Q1)  # state untouched
    other = make(w.with_(shape=(1, 8, 41)), 0)
    with pytest.raises(nlc.NlcError) as ei:
        other.load_state(bytes(blob))
    assert ei.value.status == -1
    with pytest.raises(nlc.NlcError) as ei:
        a.load_state(bytes(blob[:100]))
    assert ei.value.status == -1
    a.close()
    other.close()


def test_periodic_check_reports_a_blow_up():
    """Failure detection on the host side of a GPU run: a finite but absurd
    initial Q (|Q| = 50) overflows within a few steps; with nlc_set_check the
    step call stops with NLC_EUNSTABLE and names the step, and without the
    check the observables count the non-finite values."""
    from paper_1907_13415_gb300 import nlc
    w = wl.flat_128x8().with_(shape=(1, 8, 32), size=16)
    Q = w.initial_q5() * 150.0
    s = make(w, 1)
    s.set_fields(Q)
    nlc.nlc_set_check(s.ctx, 2)
    with pytest.raises(nlc.NlcError) as ei:
        s.step(40)
    assert ei.value.status == -4
    assert "non-finite" in nlc.nlc_last_error(s.ctx)
    s.close()
    s = make(w, 1)
    s.set_fields(Q)
    s.step(40)
    assert s.observables()["nonfinite"] > 0
    s.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_pinned_host_inputs_are_read_in_place(precision):
    """nlc_set_fields reads page-locked host arrays directly from the kernel
    instead of staging them; the state must equal the one set from ordinary
    (pageable) arrays, also with rho and u given and a non-finite value
    still refused."""
    import torch
    from paper_1907_13415_gb300 import nlc
    w = wl.sphere_256().with_(shape=(9, 12, 34), size=4.0, noise=1e-3, seed=51)
    rng = np.random.default_rng(52)
    Q = w.initial_q5()
    rho = 1.0 + 0.01 * rng.standard_normal(w.shape)
    u = 1e-3 * rng.standard_normal((3,) + w.shape)

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        return t

    pQ, prho, pu = pinned(Q), pinned(rho), pinned(u)
    a, b = make(w, precision), make(w, precision)
    a.set_fields(Q, rho, u)
    b.set_fields(pQ.numpy(), prho.numpy(), pu.numpy())
    for x, y in zip(a.get_fields(), b.get_fields()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.get_populations(), b.get_populations())
    a.step(3)
    b.step(3)
    assert np.array_equal(a.get_populations(), b.get_populations())
    b.set_fields(pQ.numpy())            # Q only: rho0 and rest
    a.set_fields(Q)
    assert np.array_equal(a.get_populations(), b.get_populations())
    pQ.numpy()[2, 1, 1, 1] = np.nan
    with pytest.raises(nlc.NlcError) as ei:
        b.set_fields(pQ.numpy())
    assert ei.value.status == -4
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "fp32", "fp32_qf64"])
@pytest.mark.parametrize("pin", [False, True], ids=["pageable", "pinned"])
def test_float32_q_input_equals_the_float64_entry(precision, pin):
    """nlc_set_fields_f32 (Q in float32, rho0 and rest) gives the state that
    nlc_set_fields gives for the same values in float64, bit for bit, also
    after steps; a non-finite value is refused."""
    import torch
    from paper_1907_13415_gb300 import nlc
    w = wl.sphere_256().with_(shape=(9, 12, 34), size=4.0, noise=1e-3, seed=57)
    Q32 = w.initial_q5().astype(np.float32)
    if pin:
        t = torch.empty(Q32.shape, dtype=torch.float32, pin_memory=True)
        t.numpy()[...] = Q32
        src = t.numpy()
    else:
        src = Q32
    a, b = make(w, precision), make(w, precision)
    a.set_fields(Q32.astype(np.float64))
    b.set_fields_f32(src)
    for x, y in zip(a.get_fields(), b.get_fields()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.get_populations(), b.get_populations())
    a.step(3)
    b.step(3)
    assert np.array_equal(a.get_fields()[0], b.get_fields()[0])
    assert np.array_equal(a.get_populations(), b.get_populations())
    bad = Q32.copy()
    bad[4, 2, 3, 5] = np.inf
    with pytest.raises(nlc.NlcError) as ei:
        b.set_fields_f32(bad)
    assert ei.value.status == -4
    a.close()
    b.close()


def test_grid_barrier_wait_runs_out_and_context_recovers():
    """A wait budget of 0 makes the adjoint's cooperative segment kernels give
    up at their first grid-wide barrier that is not already complete (no
    tile copy is in flight there): the call fails with NLC_ETIMEOUT and
    every block returns.  With the budget restored the same context steps
    and differentiates exactly as a fresh one."""
    from paper_1907_13415_gb300 import nlc
    w = wl.adjoint_disc_128().with_(shape=(1, 24, 40), size=7.0)
    loss = (7.0, 1.0, 1.0)
    a = make(w, 0)
    a.set_fields(w.initial_q5())
    a.set_wait_budget(0)
    with pytest.raises(nlc.NlcError) as ei:
        a.adjoint(*loss, nsteps=12, ckpt_every=4)
    assert ei.value.status == -5
    assert "grid-barrier" in nlc.nlc_last_error(a.ctx)
    a.set_wait_budget(-1)
    a.set_fields(w.initial_q5())
    a.step(9)
    ga = a.adjoint(*loss, nsteps=12, ckpt_every=4)
    b = make(w, 0)
    b.set_fields(w.initial_q5())
    b.step(9)
    gb = b.adjoint(*loss, nsteps=12, ckpt_every=4)
    assert np.array_equal(a.get_populations(), b.get_populations())
    assert np.array_equal(a.get_fields()[0], b.get_fields()[0])
    for k in ("loss", "dgamma", "dK", "dGamma"):
        assert ga[k] == gb[k], k
    assert np.array_equal(ga["dQ0"], gb["dQ0"])
    a.close()
    b.close()


def test_set_fields_f32_reads_device_arrays_in_place():
    """nlc_set_fields_f32 takes Q as a float32 host array or a float32
    device array of the same layout; both give the same state and the same
    steps, bit for bit."""
    import torch
    w = wl.sphere_256().with_(shape=(9, 10, 33), size=3.0, noise=1e-3, seed=12)
    Q32 = w.initial_q5().astype(np.float32)
    a = make(w, 1)
    a.set_fields_f32(Q32)
    a.step(5)
    b = make(w, 1)
    d = torch.tensor(Q32, device="cuda")
    b.set_fields_f32(d.data_ptr())
    b.step(5)
    assert np.array_equal(a.get_populations(), b.get_populations())
    assert np.array_equal(a.get_fields()[0], b.get_fields()[0])
    a.close()
    b.close()
