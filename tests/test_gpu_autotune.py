"""Chunk depth of the fused kernels (nlc_set_chunk) and the autotuner
(nlc_autotune).  The depth only changes how the lattice is split among
thread blocks, so every depth must give the same step bit for bit; the
autotuner must leave the state exactly as it found it, and its cache file
must be written once and then read back."""
import json

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


def stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def droplet(shape=(23, 20, 40), seed=31):
    base = wl.sphere_256()
    return base.with_(shape=shape, size=0.3 * min(shape), noise=1e-3, seed=seed)


def state(sim):
    Q, rho, u = sim.get_fields()
    return Q, sim.get_populations(), rho, u


CHUNKS = ((0, False), (1, False), (2, False), (3, False), (4, False), (7, False),
          (23, False), (64, False), (4, True), (6, True), (16, True))


@pytest.mark.parametrize("lattice", ["D3Q19", "D2Q9"])
@pytest.mark.parametrize("precision", ["NLC_FP32", "NLC_FP64"])
def test_every_chunk_depth_gives_the_same_step(precision, lattice):
    """Chunks of z planes on D3Q19, of 32 x 8 tiles stacked along y on D2Q9
    (a ragged 70 x 61 lattice: 8 tiles per column, the last one partial)."""
    from paper_1907_13415_gb300 import nlc
    prec = getattr(nlc, precision)
    if lattice == "D3Q19":
        w = droplet()
        length = w.shape[0]
    else:
        w = wl.disc_256().with_(shape=(1, 61, 70), size=14.0, noise=1e-3, seed=35)
        length = 8
    ref = None
    for chunk, taper in CHUNKS:
        sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=prec,
                             stream=stream())
        sim.set_chunk(chunk, taper)
        depth, tapered = sim.chunk()
        assert tapered == taper
        if chunk:
            assert depth == min(chunk, length)
        sim.set_fields(w.initial_q5())
        sim.step(7)
        got = state(sim)
        sim.close()
        if ref is None:
            ref = got
            continue
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), chunk


def test_chunk_change_between_steps_and_graphs():
    """A new depth applies to the next step, also with graph replay."""
    from paper_1907_13415_gb300 import nlc
    w = droplet(seed=32)
    sims = []
    for chunks in (((0, False), (0, False)), ((5, False), (4, True))):
        sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32,
                             stream=stream())
        sim.set_graph(3)
        sim.set_fields(w.initial_q5())
        sim.set_chunk(*chunks[0])
        sim.step(7)
        sim.set_chunk(*chunks[1])
        sim.step(6)
        sims.append(state(sim))
        sim.close()
    for a, b in zip(*sims):
        assert np.array_equal(a, b)


def test_autotune_keeps_the_state_and_the_trajectory(tmp_path, monkeypatch):
    from paper_1907_13415_gb300 import nlc
    monkeypatch.delenv("NLC_TUNE_CACHE", raising=False)
    w = droplet(shape=(40, 24, 64), seed=33)
    tuned = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32,
                           stream=stream())
    plain = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32,
                           stream=stream())
    for s in (tuned, plain):
        s.set_fields(w.initial_q5())
        s.step(3)   # an odd number: the state sits in the second buffer
    before = state(tuned)
    r = tuned.autotune(trial_steps=3)
    assert r["from_cache"] == 0 and r["candidates"] >= 2 and r["trial_steps"] == 3
    assert r["best_ms"] > 0 and r["default_ms"] >= r["best_ms"]
    assert tuned.chunk() == (r["chunk"], bool(r["taper"]))
    assert 1 <= r["chunk"] <= w.shape[0]
    after = state(tuned)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    assert tuned.observables()["step"] == 3
    for s in (tuned, plain):
        s.step(5)
    for a, b in zip(state(tuned), state(plain)):
        assert np.array_equal(a, b)
    tuned.close()
    plain.close()


def test_autotune_cache_is_written_then_read(tmp_path, monkeypatch):
    from paper_1907_13415_gb300 import nlc
    path = tmp_path / "tune.json"
    monkeypatch.setenv("NLC_TUNE_CACHE", str(path))
    w = droplet(shape=(16, 16, 32), seed=34)
    first = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32,
                           stream=stream())
    first.set_fields(w.initial_q5())
    r1 = first.autotune(trial_steps=2)
    first.close()
    assert r1["from_cache"] == 0
    cache = json.loads(path.read_text())
    assert len(cache) == 1
    (key, val), = cache.items()
    assert key.startswith("D3Q19/fp32/n1/32x16x16/std/")
    assert val == (-r1["chunk"] if r1["taper"] else r1["chunk"])
    second = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32,
                            stream=stream())
    r2 = second.autotune(trial_steps=2)
    assert r2["from_cache"] == 1 and r2["chunk"] == r1["chunk"]
    assert r2["taper"] == r1["taper"]
    assert second.chunk() == (r1["chunk"], bool(r1["taper"]))
    # another stencil is another key
    second.set_stencil(nlc.NLC_STENCIL_ISOTROPIC)
    r3 = second.autotune(trial_steps=2)
    assert r3["from_cache"] == 0
    assert len(json.loads(path.read_text())) == 2
    second.close()


def test_autotune_single_plane_keeps_the_state(monkeypatch):
    """On D2Q9 the tuner times stacks of tiles along y (a 64 x 200 lattice
    has 25 tiles per column) and restores the state."""
    from paper_1907_13415_gb300 import nlc
    monkeypatch.delenv("NLC_TUNE_CACHE", raising=False)
    w = wl.disc_256().with_(shape=(1, 200, 64), size=30, noise=1e-3, seed=36)
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32,
                         stream=stream())
    sim.set_fields(w.initial_q5())
    sim.step(3)
    before = state(sim)
    r = sim.autotune(trial_steps=2)
    assert r["candidates"] >= 3 and 1 <= r["chunk"] <= 25
    assert sim.chunk() == (r["chunk"], bool(r["taper"]))
    for a, b in zip(before, state(sim)):
        assert np.array_equal(a, b)
    with pytest.raises(nlc.NlcError):
        sim.autotune(trial_steps=0)
    with pytest.raises(nlc.NlcError):
        sim.set_chunk(-1)
    with pytest.raises(nlc.NlcError):
        nlc._check(sim.ctx, nlc.load().nlc_set_chunk(sim.ctx, 8, 2))
    sim.close()


@pytest.mark.parametrize("lattice", ["D3Q19", "D2Q9"])
@pytest.mark.parametrize("precision", ["NLC_FP32", "NLC_FP64", "NLC_FP32_QF64"])
def test_population_offsets_in_32_and_64_bits_give_the_same_step(precision, lattice,
                                                                monkeypatch):
    """The fused lb kernel addresses populations with 32-bit offsets on
    lattices with q n < 2^32 and with 64-bit ones above; NLC_POP_INDEX64=1
    forces the 64-bit form, which must give the same step bit for bit."""
    from paper_1907_13415_gb300 import nlc
    prec = getattr(nlc, precision)
    if lattice == "D3Q19":
        w = droplet(seed=41)
    else:
        w = wl.disc_256().with_(shape=(1, 61, 70), size=14.0, noise=1e-3, seed=43)
    got = []
    for wide in ("0", "1"):
        monkeypatch.setenv("NLC_POP_INDEX64", wide)
        sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=prec,
                             stream=stream())
        sim.set_chunk(3 if lattice == "D3Q19" else 2, False)
        sim.set_fields(w.initial_q5())
        sim.step(6)
        got.append(state(sim))
        sim.close()
    for a, b in zip(*got):
        assert np.array_equal(a, b)
