"""Long-horizon FP32 drift against the FP64 oracle: the circular droplet
(256^2 D2Q9, R = 32, gamma = 2.70 + delta) for its full 20000 steps in the
FP32 bulk form with FP64 reductions, against the oracle run of the same
problem; max |dQ| (normwise), the radius and max |u| (the spurious velocity,
Sec. 2.2) compared every 2000 steps.

The oracle needs minutes of host time per case (1.3 G lattice updates), so
these run only with NLC_LONG=1; with NLC_LONG_OUT set, each case appends its
figures as one JSON line to that file, with the host seconds the oracle took
(OpenMP over all host cores) and the device seconds of the GPU run of the
same steps.
"""
import json
import os
import time

import numpy as np
import pytest

from paper_1907_13415_gb300 import workloads as wl

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("NLC_LONG") != "1",
                                 reason="long run (minutes of oracle time): NLC_LONG=1")]

EVERY = 2000


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("delta", [0.0, 0.002, 0.005])
def test_disc_256_fp32_20000_steps_against_oracle(orc, delta):
    import torch
    from paper_1907_13415_gb300 import nlc
    w = wl.disc_256(delta)
    steps = w.steps
    p = wl.param_vector(w.params)
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32,
                         stream=torch.cuda.current_stream().cuda_stream)
    sim.set_graph(50)
    Q0 = w.initial_q5()
    sim.set_fields(Q0)
    f = orc.init_equilibrium(w.lattice, w.shape)
    Q = Q0
    rows = []
    done = 0
    t_gpu = t_orc = 0.0
    while done < steps:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(EVERY)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        f, Q = orc.step(w.lattice, p, f, Q, EVERY)
        t2 = time.perf_counter()
        t_gpu += t1 - t0
        t_orc += t2 - t1
        done += EVERY
        og = sim.observables()
        oo = orc.observables(w.lattice, p, f, Q)
        Qg, _, _ = sim.get_fields()
        rows.append({"step": done,
                     "max_dQ_rel": float(np.abs(Qg - Q).max() / np.abs(Q).max()),
                     "radius_gpu": og["radius"], "radius_oracle": float(oo["radius"]),
                     "max_u_gpu": og["max_u"], "max_u_oracle": float(oo["max_u"])})
    sim.close()
    dR = max(abs(r["radius_gpu"] - r["radius_oracle"]) for r in rows)
    dQ = max(r["max_dQ_rel"] for r in rows)
    du = max(abs(r["max_u_gpu"] - r["max_u_oracle"]) / r["max_u_oracle"] for r in rows)
    summary = {"case": w.name, "steps": steps, "precision": "fp32",
               "reference": "FP64 CPU oracle", "max_dQ_rel": dQ,
               "radius_drift_max": dR, "max_u_rel_diff_max": du,
               "radius_final_gpu": rows[-1]["radius_gpu"],
               "radius_final_oracle": rows[-1]["radius_oracle"],
               "gpu_s": t_gpu, "oracle_s": t_orc, "oracle_threads": orc.set_threads(0),
               "trace": rows}
    out = os.environ.get("NLC_LONG_OUT")
    if out:
        with open(out, "a") as fh:
            fh.write(json.dumps(summary) + "\n")
    # FP32 storage and arithmetic over 20000 relaxational steps: the radius
    # stays within a thousandth of a cell, Q within 1e-3 normwise
    assert dR < 1e-3
    assert dQ < 1e-3
    assert du < 1e-2


def test_sweep_members_fp32_50000_steps_against_oracle(orc):
    """Two members of the 64-lattice temperature sweep (the smallest lattice
    and the one nearest coexistence), advanced inside the full batched
    context for the sweep's 50000 steps in FP32 (graph replay), against the
    oracle run of the same lattice: max |dQ| (normwise) and the drift of the
    interface position (Sec. 2.1) every 5000 steps."""
    import torch
    from paper_1907_13415_gb300 import nlc
    ws = wl.sweep_64()
    steps, every = 50000, 5000
    gam = np.array([w.params["gamma"] for w in ws])
    picks = sorted({int(np.argmin([w.n_cells for w in ws])), int(np.argmin(np.abs(gam - 2.7)))})
    b = nlc.Batch(wl.D2Q9, [w.shape for w in ws], [w.params for w in ws],
                  precision=nlc.NLC_FP32,
                  stream=torch.cuda.current_stream().cuda_stream, graph_steps=50)
    for i, w in enumerate(ws):
        b.set_fields(i, w.initial_q5())
    state = {}
    for i in picks:
        w = ws[i]
        state[i] = (orc.init_equilibrium(w.lattice, w.shape), w.initial_q5())
    rows = {i: [] for i in picks}
    done = 0
    while done < steps:
        b.step(every)
        done += every
        for i in picks:
            w = ws[i]
            p = wl.param_vector(w.params)
            f, Q = orc.step(w.lattice, p, state[i][0], state[i][1], every)
            state[i] = (f, Q)
            og = b.observables(i)
            oo = orc.observables(w.lattice, p, f, Q)
            Qg, _, _ = b.get_fields(i)
            rows[i].append({"step": done,
                            "max_dQ_rel": float(np.abs(Qg - Q).max() / np.abs(Q).max()),
                            "x_gpu": og["x_iface"], "x_oracle": float(oo["x_iface"])})
    b.close()
    out = os.environ.get("NLC_LONG_OUT")
    for i in picks:
        dx = max(abs(r["x_gpu"] - r["x_oracle"]) for r in rows[i])
        dQ = max(r["max_dQ_rel"] for r in rows[i])
        if out:
            with open(out, "a") as fh:
                fh.write(json.dumps({"case": ws[i].name, "gamma": ws[i].params["gamma"],
                                     "steps": steps, "precision": "fp32",
                                     "reference": "FP64 CPU oracle", "max_dQ_rel": dQ,
                                     "x_iface_drift_max": dx, "trace": rows[i]}) + "\n")
        assert dx < 1e-2, (ws[i].name, dx)
        assert dQ < 1e-3, (ws[i].name, dQ)


def test_flat_128x8_fp64_2000_steps_timed(orc):
    """The 128 x 8 flat interface (FP64, 2000 steps) in full on both sides:
    the state against the oracle's (the FP64 bound) and the time each side
    takes for the whole run."""
    import torch
    from paper_1907_13415_gb300 import nlc
    w = wl.flat_128x8()
    p = wl.param_vector(w.params)
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP64,
                         stream=torch.cuda.current_stream().cuda_stream)
    sim.set_graph(50)
    Q0 = w.initial_q5()
    sim.set_fields(Q0)
    sim.step(50)  # warm-up: graph capture, module load
    sim.set_fields(Q0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.step(w.steps)
    torch.cuda.synchronize()
    t_gpu = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, Qo = orc.step(w.lattice, p, orc.init_equilibrium(w.lattice, w.shape), Q0, w.steps)
    t_orc = time.perf_counter() - t0
    Qg, _, _ = sim.get_fields()
    sim.close()
    dq = float(np.abs(Qg - Qo).max() / np.abs(Qo).max())
    out = os.environ.get("NLC_LONG_OUT")
    if out:
        with open(out, "a") as fh:
            fh.write(json.dumps({"case": w.name, "steps": w.steps, "precision": "fp64",
                                 "reference": "FP64 CPU oracle", "max_dQ_rel": dq,
                                 "gpu_s": t_gpu, "oracle_s": t_orc,
                                 "oracle_threads": orc.set_threads(0)}) + "\n")
    assert dq < 1e-12
