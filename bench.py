#!/usr/bin/env python3
"""Throughput of the hybrid LB / Beris-Edwards step on GB300.

Workload: the spherical nematic droplet, 256^3 D3Q19 lattice, R = 48,
director along z, noise 1e-4, gamma = 2.705, FP32 (populations as deviations
from w_i rho0), synthetic seeded input.  One "step" is one full time step
(force, LB collide-and-stream, predictor-corrector for Q) of the whole
lattice.  Metric: MLUPS (million lattice-cell updates per second).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With N > 1 (launched by torchrun) every rank advances its own lattice
(independent replicas, weak scaling); value = all ranks' updates / max time.
Prints one JSON line on rank 0.
"""
import argparse
import datetime
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("MLUPS of fused LB+Beris-Edwards step, % of HBM roofline; "
          "adjoint/forward time")
UNIT = "MLUPS"
WORD = 4  # FP32
Q3 = 19

# Algorithmic bytes per lattice update (LUP), FP32:
#   whole step     : read + write of the 19 populations and 5 Q components
#   fused_lb kernel: read + write of the populations, read of Q
#   fused_be kernel: read + write of Q
ALG_BYTES_STEP = 2 * (Q3 + 5) * WORD          # 192 B
ALG_BYTES = {"fused_lb": (2 * Q3 + 5) * WORD,  # 172 B
             "fused_be": 2 * 5 * WORD}         # 40 B

# precision option: (library constant name, bytes of a population word,
# bytes of a Q word, arithmetic dtype)
PRECISIONS = {"fp32": ("NLC_FP32", 4, 4, "f32"),
              "fp64": ("NLC_FP64", 8, 8, "f64"),
              "fp32_qf64": ("NLC_FP32_QF64", 4, 8, "f64")}


def alg_bytes(precision):
    """(step, per-kernel) algorithmic bytes per LUP for a precision."""
    _, gw, qw, _ = PRECISIONS[precision]
    return (2 * (Q3 * gw + 5 * qw),
            {"fused_lb": 2 * Q3 * gw + 5 * qw, "fused_be": 2 * 5 * qw})

# DRAM traffic per LUP of each kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, divided by the cells of the
# captured launch), keyed by the SHA-256 of the kernel sources it was taken
# on; reported as null once those sources change.
NCU_TRAFFIC = {
    # 256 x 256 x 64 capture (4,194,304 cells), see profiles/
    "fused_lb": ((431.065600e6 + 333.152000e6) / 4194304, "967ef2352f20c314"),
    "fused_be": ((155.785728e6 + 61.327104e6) / 4194304, "967ef2352f20c314"),
}

KERNEL_SOURCES = ["paper_1907_13415_gb300/csrc/step_fused.cuh",
                  "paper_1907_13415_gb300/csrc/physics.cuh",
                  "paper_1907_13415_gb300/csrc/step_unfused.cuh",
                  "paper_1907_13415_gb300/csrc/lattice.cuh",
                  "paper_1907_13415_gb300/csrc/common.cuh",
                  "paper_1907_13415_gb300/csrc/packed.cuh",
                  "paper_1907_13415_gb300/csrc/tma.cuh",
                  "paper_1907_13415_gb300/csrc/aux_kernels.cuh"]


def source_hash():
    """SHA-256 of the kernel sources with their comments and blank lines
    removed (a comment edit leaves the kernels, and their counters, as
    they were), and of the compiler flags."""
    import re
    from paper_1907_13415_gb300 import build as nlc_build
    h = hashlib.sha256()
    h.update(" ".join(nlc_build.ARCH + nlc_build.NVFLAGS[:5]).encode())
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(text.encode())
    return h.hexdigest()[:16]


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# -- clocks -----------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running.
    Each sample carries nvidia-smi's timestamp; `region()` marks the timed
    region on the same (local) wall clock, and the summary takes the
    samples inside it (all samples if the region is shorter than the
    sampling interval, flagged in `window`)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev),
                 f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.INTERVAL_MS)], stdout=open(self.path, "w"),
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def start(self):
        self.t0 = datetime.datetime.now()

    def stop(self):
        self.t1 = datetime.datetime.now()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        return summarize_clock_samples(lines, self.t0, self.t1)


CLOCK_REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]


def summarize_clock_samples(lines, t0=None, t1=None):
    """Median SM clock, maximum clock and the throttle reasons seen, from
    nvidia-smi lines of ClockSampler.FIELDS; the samples stamped within
    [t0, t1] when there are any, else every sample (window "run")."""
    samples = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
        except ValueError:
            ts = None
        try:
            sm, smax = float(parts[2]), float(parts[3])
        except ValueError:
            continue
        active = {n for n, v in zip(CLOCK_REASONS, parts[6:10])
                  if v.lower().startswith("active")}
        samples.append((ts, sm, smax, active))
    inside = [x for x in samples
              if t0 is not None and t1 is not None and x[0] is not None and t0 <= x[0] <= t1]
    use, window = (inside, "timed region") if inside else (samples, "run")
    if not use:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    reasons = set().union(*(x[3] for x in use))
    return {"sm_mhz": statistics.median(x[1] for x in use),
            "sm_max_mhz": max(x[2] for x in use), "reasons": sorted(reasons),
            "samples": len(use), "window": window,
            "interval_ms": ClockSampler.INTERVAL_MS}


# -- distributed helpers -------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, ws):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_rate(cells_per_rank, steps, elapsed_ms, ws):
    """Weak scaling over independent replicas: every rank advanced its own
    lattice for `steps` steps; the job's rate is all ranks' lattice updates
    over the slowest rank's time.  Returns (MLUPS, max elapsed ms)."""
    t_max = max_over_ranks(elapsed_ms, ws)
    return cells_per_rank * steps * ws / (t_max * 1e-3) / 1e6, t_max


# -- the oracle as CPU baseline / reference arm ------------------------------

def oracle_sample_rate(w, steps, shape=None):
    """Time the FP64 CPU oracle on a bounded sample of the workload.  Returns
    (MLUPS, threads, description, (f, Q) after the steps)."""
    import oracle
    from paper_1907_13415_gb300 import workloads as wl
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    orc = oracle.get()
    ws = w if shape is None else wl.scaled(w, shape)
    Q = ws.initial_q5()
    f = orc.init_equilibrium(ws.lattice, ws.shape)
    p = wl.param_vector(ws.params)
    threads = orc.set_threads(0)
    t0 = time.perf_counter()
    state = orc.step(ws.lattice, p, f, Q, steps)
    dt = time.perf_counter() - t0
    nz, ny, nx = ws.shape
    desc = (f"{steps} step(s) of the oracle on a {nx}x{ny}x{nz} D3Q19 lattice "
            f"with the droplet recipe, FP64, OpenMP")
    return nx * ny * nz * steps / dt / 1e6, threads, desc, state


def oracle_single_thread_rate(w):
    """The same oracle on one host thread, one step of an 8-plane slab of the
    workload.  Returns (MLUPS, description)."""
    import oracle
    from paper_1907_13415_gb300 import workloads as wl
    orc = oracle.get()
    nz, ny, nx = w.shape
    ws = wl.scaled(w, (min(8, nz), ny, nx))
    Q = ws.initial_q5()
    f = orc.init_equilibrium(ws.lattice, ws.shape)
    p = wl.param_vector(ws.params)
    saved = orc.set_threads(0)
    orc.set_threads(1)
    try:
        t0 = time.perf_counter()
        orc.step(ws.lattice, p, f, Q, 1)
        dt = time.perf_counter() - t0
    finally:
        orc.set_threads(saved)
    cells = ws.shape[0] * ny * nx
    return cells / dt / 1e6, (f"1 step of the oracle on a {nx}x{ny}x{ws.shape[0]} slab, "
                              f"FP64, one thread")


def mem_available_gb():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


def baseline_shape(w):
    """Full lattice when the host has room for the oracle's ~80 doubles per
    cell (plus copies), else a z slab of it."""
    nz, ny, nx = w.shape
    need_gb = 110 * 8 * nx * ny * nz / 1e9
    if mem_available_gb() > 2 * need_gb:
        return w.shape
    return (max(8, nz // 8), ny, nx)


ACC_STEPS = 2  # steps of the accuracy comparison with the oracle
ACC_HALF = 9   # half-width of the periodic box around a sampled cell


def accuracy_full(orc, w, gpu, state):
    """Normwise max |dQ| / max |Q| and max |df| / max |f| over the whole
    lattice, and the drift of mass and radius, of the GPU state after
    ACC_STEPS steps against the oracle's."""
    from paper_1907_13415_gb300 import workloads as wl
    Qg, fg, og, perm = gpu
    fo, Qo = state
    p = wl.param_vector(w.params)
    oo = orc.observables(w.lattice, p, fo, Qo)
    dq = float(np.abs(Qg - Qo).max() / np.abs(Qo).max())
    df = float(np.abs(fg - fo[perm]).max() / np.abs(fo).max())
    return {"steps": ACC_STEPS, "cells": "all",
            "max_dQ_rel": dq, "max_df_rel": df,
            "radius_gpu": og["radius"], "radius_oracle": float(oo["radius"]),
            "radius_drift": abs(og["radius"] - float(oo["radius"])),
            "mass_rel_drift": abs(og["mass"] - float(oo["mass"])) / float(oo["mass"]),
            "max_u_gpu": og["max_u"], "max_u_oracle": float(oo["max_u"])}


def accuracy_sampled(orc, w, Q0, gpu, ncells=12):
    """The same on sampled cells when the host cannot hold the oracle's
    full lattice: a cell's state after ACC_STEPS steps depends only on
    inputs within 4 ACC_STEPS cells, so the oracle on a periodic box of
    half-width ACC_HALF cut around the cell gives its exact result."""
    from paper_1907_13415_gb300 import workloads as wl
    Qg, fg, og, perm = gpu
    nz, ny, nx = w.shape
    c = (nx - 1) / 2.0
    cells = []
    for d in (np.array([1, 0, 0]), np.array([0, 1, 0]), np.array([0, 0, 1])):
        for rad in (w.size - 1.0, w.size, w.size + 1.0, 0.5 * w.size):
            q = np.rint(c + rad * d).astype(int)
            cells.append((int(q[2]), int(q[1]), int(q[0])))
    cells = cells[:ncells]
    p = wl.param_vector(w.params)
    box = 2 * ACC_HALF + 1
    dq = df = 0.0
    for (cz, cy, cx) in cells:
        iz = np.arange(cz - ACC_HALF, cz + ACC_HALF + 1) % nz
        iy = np.arange(cy - ACC_HALF, cy + ACC_HALF + 1) % ny
        ix = np.arange(cx - ACC_HALF, cx + ACC_HALF + 1) % nx
        Qb = Q0[:, iz][:, :, iy][:, :, :, ix].copy()
        fo, Qo = orc.step(w.lattice, p, orc.init_equilibrium(w.lattice, (box,) * 3), Qb,
                          ACC_STEPS)
        h = ACC_HALF
        dq = max(dq, float(np.abs(Qg[:, cz, cy, cx] - Qo[:, h, h, h]).max()))
        df = max(df, float(np.abs(fg[:, cz, cy, cx] - fo[perm][:, h, h, h]).max()))
    return {"steps": ACC_STEPS, "cells": f"{len(cells)} sampled (interface and bulk)",
            "max_dQ_rel": dq / float(np.abs(Q0).max()),
            "max_df_rel": df / float(np.abs(fg).max())}


def workload_config(args, w, ws):
    """The workload a bench line measures; the same dict on both arms."""
    nz, ny, nx = w.shape
    return {"workload": w.name, "lattice": "D3Q19", "precision": args.precision,
            "shape": [nx, ny, nz], "radius": w.size, "gamma": w.params["gamma"],
            "parallelism": f"replicas{ws}",
            "collision": "mrt" if args.mrt else "bgk",
            "l2": "inputs larger than L2 (3.2 GB of state)"}


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    # one reference step: one oracle step on a z slab of the workload, sized
    # so that warm-up + timed steps end within a few minutes
    nz, ny, nx = w.shape
    shape = (8, ny, nx)
    from paper_1907_13415_gb300 import workloads as wl
    import oracle
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    orc = oracle.get()
    ws_ = wl.scaled(w, shape)
    Q = ws_.initial_q5()
    f = orc.init_equilibrium(ws_.lattice, ws_.shape)
    p = wl.param_vector(ws_.params)
    for _ in range(args.warmup):
        f, Q = orc.step(ws_.lattice, p, f, Q, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, Q = orc.step(ws_.lattice, p, f, Q, 1)
    dt = time.perf_counter() - t0
    cells = shape[0] * shape[1] * shape[2]
    value = cells * args.steps / dt / 1e6
    sample = (f"{args.steps} oracle steps of a {nx}x{ny}x{shape[0]} slab of the "
              f"256^3 droplet lattice (FP64 CPU, OpenMP)")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args, w, ws),
        "cpu_baseline": {"value": value, "unit": UNIT,
                         "cores": int(os.environ["OMP_NUM_THREADS"]),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# -- our arm -------------------------------------------------------------------

def run_ours(args, w):
    import torch
    from paper_1907_13415_gb300 import nlc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    prec_name, _, _, dtype = PRECISIONS[args.precision]
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=getattr(nlc, prec_name),
                         stream=stream.cuda_stream,
                         schedule=(nlc.NLC_SCHED_FUSED if args.schedule == "fused"
                                   else nlc.NLC_SCHED_UNFUSED))
    if args.mrt:
        # MRT: shear moments at 1/tau (the BGK viscosity), the rest at 1.2
        rates = np.full(19, 1.2)
        rates[[9, 11, 13, 14, 15]] = 1.0 / w.params["tau"]
        sim.set_mrt(rates)
    Q0 = w.initial_q5()
    sim.set_fields(Q0)
    cells = w.n_cells

    # chunk depth of the fused kernels: autotuned on this state (the state is
    # restored afterwards), the library default, or fixed
    tune = None
    if args.chunk < 0:
        tune = sim.autotune(args.tune_steps)
    else:
        sim.set_chunk(args.chunk, args.taper)
    if args.persist > 0:
        sim.set_persistent(args.persist)

    # warm-up
    sim.step(args.warmup)
    torch.cuda.synchronize()

    # timed region: K steps, per-kernel events recorded by the library
    nlc.nlc_set_timing(sim.ctx, True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        clk.start()
        ev0.record(stream)
        if args.persist > 0:
            # the persistent form: cooperative launches of args.persist steps
            sim.step(args.steps)
        else:
            for _ in range(args.steps):
                sim.step(1)
        ev1.record(stream)
        torch.cuda.synchronize()
        clk.stop()
        barrier(ws)
    elapsed_ms = ev0.elapsed_time(ev1)
    kt = nlc.nlc_get_timing(sim.ctx)
    nlc.nlc_set_timing(sim.ctx, False)
    clocks = clk.summary()
    value, t_max = whole_job_rate(cells, args.steps, elapsed_ms, ws)
    launches = sum(n for _, n in kt.values())

    # roofline of the step (the pair of fused kernels that makes one time
    # step): algorithmic bytes 2 (q + 5) words per lattice update over the
    # device time of a step, against the measured HBM copy bandwidth; the
    # per-kernel figures sit under "kernels"
    peak, peak_src = hbm_peak()
    step_bytes, kern_bytes = alg_bytes(args.precision)
    step_s = t_max / args.steps * 1e-3
    src_ok = source_hash()
    ncu_ok = args.precision == "fp32" and not args.mrt
    kernels = {}
    ktot = max(sum(x[0] for x in kt.values()), 1e-30)
    for k, (ms, n) in kt.items():
        if not n:
            continue
        ab = kern_bytes.get(k)
        ent = {"ms_per_launch": ms / n, "launches": n, "share": ms / ktot}
        if ab is not None:
            ach = ab * cells / (ms / n * 1e-3) / 1e9
            ent.update({"alg_bytes_per_lup": ab, "achieved_gbs": ach, "frac": ach / peak})
            tr = NCU_TRAFFIC.get(k)
            if tr and tr[1] == src_ok and ncu_ok:
                ent["ncu_bytes_per_lup"] = tr[0]
                ent["ncu_gbs"] = tr[0] * cells / (ms / n * 1e-3) / 1e9
                ent["ncu_frac"] = ent["ncu_gbs"] / peak
        kernels[k] = ent
    step_traffic = None
    if ncu_ok and all(NCU_TRAFFIC.get(k, (0, ""))[1] == src_ok for k in kern_bytes):
        step_traffic = sum(NCU_TRAFFIC[k][0] for k in kern_bytes) * cells
    achieved = step_bytes * cells / step_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": step_traffic,
                "kernel": "step (fused_lb + fused_be)", "peak_source": peak_src,
                "alg_bytes_per_lup": step_bytes,
                "numerator": (f"{step_bytes} B/LUP x {cells} cells (read + write of the "
                              f"{Q3} populations and 5 Q components) / device time of "
                              f"one step (ms_per_step)"),
                "denominator": f"hbm_gbs of MEASURED_PEAKS.json ({peak_src} copy bandwidth)",
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per LUP "
                                   "of both kernels (256x256x64 capture) x cells"
                                   if step_traffic else None)}

    # end to end through the public API with host buffers: upload Q from
    # pinned host memory (float32 for a float32 state, nlc_set_fields_f32;
    # float64 otherwise), one step, observables back to the host
    e2e = None
    if not args.no_e2e:
        f32_in = args.precision == "fp32"
        hdt = torch.float32 if f32_in else torch.float64
        pinned = torch.empty(Q0.shape, dtype=hdt, pin_memory=True)
        pinned.numpy()[...] = Q0
        qhost = pinned.numpy()
        upload = sim.set_fields_f32 if f32_in else sim.set_fields
        if f32_in:
            # every step's Q goes from pinned host memory to one of two device
            # buffers on a copy stream, the copy of step k + 1 overlapping the
            # set-up, step and observables of step k (nlc_set_fields_f32 reads
            # a device array in place)
            copy = torch.cuda.Stream()
            dbuf = [torch.empty(Q0.shape, dtype=torch.float32, device="cuda") for _ in range(2)]
            copied = [torch.cuda.Event() for _ in range(2)]
            used = [torch.cuda.Event() for _ in range(2)]
            for e in used:
                e.record(stream)

            def issue_copy(k):
                b = k % 2
                copy.wait_event(used[b])
                with torch.cuda.stream(copy):
                    dbuf[b].copy_(pinned, non_blocking=True)
                    copied[b].record(copy)

            def run(nsteps):
                issue_copy(0)
                for k in range(nsteps):
                    if k + 1 < nsteps:
                        issue_copy(k + 1)
                    stream.wait_event(copied[k % 2])
                    sim.set_fields_f32(dbuf[k % 2].data_ptr())
                    used[k % 2].record(stream)
                    sim.step(1)
                    sim.observables()
            how = ("Q copied from pinned host memory to a device buffer on a copy stream "
                   "(the copy of step k + 1 overlapping step k) + nlc_set_fields_f32 + "
                   "nlc_step(1) + nlc_observables() per step")
        else:
            def run(nsteps):
                for _ in range(nsteps):
                    upload(qhost)
                    sim.step(1)
                    sim.observables()
            how = "nlc_set_fields(Q from pinned host) + nlc_step(1) + nlc_observables() per step"
        run(2)
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(args.e2e_steps)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
        e2e = {"value": cells * args.e2e_steps * ws / e2e_s / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(qhost.nbytes),
               "d2h_bytes_per_step": int(np.dtype(np.float64).itemsize * 8 + 32),
               "steps": args.e2e_steps, "what": how}
    # accuracy against the FP64 oracle, outside the timed region: the state
    # ACC_STEPS steps after the initial fields, in the launch configuration
    # timed above
    gpu_state = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.no_accuracy:
        sim.set_fields(Q0)
        sim.step(ACC_STEPS)
        Qg, _, _ = sim.get_fields()
        fg = sim.get_populations()
        og = sim.observables()
        c_g, _ = nlc.nlc_lattice_velocities(w.lattice)
        gpu_state = (Qg, fg, og, c_g)
    nlc_chunk = sim.chunk()
    sim.close()

    cpu = None
    accuracy = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        shape = baseline_shape(w)
        # the timed oracle sample is ACC_STEPS steps, so that on the full
        # lattice its result is also the accuracy reference
        rate, cores, desc, state = oracle_sample_rate(w, ACC_STEPS, shape)
        rate1, desc1 = oracle_single_thread_rate(w)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": desc,
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": desc1}}
        if gpu_state is not None:
            orc = oracle.get()
            c_o, _ = orc.lattice(w.lattice)
            perm = [int(np.where((c_o == cv).all(axis=1))[0][0]) for cv in gpu_state[3]]
            gpu = gpu_state[:3] + (perm,)
            del gpu_state
            if tuple(shape) == tuple(w.shape):
                accuracy = accuracy_full(orc, w, gpu, state)
            else:
                accuracy = accuracy_sampled(orc, w, Q0, gpu)
            accuracy["reference"] = "FP64 CPU oracle"
        del state

    # the other two figures the metric names, on their own workloads:
    # adjoint/forward time (128^2 droplet, 2000 steps, checkpoints every 100)
    # and the batched temperature sweep against sequential contexts
    adjoint = sweep = None
    if rank == 0 and ws == 1 and not args.no_extras:
        adjoint = adjoint_figures(args)
        sweep = sweep_figures(args)

    if rank == 0:
        nz, ny, nx = w.shape
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic",
            "config": workload_config(args, w, ws),
            "tuning": {"chunk": nlc_chunk[0], "taper": nlc_chunk[1], "autotune": tune,
                       "persistent_steps": args.persist},
            "roofline": roofline,
            "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
            "accuracy": accuracy, "adjoint": adjoint, "sweep": sweep,
            "gpu_launches": launches, "clocks": clocks,
            "kernel_source": source_hash(),
        }
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def sweep_figures(args):
    """Batched temperature sweep: 64 flat-interface D2Q9 lattices of uneven
    extents (gamma over [2.60, 2.80]) advanced by the same launches and
    replayed as CUDA graphs, against the same lattices stepped one context
    after another.  Returns the figures as a dict."""
    import torch
    from paper_1907_13415_gb300 import nlc
    from paper_1907_13415_gb300 import workloads as wl
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ws = wl.sweep_64()
    cells = sum(w.n_cells for w in ws)
    b = nlc.Batch(wl.D2Q9, [w.shape for w in ws], [w.params for w in ws],
                  precision=nlc.NLC_FP32, stream=stream.cuda_stream,
                  graph_steps=args.graph_steps)
    for i, w in enumerate(ws):
        b.set_fields(i, w.initial_q5())
    # both arms run the chunk lists the autotuner picks for them (the state
    # is restored after tuning), or the one --chunk gives
    tune_b = None
    if args.chunk < 0:
        tune_b = b.autotune(args.tune_steps)
    else:
        b.set_chunk(args.chunk, args.taper)

    def timed(fn, steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    b.step(max(args.warmup, args.graph_steps))
    t_batch = timed(b.step, args.steps)
    # the same batch as cooperative launches of the persistent kernel, each
    # advancing persist_steps steps (inside the same graphs)
    t_pers = None
    if args.persist_steps > 0:
        for i, w in enumerate(ws):
            b.set_fields(i, w.initial_q5())
        b.set_persistent(args.persist_steps)
        b.step(max(args.warmup, args.graph_steps))
        t_pers = timed(b.step, args.steps)
        b.set_persistent(0)
    b.close()
    sims = []
    for w in ws:
        s = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32,
                           stream=stream.cuda_stream)
        s.set_fields(w.initial_q5())
        if args.chunk < 0:
            s.autotune(args.tune_steps)
        else:
            s.set_chunk(args.chunk, args.taper)
        sims.append(s)

    def seq(steps):
        for _ in range(steps):
            for s in sims:
                s.step(1)

    seq(args.warmup)
    t_seq = timed(seq, args.steps)
    for s in sims:
        s.close()
    v_b = cells * args.steps / (t_batch * 1e-3) / 1e6
    v_s = cells * args.steps / (t_seq * 1e-3) / 1e6
    return {"workload": "sweep_64 flat interfaces, D2Q9, Lx in {256..2048}, "
                        "Ly in {8,16,64}, gamma in [2.60, 2.80], FP32",
            "instances": len(ws), "cells": cells, "steps": args.steps,
            "graph_steps": args.graph_steps,
            "batched": {"value": v_b, "unit": UNIT, "ms_per_step": t_batch / args.steps,
                        "form": "two kernels per step, graphs of graph_steps steps"},
            "persistent": (None if t_pers is None else
                           {"value": cells * args.steps / (t_pers * 1e-3) / 1e6, "unit": UNIT,
                            "ms_per_step": t_pers / args.steps,
                            "persist_steps": args.persist_steps,
                            "form": "one cooperative launch per persist_steps steps, "
                                    "inside the same graphs",
                            "over_two_kernel_form": t_batch / t_pers}),
            "sequential": {"value": v_s, "unit": UNIT, "ms_per_step": t_seq / args.steps,
                           "launches_per_step": 2 * len(ws)},
            "tuning": {"batched": tune_b, "chunk": args.chunk, "taper": args.taper},
            "batched_over_sequential": t_seq / t_batch,
            "persistent_over_sequential": None if t_pers is None else t_seq / t_pers}


def run_sweep(args):
    f = sweep_figures(args)
    out = {"metric": "MLUPS, batched temperature sweep vs sequential contexts",
           "value": f["batched"]["value"], "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": f["batched"]["ms_per_step"], "higher_is_better": True,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": f["workload"], "instances": f["instances"],
                      "cells": f["cells"], "graph_steps": f["graph_steps"]},
           "tuning": f["tuning"], "sequential": f["sequential"],
           "batched_over_sequential": f["batched_over_sequential"]}
    print(json.dumps(out), flush=True)
    return 0


def adjoint_figures(args):
    """Adjoint cost: the 128x128 D2Q9 droplet (R = 24, gamma = 2.70),
    2000 steps with checkpoints every 100, FP32.  Ratio of one nlc_adjoint
    call (its forward sweep, the recomputation and the reverse sweep) to one
    plain forward run of the same steps, and to the same forward run
    replayed as CUDA graphs of ckpt_every steps (the library's fastest
    forward).  Returns the figures as a dict."""
    import torch
    from paper_1907_13415_gb300 import nlc
    from paper_1907_13415_gb300 import workloads as wl
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    w = wl.adjoint_disc_128()
    steps, ckpt = (args.adjoint_steps or w.steps), w.extra["ckpt_every"]
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32,
                         stream=stream.cuda_stream)
    Q0 = w.initial_q5()

    def fwd(graph_steps=0):
        sim.set_graph(graph_steps)
        sim.set_fields(Q0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(steps)
        torch.cuda.synchronize()
        sim.set_graph(0)
        return time.perf_counter() - t0

    def adj():
        sim.set_fields(Q0)
        t0 = time.perf_counter()
        g = sim.adjoint(24.0, 1.0, 1.0, nsteps=steps, ckpt_every=ckpt)
        return time.perf_counter() - t0, g

    if args.adjoint_once:
        # one adjoint call and nothing else (for a launch list under a
        # profiler; no timing is reported from such a run)
        ta, g = adj()
        sim.close()
        return {"workload": w.name, "steps": steps, "ckpt_every": ckpt,
                "adjoint_s_unwarmed": ta, "note": "single call for profiling"}
    fwd()
    fwd(ckpt)
    adj()
    tf = min(fwd() for _ in range(3))
    tfg = min(fwd(ckpt) for _ in range(3))
    runs = [adj() for _ in range(3)]
    ta = min(r[0] for r in runs)
    g = runs[0][1]
    sim.close()
    return {"workload": w.name, "steps": steps, "ckpt_every": ckpt, "dtype": "f32",
            "forward_s": tf, "adjoint_s": ta, "forward_graph_s": tfg,
            "ratio_vs_forward": ta / tf, "ratio_vs_graph_forward": ta / tfg,
            "timer": "host wall clock around each call, stream synchronised, best of 3",
            "gradient": {k: g[k] for k in ("loss", "radius", "dgamma", "dK", "dGamma")}}


def run_adjoint(args):
    f = adjoint_figures(args)
    if args.adjoint_once:
        print(json.dumps(f), flush=True)
        return 0
    out = {"metric": "adjoint/forward time", "value": f["ratio_vs_forward"],
           "unit": "ratio", "higher_is_better": False, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": f["workload"], "steps": f["steps"],
                      "ckpt_every": f["ckpt_every"]}}
    out.update({k: v for k, v in f.items() if k not in ("workload", "steps", "ckpt_every")})
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the comparison with the oracle after the timed region")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint and batched-sweep figures of the default line")
    ap.add_argument("--shape", default=None,
                    help="nz,ny,nx of a smaller lattice with the same recipe "
                         "(profiling captures); the reported workload is "
                         "the default 256^3")
    ap.add_argument("--schedule", default="fused", choices=["fused", "unfused"])
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS),
                    help="fp32 (default), fp64, or fp32_qf64 (float populations, "
                         "double Q and arithmetic)")
    ap.add_argument("--mrt", action="store_true",
                    help="time the MRT collision instead of BGK")
    ap.add_argument("--workload", default="sphere256",
                    choices=["sphere256", "sweep64", "adjoint128"],
                    help="sweep64: batched vs sequential temperature sweep")
    ap.add_argument("--adjoint-steps", type=int, default=0,
                    help="steps of the adjoint workload (default: its own 2000)")
    ap.add_argument("--persist", type=int, default=0,
                    help="sphere256: run the step as cooperative launches of the persistent "
                         "kernel, this many steps each (0: two kernels per step)")
    ap.add_argument("--adjoint-once", action="store_true",
                    help="adjoint128: one nlc_adjoint call, no timing (launch lists)")
    ap.add_argument("--graph-steps", type=int, default=50)
    ap.add_argument("--persist-steps", type=int, default=50,
                    help="sweep: steps per cooperative launch of the persistent kernel "
                         "(0: skip that arm)")
    ap.add_argument("--chunk", type=int, default=-1,
                    help="z planes per block of the fused kernels: -1 autotune "
                         "(default), 0 the library default, N fixed")
    ap.add_argument("--taper", action="store_true",
                    help="with --chunk N: tapered chunk list")
    ap.add_argument("--tune-steps", type=int, default=8,
                    help="steps timed per candidate chunk depth by the autotuner")
    args = ap.parse_args()
    # at least three untimed warm-up steps (reported as the count used)
    args.warmup = max(args.warmup, 3)
    from paper_1907_13415_gb300 import workloads as wl
    if args.workload == "sweep64":
        return run_sweep(args)
    if args.workload == "adjoint128":
        return run_adjoint(args)
    w = wl.sphere_256()
    if args.shape:
        nz, ny, nx = (int(v) for v in args.shape.split(","))
        w = wl.scaled(w, (nz, ny, nx), size=48 * min(nx, ny, nz) / 256)
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
