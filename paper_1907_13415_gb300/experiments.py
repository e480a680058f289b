"""The paper's experiments on the GPU library (Sec. 2), with the FP32 runs
compared against FP64 runs of the same problem.

  python -m paper_1907_13415_gb300.experiments flat   [--gamma 2.7 --steps 2000]
  python -m paper_1907_13415_gb300.experiments disc   [--delta 0.002 --steps 20000]
  python -m paper_1907_13415_gb300.experiments sweep  [--steps 50000]

flat  : flat interface (Sec. 2.1): interface position and velocity.
disc  : circular droplet (Sec. 2.2): radius against time, spurious velocity.
sweep : temperature sweep (Sec. 2.1, Fig. 1D inset): interface velocity
        against gamma for the 64 uneven lattices of the batched workload, in
        one batched context, next to the Allen-Cahn estimate.
paper_circle : the almost static circle of Sec. 2.2 with the paper's own
        parameters, for the spurious-velocity estimate (with --dump, the
        final Q, u and vorticity fields as .npz).
flat_paper : the flat interface of Sec. 2.1 with the paper's own parameters
        to t = 350000: interface velocity and the profile against Eq. 7.
Each prints one JSON object.  FP32 results carry max|dQ| (normwise, against
the FP64 run of the same problem) and the drift of the interface position or
radius.
"""
import argparse
import json
import math
import sys

import numpy as np

from . import nlc
from . import workloads as wl


# whole runs of this many steps replay a captured CUDA graph (the same
# arithmetic as stepping kernel by kernel, without the launch overhead that
# dominates the small lattices of the paper's experiments)
GRAPH_STEPS = 50


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _run(w, precision, steps, every, stencil=0):
    """Runs w, returning observables every `every` steps and the final Q."""
    s = nlc.Simulation(w.lattice, w.shape, w.params, precision=precision,
                       stream=_stream())
    s.set_graph(GRAPH_STEPS)
    s.set_stencil(stencil)
    s.set_fields(w.initial_q5())
    trace = [s.observables()]
    done = 0
    while done < steps:
        k = min(every, steps - done)
        s.step(k)
        done += k
        trace.append(s.observables())
    Q, _, _ = s.get_fields()
    s.close()
    return trace, Q


def _drift(key, t32, t64, Q32, Q64):
    a32 = np.array([o[key] for o in t32])
    a64 = np.array([o[key] for o in t64])
    return {"max_dQ_rel": float(np.abs(Q32 - Q64).max() / np.abs(Q64).max()),
            f"{key}_drift_final": float(a32[-1] - a64[-1]),
            f"{key}_drift_max": float(np.abs(a32 - a64).max())}


def flat(gamma=2.7, steps=2000, lx=128, ly=8, every=100):
    w = wl.flat_128x8().with_(shape=(1, ly, lx), size=lx // 2,
                              params=dict(wl.BASE_PARAMS, gamma=gamma))
    t64, Q64 = _run(w, nlc.NLC_FP64, steps, every)
    t32, Q32 = _run(w, nlc.NLC_FP32, steps, every)
    x = np.array([o["x_iface"] for o in t64])
    half = len(x) // 2
    v = float((x[-1] - x[half]) / ((len(x) - 1 - half) * every)) if len(x) > 2 else 0.0
    return {"experiment": "flat interface", "gamma": gamma, "lattice": [lx, ly],
            "steps": steps, "x_iface_fp64": float(x[-1]),
            "velocity_fp64": v, "max_u_fp64": float(t64[-1]["max_u"]),
            "fp32_vs_fp64": _drift("x_iface", t32, t64, Q32, Q64)}


def disc(delta=0.0, steps=20000, n=256, radius=32, every=500, stencil=0):
    w = wl.disc_256(delta).with_(shape=(1, n, n), size=radius)
    t64, Q64 = _run(w, nlc.NLC_FP64, steps, every, stencil)
    t32, Q32 = _run(w, nlc.NLC_FP32, steps, every, stencil)
    R = np.array([o["radius"] for o in t64])
    tail = max(2, len(R) // 4)
    dRdt = float((R[-1] - R[-tail]) / ((tail - 1) * every))
    return {"experiment": "circular droplet", "delta": delta,
            "stencil": "isotropic" if stencil else "standard",
            "gamma": w.params["gamma"], "lattice": [n, n], "radius0": radius,
            "steps": steps, "radius_fp64": [float(r) for r in R[:: max(1, len(R) // 10)]],
            "dRdt_fp64": dRdt,
            "max_u_fp64": float(t64[-1]["max_u"]),
            "fp32_vs_fp64": _drift("radius", t32, t64, Q32, Q64)}


def vorticity(u):
    """omega_z = d_x u_y - d_y u_x of a (3, nz, ny, nx) velocity field by
    periodic central differences (the field the paper's Fig. 2B colours)."""
    ux, uy = u[0], u[1]
    return ((np.roll(uy, -1, axis=-1) - np.roll(uy, 1, axis=-1))
            - (np.roll(ux, -1, axis=-2) - np.roll(ux, 1, axis=-2))) / 2.0


def paper_circle(angle_deg=0.0, steps=35000, every=1000, gamma=2.707681,
                 lattice=wl.D2Q9, dump=None, stencil=0):
    """Sec. 2.2 / Fig. 2 with the paper's parameters (tau = 1.5, K = 0.04,
    Gamma = 0.34, xi = 0.7, A0 = 0.1): a 100 x 100 lattice, disc of radius 25,
    director at angle_deg from y, gamma = 2.707681.  Reports the interface
    velocity dR/dt and max |u| at the end (the paper: u_i ~ 1.89e-7,
    u_max = 8.97e-7 at 0 deg and 1.13e-6 at 20 deg, on D3Q19 with MRT).
    lattice: D2Q9, or D3Q19 on a single plane (nz = 1) as in the paper.
    dump: path of an .npz file for the final Q, u and vorticity fields."""
    a = math.radians(angle_deg)
    p = dict(wl.PAPER_PARAMS, gamma=gamma)
    w = wl.Workload("paper_circle", lattice, (1, 100, 100), p, steps, "ball", 25,
                    (math.sin(a), math.cos(a), 0.0), 0.0, 0)
    s = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP64,
                       stream=_stream())
    s.set_graph(GRAPH_STEPS)
    s.set_stencil(stencil)
    s.set_fields(w.initial_q5())
    trace = [s.observables()]
    done = 0
    while done < steps:
        k = min(every, steps - done)
        s.step(k)
        done += k
        trace.append(s.observables())
    Q, rho, u = s.get_fields()
    s.close()
    om = vorticity(u)
    if dump:
        np.savez_compressed(dump, Q=Q, rho=rho, u=u, vorticity=om)
    R = np.array([o["radius"] for o in trace])
    tail = max(2, len(R) // 4)
    return {"experiment": "paper circle", "angle_deg": angle_deg, "gamma": gamma,
            "lattice": "D2Q9" if lattice == wl.D2Q9 else "D3Q19 (nz = 1)",
            "stencil": "isotropic" if stencil else "standard",
            "steps": steps, "radius_final": float(R[-1]),
            "dRdt_final": float((R[-1] - R[-tail]) / ((tail - 1) * every)),
            "max_u_final": float(trace[-1]["max_u"]),
            "max_abs_vorticity": float(np.abs(om).max())}


def tanh_fit(profile, x_guess, lam=None, s_n=None, window=6.0):
    """FP64 least-squares fit of Eq. 7, S = S_n/2 [1 - tanh((x - x_i)/(2 lambda))],
    to a mean S(x) profile around one descending interface.  x_i is always
    free; S_n and lambda are fitted unless given.  Returns (x_i, S_n, lambda,
    rms residual)."""
    from scipy.optimize import least_squares
    prof = np.asarray(profile, dtype=np.float64)
    x = np.arange(prof.size, dtype=np.float64)
    lam0 = 2.0 if lam is None else lam
    sel = np.abs(x - x_guess) < window * lam0
    xs, ys = x[sel], prof[sel]

    def unpack(v):
        k = 1
        sn = s_n if s_n is not None else v[k]
        k += s_n is None
        la = lam if lam is not None else v[k]
        return v[0], sn, la

    def resid(v):
        xi, sn, la = unpack(v)
        return sn / 2 * (1 - np.tanh((xs - xi) / (2 * la))) - ys

    v0 = [x_guess] + ([] if s_n is not None else [max(ys.max(), 1e-6)]) + \
         ([] if lam is not None else [lam0])
    r = least_squares(resid, v0, method="lm", xtol=1e-15, ftol=1e-15)
    xi, sn, la = unpack(r.x)
    return float(xi), float(sn), float(la), float(np.sqrt(np.mean(r.fun ** 2)))


def flat_paper(gamma=2.7, steps=350000, lx=200, ly=8, every=10000):
    """Sec. 2.1 / Fig. 1 with the paper's parameters: a nematic slab in the
    middle of an lx x ly lattice (director along y), run to t = 350000.
    Reports the right interface's position and velocity, max |u|, and the
    largest deviation of the S(x) profile from Eq. 7 with S_n = 1/3 and
    lambda = 2 (fitted interface position), FP64."""
    p = dict(wl.PAPER_PARAMS, gamma=gamma)
    w = wl.Workload("flat_paper", wl.D2Q9, (1, ly, lx), p, steps, "slab", lx // 2,
                    (0, 1, 0), 0.0, 0)
    # nematic in the centre: S = 1/3 for lx/4 <= x < 3 lx/4
    S = np.where((np.arange(lx) >= lx // 4) & (np.arange(lx) < 3 * lx // 4), wl.S_COEX, 0.0)
    Q0 = wl.uniaxial_q5(np.broadcast_to(S, (1, ly, lx)).copy(), (0, 1, 0))
    s = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP64,
                       stream=_stream())
    s.set_graph(GRAPH_STEPS)
    s.set_fields(Q0)
    xs, done = [], 0
    while done < steps:
        k = min(every, steps - done)
        s.step(k)
        done += k
        xs.append(s.observables()["x_iface"])
    o = s.observables(profile=True)
    s.close()
    prof = np.asarray(o["s_profile"])
    x = np.arange(lx, dtype=np.float64)
    lam, Sn = 2.0, 1.0 / 3.0
    xr = o["x_iface"]
    # Eq. 7 around the right interface: S = S_n/2 [1 - tanh((x - x_i)/(2 lambda))]
    win = np.abs(x - xr) < 6 * lam
    best = min((np.abs(prof[win] - Sn / 2 * (1 - np.tanh((x[win] - xi) / (2 * lam)))).max(), xi)
               for xi in np.linspace(xr - 0.5, xr + 0.5, 201))
    xs = np.array(xs)
    half = len(xs) // 2
    v = float(np.polyfit(np.arange(half, len(xs)) * every, xs[half:], 1)[0]) if len(xs) > 3 else 0.0
    xf, snf, laf, rms = tanh_fit(prof, xr)
    return {"experiment": "flat interface (paper parameters)", "gamma": gamma,
            "lattice": [lx, ly], "steps": steps, "x_iface": float(xr),
            "velocity": v, "max_u": float(o["max_u"]),
            "eq7_max_deviation": float(best[0]), "eq7_fit_x_iface": float(best[1]),
            "tanh_fit": {"x_i": xf, "S_n": snf, "lambda": laf, "rms": rms}}


def sweep(steps=50000, every=2500, graph_steps=50):
    """Interface velocity against gamma from one batched context."""
    ws = wl.sweep_64()
    b = nlc.Batch(wl.D2Q9, [w.shape for w in ws], [w.params for w in ws],
                  precision=nlc.NLC_FP32, stream=_stream(), graph_steps=graph_steps)
    for i, w in enumerate(ws):
        b.set_fields(i, w.initial_q5())
    xs = [[] for _ in ws]
    done = 0
    while done < steps:
        b.step(every)
        done += every
        for i in range(len(ws)):
            xs[i].append(b.observables(i)["x_iface"])
    out = []
    for i, w in enumerate(ws):
        x = np.array(xs[i])
        g = w.params["gamma"]
        # fit over the second half, while an interface exists
        sel = x[len(x) // 2:]
        ok = bool(np.all(sel >= 0))
        v = float(np.polyfit(np.arange(len(sel)) * every, sel, 1)[0]) if ok else None
        lam = math.sqrt(27 * w.params["K"] / (w.params["A0"] * g))
        v_est = 10 / 9 * w.params["Gamma"] * w.params["A0"] * lam * (g - 2.7)
        out.append({"gamma": g, "lattice": [w.shape[2], w.shape[1]],
                    "velocity": v, "allen_cahn_estimate": v_est,
                    "interface_survives": ok,
                    # below the spinodal 8/3 the bulk nematic is unstable
                    "nematic_unstable": bool(g < 8.0 / 3.0)})
    b.close()
    return {"experiment": "temperature sweep", "steps": steps, "instances": out}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["flat", "disc", "sweep", "paper_circle", "flat_paper"])
    ap.add_argument("--angle", type=float, default=0.0)
    ap.add_argument("--lattice", choices=["d2q9", "d3q19"], default="d2q9")
    ap.add_argument("--dump", default=None, help="paper_circle: .npz of the final fields")
    ap.add_argument("--isotropic", action="store_true",
                    help="disc, paper_circle: isotropic finite-difference stencils")
    ap.add_argument("--gamma", type=float, default=2.7)
    ap.add_argument("--delta", type=float, default=0.0)
    ap.add_argument("--steps", type=int, default=None)
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    if args.which == "flat":
        r = flat(args.gamma, args.steps or 2000)
    elif args.which == "disc":
        r = disc(args.delta, args.steps or 20000, stencil=int(args.isotropic))
    elif args.which == "paper_circle":
        r = paper_circle(args.angle, args.steps or 35000,
                         lattice=wl.D3Q19 if args.lattice == "d3q19" else wl.D2Q9,
                         dump=args.dump, stencil=int(args.isotropic))
    elif args.which == "flat_paper":
        r = flat_paper(args.gamma, args.steps or 350000)
    else:
        r = sweep(args.steps or 50000)
    print(json.dumps(r))
    return 0


if __name__ == "__main__":
    sys.exit(main())
