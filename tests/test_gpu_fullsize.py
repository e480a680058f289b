"""Parity at the full sizes of the measured workloads.

The 256^3 D3Q19 spherical droplet in FP32, in the bench's launch
configuration (the chunk list the autotuner picks), two steps:

The oracle cannot step the whole lattice in seconds, so it checks sampled
cells one by one: one step at a cell depends only on inputs within four
cells (Q) and three cells (populations), so two steps of the oracle on a
periodic 19^3 box cut around a cell give that cell's exact result at the box
centre.  Samples sit on the droplet interface, in the bulk inside and
outside, on every lattice face (periodic wrap), and on tile and z-chunk
boundaries.  Properties that hold at any size are checked over the whole
lattice: mass is conserved and the total momentum stays zero (the force is
the divergence of the stress, which sums to zero on a periodic lattice).

The 256^2 circular droplet and members of the 64-lattice temperature sweep
are small enough to compare every cell with the oracle; the adjoint
workload (128^2, 2000 steps) is checked against central differences of the
forward run.
"""
import numpy as np
import pytest

from paper_1907_13415_gb300 import workloads as wl

from helpers import PARAM_SETS, fp32_tolerance, perm_to_oracle

pytestmark = pytest.mark.gpu

STEPS = 2
HALF = 9  # box half-width: 2 steps x 4 cells of dependence, plus one


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def sample_cells(w, chunk_bounds):
    nz, ny, nx = w.shape
    c = (nx - 1) / 2.0
    r = w.size
    cells = []
    # on the interface along each axis and a diagonal, inside and outside
    for d in (np.array([1, 0, 0]), np.array([0, 1, 0]), np.array([0, 0, 1]),
              np.array([1, 1, 1]) / np.sqrt(3)):
        for rad in (r - 1.0, r, r + 1.0, 0.5 * r, 1.5 * r):
            p = np.rint(c + rad * d).astype(int)
            cells.append((int(p[2]), int(p[1]), int(p[0])))
    # lattice faces, edges and corners (periodic wrap)
    cells += [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (0, 128, 255), (255, 0, 128),
              (128, 255, 0)]
    # tile boundaries (32 x 8) and z-chunk boundaries of the launch
    cells += [(100, 7, 31), (100, 8, 32), (140, 127, 96)]
    for b in chunk_bounds[1:-1][:3]:
        cells += [(b - 1, 120, 64), (b, 121, 65)]
    return cells


@pytest.mark.parametrize("pset", ["tau1", "paper"])
def test_sampled_cells_match_oracle_at_full_size(orc, pset):
    """With the workload's parameters (tau = 1) and with the paper's
    (tau = 1.5, K = 0.04, Gamma = 0.34; Sec. 2), where the collision keeps
    a third of the incoming populations."""
    import torch
    from paper_1907_13415_gb300 import nlc
    w = wl.sphere_256()
    w = w.with_(params=dict(PARAM_SETS[pset], gamma=w.params["gamma"]))
    nz, ny, nx = w.shape
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32,
                         stream=torch.cuda.current_stream().cuda_stream)
    Q0 = w.initial_q5()
    sim.set_fields(Q0)
    tune = sim.autotune(2)
    m0 = sim.observables()
    sim.step(STEPS)
    obs = sim.observables()
    Q, _, _ = sim.get_fields()
    f = sim.get_populations()
    sim.close()

    # the chunk list the kernels ran with (csrc/chunks.h)
    depth, taper = tune["chunk"], bool(tune["taper"])
    bounds = [0]
    z = 0
    if not taper:
        while z < nz:
            z = min(z + depth, nz)
            bounds.append(z)
    else:
        while nz - z > 2 * depth:
            z += depth
            bounds.append(z)
        rr = nz - z
        while rr > 0:
            cc = (rr + 1) // 2 if rr > 8 else rr
            if 0 < rr - cc < 4:
                cc = rr
            z += cc
            rr -= cc
            bounds.append(z)

    # properties over the whole lattice
    assert obs["nonfinite"] == 0
    assert abs(obs["mass"] - m0["mass"]) < 1e-6 * m0["mass"]
    for k in ("mom_x", "mom_y", "mom_z"):
        assert abs(obs[k]) < 1e-6 * m0["mass"], k

    perm = perm_to_oracle(orc, w.lattice)
    p = wl.param_vector(w.params)
    box = 2 * HALF + 1
    tol = fp32_tolerance(STEPS)
    f_scale = np.abs(f).max()
    q_scale = np.abs(Q0).max()
    for (cz, cy, cx) in sample_cells(w, bounds):
        iz = np.arange(cz - HALF, cz + HALF + 1) % nz
        iy = np.arange(cy - HALF, cy + HALF + 1) % ny
        ix = np.arange(cx - HALF, cx + HALF + 1) % nx
        Qb = Q0[:, iz][:, :, iy][:, :, :, ix].copy()
        f0 = orc.init_equilibrium(w.lattice, (box, box, box))
        fo, Qo = orc.step(w.lattice, p, f0, Qb, STEPS)
        dq = np.abs(Q[:, cz, cy, cx] - Qo[:, HALF, HALF, HALF]).max()
        df = np.abs(f[:, cz, cy, cx] - fo[perm][:, HALF, HALF, HALF]).max()
        assert dq < tol * q_scale, ((cz, cy, cx), dq)
        assert df < tol * f_scale, ((cz, cy, cx), df)


def run_gpu_steps(w, steps, precision):
    import torch
    from paper_1907_13415_gb300 import nlc
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=precision,
                         stream=torch.cuda.current_stream().cuda_stream)
    sim.set_fields(w.initial_q5())
    sim.step(steps)
    Q, _, _ = sim.get_fields()
    f = sim.get_populations()
    obs = sim.observables()
    sim.close()
    return Q, f, obs


@pytest.mark.parametrize("delta,pset", [(0.0, "tau1"), (0.005, "tau1"), (0.0, "paper")])
def test_disc_256_fp32_matches_oracle_in_full(orc, delta, pset):
    """The circular droplet (256^2 D2Q9, R = 32) at its full size in the FP32
    bulk form, every cell against the FP64 oracle, with the FP64 drift of
    mass and radius (also with the paper's parameters, tau = 1.5)."""
    w = wl.disc_256(delta)
    w = w.with_(params=dict(PARAM_SETS[pset], gamma=w.params["gamma"]))
    steps = 50
    Q, f, obs = run_gpu_steps(w, steps, precision=1)
    p = wl.param_vector(w.params)
    f0 = orc.init_equilibrium(w.lattice, w.shape)
    fo, Qo = orc.step(w.lattice, p, f0, w.initial_q5(), steps)
    oo = orc.observables(w.lattice, p, fo, Qo)
    perm = perm_to_oracle(orc, w.lattice)
    tol = fp32_tolerance(steps)
    assert np.abs(Q - Qo).max() < tol * np.abs(Qo).max()
    assert np.abs(f - fo[perm]).max() < tol * np.abs(fo).max()
    assert abs(obs["radius"] - float(oo["radius"])) < 1e-4
    assert abs(obs["mass"] - float(oo["mass"])) < 1e-6 * float(oo["mass"])


def test_sweep_64_members_match_oracle(orc):
    """The batched temperature sweep at its full size (64 lattices in one
    tile list, steps replayed as CUDA graphs as the bench runs it): the
    largest, the smallest and a middle member, every cell against the
    oracle."""
    import torch
    from paper_1907_13415_gb300 import nlc
    ws = wl.sweep_64()
    steps = 10
    b = nlc.Batch(wl.D2Q9, [w.shape for w in ws], [w.params for w in ws],
                  precision=nlc.NLC_FP32,
                  stream=torch.cuda.current_stream().cuda_stream, graph_steps=5)
    for i, w in enumerate(ws):
        b.set_fields(i, w.initial_q5())
    b.step(steps)
    cells = [w.n_cells for w in ws]
    picks = {int(np.argmax(cells)), int(np.argmin(cells)), len(ws) // 2}
    perm = perm_to_oracle(orc, wl.D2Q9)
    tol = fp32_tolerance(steps)
    for i in sorted(picks):
        w = ws[i]
        Q, _, _ = b.get_fields(i)
        f = b.get_populations(i)
        p = wl.param_vector(w.params)
        fo, Qo = orc.step(w.lattice, p, orc.init_equilibrium(w.lattice, w.shape),
                          w.initial_q5(), steps)
        assert np.abs(Q - Qo).max() < tol * np.abs(Qo).max(), i
        assert np.abs(f - fo[perm]).max() < tol * np.abs(fo).max(), i
    b.close()


@pytest.mark.parametrize("pset", ["tau1", "paper"])
def test_adjoint_workload_in_full_matches_central_differences(pset):
    """The adjoint workload at its full size (128^2 D2Q9 disc, 2000 steps,
    checkpoints every 100): the FP64 adjoint's dL/dgamma against central
    differences (h = 1e-6) of the FP64 forward run, and the FP32 adjoint
    within 1e-4 of the FP64 one (measured: below 1e-5).  (The oracle's own derivative, by complex
    step, is the check at smaller sizes.)  Also with the paper's parameters
    (tau = 1.5), where the adjoint of the collision carries a third of each
    population's adjoint back."""
    import torch
    from paper_1907_13415_gb300 import nlc
    w = wl.adjoint_disc_128()
    w = w.with_(params=dict(PARAM_SETS[pset], gamma=w.params["gamma"]))
    steps, ckpt, target = w.steps, w.extra["ckpt_every"], w.extra["target_radius"]
    st = torch.cuda.current_stream().cuda_stream

    def adjoint(precision):
        s = nlc.Simulation(w.lattice, w.shape, w.params, precision=precision, stream=st)
        s.set_fields(w.initial_q5())
        g = s.adjoint(target, 1.0, 1.0, nsteps=steps, ckpt_every=ckpt, want_dQ0=False)
        s.close()
        return g

    g64, g32 = adjoint(0), adjoint(1)
    h = 1e-6
    Ls = []
    for sgn in (1, -1):
        p = dict(w.params, gamma=w.params["gamma"] + sgn * h)
        s = nlc.Simulation(w.lattice, w.shape, p, precision=0, stream=st)
        s.set_fields(w.initial_q5())
        s.step(steps)
        o = s.observables()
        Ls.append((o["radius"] - target) ** 2 + o["u_l2"])
        s.close()
    fd = (Ls[0] - Ls[1]) / (2 * h)
    assert g64["dgamma"] == pytest.approx(fd, rel=1e-5)
    for k in ("dgamma", "dK", "dGamma"):
        assert g32[k] == pytest.approx(g64[k], rel=1e-4), k


def test_whole_256cubed_lattice_fp32_matches_oracle(orc):
    """Every cell of the 256^3 droplet (the bench's workload and autotuned
    launch configuration) after 2 FP32 steps against 2 steps of the FP64
    oracle on the whole lattice (about 1e7 cell updates on the host cores,
    a few seconds): normwise max |dQ| and max |df| within the FP32 bound,
    and the droplet radius and mass of the two runs."""
    import torch
    from paper_1907_13415_gb300 import nlc
    w = wl.sphere_256()
    sim = nlc.Simulation(w.lattice, w.shape, w.params, precision=nlc.NLC_FP32,
                         stream=torch.cuda.current_stream().cuda_stream)
    Q0 = w.initial_q5()
    sim.set_fields(Q0)
    sim.autotune(2)
    sim.step(STEPS)
    Q, _, _ = sim.get_fields()
    f = sim.get_populations()
    og = sim.observables()
    sim.close()
    p = wl.param_vector(w.params)
    fo, Qo = orc.step(w.lattice, p, orc.init_equilibrium(w.lattice, w.shape), Q0, STEPS)
    perm = perm_to_oracle(orc, w.lattice)
    tol = fp32_tolerance(STEPS)
    assert np.abs(Q - Qo).max() < tol * np.abs(Qo).max()
    del Q
    assert np.abs(f - fo[perm]).max() < tol * np.abs(fo).max()
    del f
    oo = orc.observables(w.lattice, p, fo, Qo)
    assert abs(og["radius"] - float(oo["radius"])) < 1e-6
    assert abs(og["mass"] - float(oo["mass"])) < 1e-9 * float(oo["mass"])
