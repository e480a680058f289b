"""Parity at the full size the bench measures: the 256^3 D3Q19 spherical
droplet in FP32, in the bench's launch configuration (the chunk list the
autotuner picks), two steps.

The oracle cannot step the whole lattice in seconds, so it checks sampled
cells one by one: one step at a cell depends only on inputs within four
cells (Q) and three cells (populations), so two steps of the oracle on a
periodic 19^3 box cut around a cell give that cell's exact result at the box
centre.  Samples sit on the droplet interface, in the bulk inside and
outside, on every lattice face (periodic wrap), and on tile and z-chunk
boundaries.  Properties that hold at any size are checked over the whole
lattice: mass is conserved and the total momentum stays zero (the force is
the divergence of the stress, which sums to zero on a periodic lattice).
"""
import numpy as np
import pytest

from paper_1907_13415_gb300 import workloads as wl

from helpers import fp32_tolerance, perm_to_oracle

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


def test_sampled_cells_match_oracle_at_full_size(orc):
    import torch
    from paper_1907_13415_gb300 import nlc
    w = wl.sphere_256()
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
