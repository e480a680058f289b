"""Exact floating-point operation counts of the pointwise physics
(tests/flop_count.cu runs the library's templates on an op-counting scalar),
and the per-lattice-update total of one fused D3Q19 step assembled from them.
The stencil arithmetic is counted by hand from step_fused.cuh (noted inline).
CPU only."""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def counts(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = tmp_path / "flop_count"
    subprocess.check_call([gxx, "-O1", "-std=c++17", "-x", "c++",
                           os.path.join(HERE, "flop_count.cu"), "-o", str(exe)])
    return json.loads(subprocess.check_output([str(exe)]).decode())


def step_flops(c, d=3):
    """Algorithmic operations per lattice update of one D3Q19 step (each
    quantity once per cell; the fused kernels' ring recomputation excluded)."""
    q_stencil = 5 * (d + (2 * d - 1) + 2)        # d differences, Laplacian adds + 1 FMA
    force = d * (d + (d - 1) + 1)                  # differences, adds, the 1/2
    lb = q_stencil + c["H"] + c["Pi_3d"] + force + c["moments_d3q19"] + c["bgk_d3q19"]
    adv = 5 * (2 * (d - 1) + 1)                    # u . (2 dQ): FMAs + 1 multiply
    u_stencil = d * d                              # differences (2 G, exact)
    rhs = q_stencil + adv + u_stencil + c["R_from_adv"]
    be = 2 * rhs + 5 + 5 * 3                       # Q^P = Q + R; [Q + Q^P + R(Q^P)]/2
    return lb, be


def test_operation_counts(tmp_path):
    c = counts(tmp_path)
    # the molecular field, the stress and the co-rotation term in the ranges
    # their formulas imply (Eq. 3, Eq. 5, Eq. 1)
    assert 60 <= c["H"] <= 90
    assert 200 <= c["Pi_3d"] <= 260 and c["Pi_2d"] < c["Pi_3d"]
    assert 90 <= c["S"] <= 130
    # R from the advection term = H + S + the assembly with the projection
    assert c["R_from_adv"] == c["H"] + c["S"] + 25
    # MRT costs two transforms of the non-conserved moments on top of BGK
    assert c["mrt_d3q19"] > 2.5 * c["bgk_d3q19"]
    lb, be = step_flops(c)
    assert 1200 <= lb + be <= 1700
    print(json.dumps({"counts": c, "lb_per_lup": lb, "be_per_lup": be,
                      "step_per_lup": lb + be}))
