"""FP64 CPU oracle of the hybrid LB / Beris-Edwards step (arxiv 1907.13415).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the product path never imports it.  The C source
(`nlc_oracle.c`) follows the paper's Eqs. 1-6 cell by cell; this module is a
ctypes wrapper over it working on numpy arrays.

Array layouts (x fastest):
  f   (q, nz, ny, nx)   pre-collision populations at time n
  Q5  (5, nz, ny, nx)   Q components (xx, xy, xz, yy, yz); Qzz = -Qxx - Qyy
  params: (A0, K, gamma, Gamma, xi, tau)
"""
from .oracle import (D2Q9, D3Q19, Oracle, PARAM_NAMES, get, nvel)  # noqa: F401
