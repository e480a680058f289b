"""The C-ABI library builds, loads without a GPU and exports every symbol
include/nlc.h declares; argument checks that need no device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "nlc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nlc_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("nlc_create", "nlc_step", "nlc_observables", "nlc_destroy",
              "nlc_set_fields", "nlc_get_fields", "nlc_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_1907_13415_gb300 import nlc
    lib = nlc.load()
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(nlc.exported_symbols()) >= set(declared_symbols())


def test_lattice_tables_without_gpu():
    from paper_1907_13415_gb300 import nlc
    import numpy as np
    for lat, q in ((nlc.NLC_D2Q9, 9), (nlc.NLC_D3Q19, 19)):
        c, w = nlc.nlc_lattice_velocities(lat)
        assert len(w) == q and abs(w.sum() - 1) < 1e-15
        assert np.allclose(w @ c, 0)
    assert nlc.load().nlc_lattice_velocities(5, None, None) == -1
    assert "sm_103a" in nlc.nlc_version()


def test_create_rejects_bad_arguments_before_touching_the_device():
    from paper_1907_13415_gb300 import nlc
    good = dict(A0=0.1, K=0.02, gamma=2.7, Gamma=0.3, xi=0.7, tau=1.0)
    bad_cases = [
        ((0, 8, 1, nlc.NLC_D2Q9, 0), good),
        ((8, 8, 2, nlc.NLC_D2Q9, 0), good),
        ((8, 8, 1, 7, 0), good),
        ((8, 8, 1, nlc.NLC_D2Q9, 9), good),
        ((8, 8, 1, nlc.NLC_D2Q9, 0), dict(good, tau=0.5)),
        ((8, 8, 1, nlc.NLC_D2Q9, 0), dict(good, gamma=float("nan"))),
    ]
    for g, p in bad_cases:
        grid = nlc.nlc_grid(*g)
        par = nlc.nlc_params(p["A0"], p["K"], p["gamma"], p["Gamma"], p["xi"],
                             p["tau"], 1.0)
        with pytest.raises(nlc.NlcError) as ei:
            nlc.nlc_create(grid, par)
        assert ei.value.status == -1
    lib = nlc.load()
    assert lib.nlc_step(None, 1) == -1
    assert lib.nlc_last_error(None) == b"context is NULL"
    lib.nlc_destroy(None)
