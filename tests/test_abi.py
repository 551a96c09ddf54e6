"""The C ABI library builds, loads and exports every entry point declared in include/pfmm.h;
argument validation needs no GPU (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2106_15911_gb300.pfmm as P
from paper_2106_15911_gb300.inputs import cube_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pfmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pfmm_[A-Za-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported_and_bound():
    L = P.lib()
    names = _declared()
    assert "pfmm_build_trees" in names and "pfmm_apply_V" in names and "pfmm_apply_K" in names
    for n in names:
        assert hasattr(L, n), n
        assert n in P.SIGNATURES, n


def test_default_params():
    p = P.pfmm_default_params()
    assert (p.m_t, p.m_x, p.c_st, p.n_tr, p.leaf_steps, p.precision) == (4, 4, 1.0, -1, 2, P.PFMM_FP64)


def test_invalid_arguments_are_rejected_before_any_device_work():
    L = P.lib()
    assert L.pfmm_build_trees(None, None, None, None) == -1
    assert L.pfmm_apply_V(None, None, None, 1, None) == -1
    assert L.pfmm_apply_K(None, None, None, 1, None) == -1
    assert L.pfmm_default_params(None) == -1
    assert L.pfmm_last_error()
    V, T = cube_mesh(2)
    for bad in ({"n_steps": 12}, {"n_steps": 0}, {"alpha": -1.0}):
        kw = dict(T=1.0, n_steps=16, alpha=1.0)
        kw.update(bad)
        with pytest.raises(P.PfmmError):
            P.pfmm_build_trees(V, T, kw["T"], kw["n_steps"], kw["alpha"], stream=0)
    Tbad = T.copy()
    Tbad[0, 0] = 10_000
    with pytest.raises(P.PfmmError, match="INVALID_ARG"):
        P.pfmm_build_trees(V, Tbad, 1.0, 16, stream=0)
    Vn = V.copy()
    Vn[3, 1] = np.nan
    with pytest.raises(P.PfmmError, match="NONFINITE"):
        P.pfmm_build_trees(Vn, T, 1.0, 16, stream=0)
