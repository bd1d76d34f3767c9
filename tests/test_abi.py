"""The C-ABI library loads and exports every entry point include/pmsp.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pmsp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pmsp_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2211_16266_gb300 as pm
    return pm


def test_header_declares_calls():
    names = _declared()
    for required in ("pmsp_create", "pmsp_destroy", "pmsp_densify", "pmsp_consistency_filter",
                     "pmsp_cost_map", "pmsp_halfsweep", "pmsp_last_error", "pmsp_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    assert set(_declared()) <= set(lib.C_SYMBOLS) | {"pmsp_default_params"}
    for n in _declared():
        assert callable(getattr(lib, n))


def test_default_params(lib):
    p = lib.pmsp_default_params()
    assert (p.patch_w, p.patch_stride, p.iterations, p.best_k, p.n_refine) == (11, 2, 8, 3, 6)
    assert abs(p.d_min - 0.3) < 1e-7 and abs(p.d_max - 10.0) < 1e-6
