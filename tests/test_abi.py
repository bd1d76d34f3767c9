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


def _zero_args(fn):
    """NULL for every pointer argument, 0 for every number."""
    out = []
    for t in fn.argtypes:
        if t in (ctypes.c_float, ctypes.c_double):
            out.append(0.0)
        elif t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64):
            out.append(0)
        else:
            out.append(None)
    return out


def test_every_call_refuses_a_null_context(lib):
    """The header's error convention at its simplest: a NULL context is PMSP_EINVAL from
    every call that takes one (no crash, no CUDA call), destroying NULL is a no-op, and
    the error text of a NULL context says so."""
    so = lib._lib
    skip = {"pmsp_create", "pmsp_destroy", "pmsp_last_error", "pmsp_default_params"}
    for name in _declared():
        if name in skip:
            continue
        fn = getattr(so, name)
        assert fn(*_zero_args(fn)) == lib.PMSP_EINVAL, name
    assert so.pmsp_destroy(None) == lib.PMSP_OK
    assert so.pmsp_last_error(None) == b"NULL context"
    assert so.pmsp_create(None, None) == lib.PMSP_EINVAL
    so.pmsp_default_params(None)  # ignored


def test_create_without_a_gpu_reports_a_cuda_error(lib):
    """With no usable GPU a context cannot be made: pmsp_create returns PMSP_ECUDA and
    leaves the handle NULL rather than failing later."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p(1)
    assert lib._lib.pmsp_create(ctypes.byref(h), None) == lib.PMSP_ECUDA
    assert h.value is None
