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


def test_create_refuses_an_unknown_scheduler(lib):
    """The serving scheduler is checked before any CUDA call: an unknown value is
    PMSP_EINVAL on any machine, and the handle stays NULL."""
    for bad in (2, -1, 7):
        h = ctypes.c_void_p(1)
        opts = lib.pmsp_ctx_opts(0, None, 0, 0, 0, bad)
        assert lib._lib.pmsp_create(ctypes.byref(h), ctypes.byref(opts)) == lib.PMSP_EINVAL
        assert h.value is None


STRUCTS = ("pmsp_image", "pmsp_pose", "pmsp_params", "pmsp_maps", "pmsp_ctx_opts", "pmsp_batch_item",
           "pmsp_tuning", "pmsp_request", "pmsp_serving_stats", "pmsp_peaks")


def test_binding_structs_match_the_header_layout(lib, tmp_path):
    """Every struct the binding marshals has the size and field offsets the C compiler
    gives the header's declaration (a field added, dropped or reordered on one side
    would pass garbage across the boundary)."""
    import subprocess
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pmsp.h"', 'int main(void) {']
    for s in STRUCTS:
        lines.append(f'    printf("{s} size %zu\\n", sizeof({s}));')
        for name, _ in getattr(lib, s)._fields_:
            lines.append(f'    printf("{s} {name} %zu\\n", offsetof({s}, {name}));')
    lines += ['    return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        s, name, value = line.split()
        got[(s, name)] = int(value)
    for s in STRUCTS:
        cls = getattr(lib, s)
        assert got[(s, "size")] == ctypes.sizeof(cls), s
        for name, _ in cls._fields_:
            assert got[(s, name)] == getattr(cls, name).offset, (s, name)


def test_binding_constants_match_the_header(lib, tmp_path):
    """Status codes, formats, memory kinds, flags and limits have the header's values."""
    import subprocess
    names = {n: n for n in ("PMSP_OK", "PMSP_EINVAL", "PMSP_ENOMEM", "PMSP_EADMIT", "PMSP_EBUSY", "PMSP_ETIMEDOUT",
                            "PMSP_ECUDA", "PMSP_EDEVICE", "PMSP_ENOTFOUND", "PMSP_U8", "PMSP_F16", "PMSP_F32",
                            "PMSP_HOST", "PMSP_DEVICE", "PMSP_BATCH_GRAPH", "PMSP_NOALLOC_MAX_ITEMS",
                            "PMSP_SCHED_LANES", "PMSP_SCHED_STEPS")}
    names["MAX_SOURCES"] = "PMSP_MAX_SOURCES"
    lines = ['#include <stdio.h>', '#include "pmsp.h"', 'int main(void) {']
    lines += [f'    printf("{py} %lld\\n", (long long)({c}));' for py, c in names.items()]
    lines += ['    return 0;', '}']
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        py, value = line.split()
        assert getattr(lib, py) == int(value), py


def _prototypes():
    """name -> list of parameter declarations, from the header's prototypes."""
    src = open(os.path.join(ROOT, "include", "pmsp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pmsp_\w+)\s*\(([^;]*?)\)\s*;", src, flags=re.M | re.S):
        params = " ".join(m.group(2).split())
        out[m.group(1)] = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
    return out


def test_binding_argument_lists_match_the_prototypes(lib):
    """Each call's binding passes as many arguments as the header's prototype declares,
    pointers where it declares pointers and numbers where it declares numbers."""
    protos = _prototypes()
    assert set(protos) == set(_declared())
    so = lib._lib
    for name, params in protos.items():
        fn = getattr(so, name)
        assert fn.argtypes is not None and len(fn.argtypes) == len(params), name
        for decl, t in zip(params, fn.argtypes):
            is_ptr = "*" in decl
            t_is_ptr = t is ctypes.c_void_p or t is ctypes.c_char_p or hasattr(t, "_type_") and \
                isinstance(t, type) and issubclass(t, ctypes._Pointer)
            assert is_ptr == t_is_ptr, (name, decl, t)


@pytest.mark.parametrize("lang,std", [("c", "c99"), ("c", "c11"), ("c++", "c++11"), ("c++", "c++17")])
def test_header_compiles_standalone(tmp_path, lang, std):
    """include/pmsp.h compiles on its own, warning-free, as C and as C++ (extern "C")."""
    import subprocess
    src = tmp_path / ("t.c" if lang == "c" else "t.cpp")
    src.write_text('#include "pmsp.h"\nint pmsp_header_check(void) { return PMSP_ABI_VERSION; }\n')
    cc = "gcc" if lang == "c" else "g++"
    subprocess.check_call([cc, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only",
                           "-I", os.path.join(ROOT, "include"), str(src)])
