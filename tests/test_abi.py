"""The C-ABI library builds, loads, and exports every entry point that
include/dwf.h declares (no GPU needed: nothing here launches a kernel)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dwf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dwf_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2203_17119_gb300 import build
    if not os.path.exists(build.LIB):
        try:
            build.build()
        except RuntimeError as e:   # no CUDA toolkit in this environment
            pytest.skip(str(e))
    return build.LIB


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ("dwf_dslash_eo", "dwf_mooee", "dwf_mooee_inv", "dwf_dirichlet_block",
              "dwf_cgne_solve", "dwf_mpc", "dwf_create", "dwf_set_gauge"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(libpath):
    from paper_2203_17119_gb300 import dwf
    L = dwf.lib()
    for n in declared_functions():
        assert getattr(L, n).restype is not None


def test_argument_errors_without_gpu(libpath):
    """Argument checks fire before any CUDA call."""
    from paper_2203_17119_gb300 import dwf
    L = dwf.lib()
    h = ctypes.c_void_p()
    p = dwf.Params((ctypes.c_int * 4)(3, 4, 4, 4), 8, 1.8, 0.01, 1.0, 0.0)   # Lx odd
    assert L.dwf_create(ctypes.byref(h), ctypes.byref(p), None, 0, 1) == 1
    assert b"even" in L.dwf_last_error()
    p = dwf.Params((ctypes.c_int * 4)(4, 4, 4, 4), 7, 1.8, 0.01, 1.0, 0.0)   # Ls odd
    assert L.dwf_create(ctypes.byref(h), ctypes.byref(p), None, 0, 1) == 1
    assert L.dwf_mpc(None, None, None, 0, 0, 1, None) == 1


def declared_arity():
    """dwf_* prototype -> number of parameters, parsed from include/dwf.h."""
    text = open(os.path.join(ROOT, "include", "dwf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(dwf_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_matches_every_prototype():
    """The ctypes binding declares every entry point of the header with the
    header's number of arguments (a mismatch would corrupt a call silently)."""
    pytest.importorskip("torch")
    from paper_2203_17119_gb300 import dwf as G
    arity = declared_arity()
    sig = G.signatures()
    missing = sorted(set(arity) - set(sig) - {"dwf_last_error"})
    assert not missing, missing
    wrong = {n: (len(a), arity[n]) for n, a in sig.items() if len(a) != arity.get(n, -1)}
    assert not wrong, wrong


def test_release_build_has_no_debug_checks(libpath):
    """The release library reports itself as such; dwf_check_range is the
    debug build's alone."""
    from paper_2203_17119_gb300 import dwf
    L = dwf.lib()
    on = ctypes.c_int(-1)
    assert L.dwf_debug_build(ctypes.byref(on)) == 0 and on.value == 0
    assert L.dwf_check_range(None, 8) == 6          # DWF_ERR_UNSUPPORTED
