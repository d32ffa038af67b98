"""The C-ABI library builds, loads without a GPU and exports every function that
include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\([^;{]*\)\s*;", text):
            name = m.group(1)
            if name not in {"if", "while", "for", "return", "sizeof"}:
                names.add(name)
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1906_04051_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("gmres_create", "gmres_solve", "gmres_adjoint_solve", "gmres_batch_solve",
                     "gmres_destroy", "gmres_last_error", "q1_assemble", "q1_kappa_grad"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_1906_04051_gb300 import _native
    assert set(_declared_functions()) == set(_native.SIGNATURES)


def test_host_only_calls(lib):
    from paper_1906_04051_gb300 import _native as N
    L = N.load()
    assert L.q1_nnz(64) == 35977 and L.q1_nnz(0) == 0
    o = N.gmres_opts()
    L.gmres_opts_default(ctypes.byref(o))
    assert (o.precision, o.deflation_mode, o.mu_mode, o.fixed_iterations) == (0, 0, 0, 0)
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    assert L.gmres_create(ctypes.byref(h), None, None, None, None) == N.GMRES_ERR_INVALID_ARG
    assert b"null" in L.gmres_last_error(None)
    assert L.gmres_solve(None, None, None, 30, 1e-8, 10, None, None) == N.GMRES_ERR_INVALID_ARG
