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


def test_q2_nnz_closed_form_matches_the_oracle_count(lib, orc):
    # the library's closed form (also the row pointer of the device assembly) against the
    # oracle's row-by-row count, including Table 1's sizes
    from paper_1906_04051_gb300 import _native as N
    L = N.load()
    assert L.q2_nnz(0) == 0
    for n in list(range(1, 41)) + [45, 50, 55, 60]:
        assert L.q2_nnz(n) == orc.q2_nnz(n), n
    for n in (1, 2, 7, 64, 255, 1024, 2048):
        assert L.q1_nnz(n) == orc.q1_nnz(n), n


def test_option_validation_before_device_work(lib):
    from paper_1906_04051_gb300 import _native as N
    L = N.load()
    o = N.gmres_opts()
    L.gmres_opts_default(ctypes.byref(o))
    assert (o.rmax, o.ninv, o.ortho) == (20, 20, N.ORTHO_CGS2)
    csr = N.gmres_csr(4, 4, 1, 1, 1)  # non-null placeholders: never dereferenced here
    h = ctypes.c_void_p()

    def create(**kw):
        oo = N.gmres_opts()
        L.gmres_opts_default(ctypes.byref(oo))
        for k, v in kw.items():
            setattr(oo, k, v)
        return L.gmres_create(ctypes.byref(h), ctypes.byref(csr), None, ctypes.byref(oo), None)

    bad = [dict(precision=3), dict(deflation_mode=4), dict(mu_mode=3), dict(ortho=3),
           dict(ortho=N.ORTHO_MGS, precision=N.FP32_INNER),
           dict(ortho=N.ORTHO_MGS_LOWSYNC, precision=N.BF16_BASIS),
           dict(deflation_mode=N.DEFL_ADAPTIVE, precision=N.FP32_INNER),
           dict(deflation_mode=N.DEFL_ADAPTIVE, rmax=0),
           dict(deflation_mode=N.DEFL_ADAPTIVE, rmax=33),
           dict(deflation_mode=N.DEFL_ADAPTIVE, ninv=0)]
    for kw in bad:
        assert create(**kw) == N.GMRES_ERR_INVALID_ARG, kw
        assert L.gmres_last_error(None), kw
    # W given both as aggregates and as dense columns, or with too many dense columns
    for defl in (N.gmres_defl(2, 1, 1), N.gmres_defl(33, None, 1)):
        assert L.gmres_create(ctypes.byref(h), ctypes.byref(csr), ctypes.byref(defl), None,
                              None) == N.GMRES_ERR_INVALID_ARG


def test_assembly_and_batch_validation_before_device_work(lib):
    # every call here is refused on the host, before any CUDA call: the placeholder
    # pointers (1) are never dereferenced
    from paper_1906_04051_gb300 import _native as N
    L = N.load()
    E = N.GMRES_ERR_INVALID_ARG
    nan = float("nan")
    assert L.q1_assemble(0, 1, 0.0, 0.0, 1, None, 1, 1, 1, 1, None) == E
    assert L.q1_assemble(8, None, 0.0, 0.0, 1, None, 1, 1, 1, 1, None) == E
    assert L.q1_assemble(50000, 1, 0.0, 0.0, 1, None, 1, 1, 1, 1, None) == E  # nnz >= 2^31
    assert b"int32" in L.gmres_last_error(None)
    assert L.q1_kappa_grad(0, 1, 1, 1, None) == E
    assert L.q2_bratu_assemble(0, 6.8, None, 1, 1, 1, 1, None) == E
    assert L.q2_bratu_assemble(2, 6.8, None, None, 1, 1, 1, None) == E
    assert L.q2_bratu_assemble(2, nan, None, 1, 1, 1, 1, None) == E
    assert b"lambda" in L.gmres_last_error(None)
    # n = 162 is the first mesh whose nnz overflows int32 (N = 325^3 still fits)
    assert L.q2_nnz(161) < 2 ** 31 <= L.q2_nnz(162)
    assert L.q2_bratu_assemble(162, 6.8, None, 1, 1, 1, 1, None) == E
    info = N.q2_newton_info()
    assert L.q2_bratu_newton(0, 6.8, None, None, 50, 1e-8, 100, 1e-9, 10, 1,
                             ctypes.byref(info), None) == E
    assert L.q2_bratu_newton(4, 6.8, None, None, 50, 1e-8, 100, 1e-9, 0, 1,
                             ctypes.byref(info), None) == E
    assert L.q2_bratu_newton(4, 6.8, None, None, 50, 1e-8, 100, nan, 10, 1,
                             ctypes.byref(info), None) == E
    assert L.q2_bratu_newton(162, 6.8, None, None, 50, 1e-8, 100, 1e-9, 10, 1,
                             ctypes.byref(info), None) == E
    # batched solve: an empty batch is a no-op; a negative count or null arrays are refused
    assert L.gmres_batch_solve(0, None, None, None, 30, 1e-8, 10, None, None, None) == N.GMRES_OK
    assert L.gmres_batch_solve(-1, None, None, None, 30, 1e-8, 10, None, None, None) == E
    assert L.gmres_batch_solve(2, None, None, None, 30, 1e-8, 10, None, None, None) == E
    # handle-less queries
    lay = N.gmres_layout()
    assert L.gmres_layout_query(None, ctypes.byref(lay)) == E
    q = ctypes.c_int32()
    assert L.gmres_adaptive_space(None, ctypes.byref(q), None, 0, None) == E
    assert L.gmres_profile(None, 1, 0, None, None) == E
