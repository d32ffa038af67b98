"""gmres_solve_noalloc, called through the C ABI, against gmres_solve on the same handle.

gmres_solve_noalloc serves callers that must not allocate once set up (a real-time loop
with a frozen memory budget, or a process whose device memory is owned by a framework's
caching allocator): its workspace lives in a static 32 MiB device array of the library
instead of handle-owned allocations.  This file is collected after the parity files on
purpose, so that a run stopping at the first failure has already run them; it also passes
on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from helpers import relerr, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_04051_gb300 import _native as N
    from paper_1906_04051_gb300 import build as B
    B.build()
    return N


def _handle(N, orc, p, **opts):
    import paper_1906_04051_gb300 as G
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    s = G.Solver(to_dev(A.rowptr), to_dev(A.col), to_dev(A.val), to_dev(p.agg), p.r, **opts)
    return s, to_dev(b)


def _call(N, fn, s, b, m, tol, maxit, x=None):
    x = torch.empty_like(b) if x is None else x
    info = N.gmres_info()
    st = getattr(N.load(), fn)(s.handle, b.data_ptr(), None, m, tol, maxit, x.data_ptr(),
                               C.byref(info))
    torch.cuda.synchronize()
    return st, x.cpu().numpy(), info.as_dict()


@pytest.mark.parametrize("prec,dmode", [(0, 0), (1, 0), (2, 0), (0, 1)])
def test_noalloc_matches_gmres_solve_twice(lib, orc, prec, dmode):
    # precision 0/1/2: FP64, FP32 inner, BF16 basis; deflation 0/1: EBP, projector
    N = lib
    p = W.workload1()
    s, b = _handle(N, orc, p, precision=prec, deflation_mode=dmode)
    tol = 1e-12 if prec == 0 else 1e-10
    st_ref, x_ref, i_ref = _call(N, "gmres_solve", s, b, 30, tol, 20000)
    assert st_ref == 0
    xd = torch.empty_like(b)
    torch.cuda.synchronize()
    for call in range(2):  # two calls in a row share (and reuse) the static scratch
        free0 = torch.cuda.mem_get_info()[0]
        st, x, info = _call(N, "gmres_solve_noalloc", s, b, 30, tol, 20000, xd)
        free1 = torch.cuda.mem_get_info()[0]
        assert st == 0, N.load().gmres_last_error(s.handle)
        assert info["iters"] == i_ref["iters"]
        assert relerr(x, x_ref) <= 1e-9
        assert info["rel_res_true"] <= tol
        if call == 1:  # the call itself took no device memory (x is allocated before it)
            assert free1 == free0
    s.close()


def test_noalloc_rejects_workspace_beyond_the_static_scratch(lib, orc):
    N = lib
    p = W.convdiff(512, pe=20.0, sigma=0.3, seed=5, px=2, py=4)
    s, b = _handle(N, orc, p)
    st, _, _ = _call(N, "gmres_solve_noalloc", s, b, 50, 1e-8, 10)
    assert st == N.GMRES_ERR_INVALID_ARG
    assert b"static scratch" in N.load().gmres_last_error(s.handle)
    s.close()
