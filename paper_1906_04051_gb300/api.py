"""PyTorch-facing wrappers of the C ABI: device tensors in, device tensors out.

PyTorch provides device memory and the current CUDA stream; every arithmetic step runs in
the library's kernels.  Each call passes ``tensor.data_ptr()`` and
``torch.cuda.current_stream().cuda_stream`` straight to the corresponding C function.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _native as N


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check(status: int, handle=None):
    if status < 0:
        msg = N.load().gmres_last_error(handle)
        raise N.GmresError(status, msg.decode() if msg else "")
    return status


def _dev(t: torch.Tensor, dtype, name: str, n: int | None = None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} entries, got {t.numel()}")
    return t


class Solver:
    """Deflated restarted GMRES(m) on one CSR matrix (handle from gmres_create)."""

    def __init__(self, rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor,
                 agg: torch.Tensor | None = None, r: int = 0, *, precision=N.FP64,
                 deflation_mode=N.DEFL_EBP, mu_mode=N.MU_RITZ_FIRST_CYCLE, mu_user=0.0,
                 fixed_iterations=False, r0_norm_ref=0.0, timeout_ms=0, inner_tol=0.0,
                 profile=False, rmax=20, ninv=20, ortho=N.ORTHO_CGS2, w_dense=None,
                 dot_arith=N.DOT_FP64, stream=None):
        L = N.load()
        n = rowptr.numel() - 1
        _dev(rowptr, torch.int32, "rowptr")
        _dev(col, torch.int32, "col")
        _dev(val, torch.float64, "val", col.numel())
        self.n = n
        self.nnz = col.numel()
        self.device = rowptr.device
        csr = N.gmres_csr(n, self.nnz, rowptr.data_ptr(), col.data_ptr(), val.data_ptr())
        defl = None
        if agg is not None and r > 0:
            _dev(agg, torch.int32, "agg", n)
            defl = N.gmres_defl(int(r), agg.data_ptr(), None)
        if w_dense is not None:  # W as dense columns (n x r, any strides): a column-major copy
            if agg is not None and r > 0:
                raise ValueError("give W as aggregates or as dense columns, not both")
            if w_dense.dim() != 2 or w_dense.shape[0] != n:
                raise ValueError(f"w_dense must be n x r, n = {n}")
            self._wd = w_dense.to(torch.float64).t().contiguous()  # row c = column c of W
            _dev(self._wd, torch.float64, "w_dense")
            defl = N.gmres_defl(int(w_dense.shape[1]), None, self._wd.data_ptr())
        opts = N.gmres_opts()
        L.gmres_opts_default(C.byref(opts))
        opts.precision = int(precision)
        opts.deflation_mode = int(deflation_mode)
        opts.mu_mode = int(mu_mode)
        opts.mu_user = float(mu_user)
        opts.fixed_iterations = 1 if fixed_iterations else 0
        opts.r0_norm_ref = float(r0_norm_ref)
        opts.timeout_ms = int(timeout_ms)
        opts.inner_tol = float(inner_tol)
        opts.profile = 1 if profile else 0
        opts.rmax = int(rmax)
        opts.ninv = int(ninv)
        opts.ortho = int(ortho)
        opts.dot_arith = int(dot_arith)
        self._stream = stream
        h = C.c_void_p()
        st = L.gmres_create(C.byref(h), C.byref(csr), C.byref(defl) if defl else None,
                            C.byref(opts), _stream_ptr(stream))
        _check(st, None)
        self._h = h
        self.r = int(r) if (defl and w_dense is None) else 0
        self.precision = int(precision)

    @property
    def handle(self):
        return self._h

    def _set_stream(self):
        N.load().gmres_set_stream(self._h, _stream_ptr(self._stream))

    def solve(self, b: torch.Tensor, x0: torch.Tensor | None = None, *, m=30, tol=1e-8,
              maxit=10000, out: torch.Tensor | None = None):
        """Returns (x, info dict).  Raises GmresError on a negative status."""
        _dev(b, torch.float64, "b", self.n)
        if x0 is not None:
            _dev(x0, torch.float64, "x0", self.n)
        x = out if out is not None else torch.empty_like(b)
        _dev(x, torch.float64, "x", self.n)
        self._set_stream()
        info = N.gmres_info()
        st = N.load().gmres_solve(self._h, b.data_ptr(),
                                  x0.data_ptr() if x0 is not None else None, int(m),
                                  float(tol), int(maxit), x.data_ptr(), C.byref(info))
        _check(st, self._h)
        return x, info.as_dict()

    def adjoint_solve(self, g: torch.Tensor, lam0: torch.Tensor | None = None, *, m=30,
                      tol=1e-8, maxit=10000, out: torch.Tensor | None = None):
        """Solves A^T lam = g; returns (lam, info dict)."""
        _dev(g, torch.float64, "g", self.n)
        if lam0 is not None:
            _dev(lam0, torch.float64, "lam0", self.n)
        lam = out if out is not None else torch.empty_like(g)
        self._set_stream()
        info = N.gmres_info()
        st = N.load().gmres_adjoint_solve(self._h, g.data_ptr(),
                                          lam0.data_ptr() if lam0 is not None else None,
                                          int(m), float(tol), int(maxit), lam.data_ptr(),
                                          C.byref(info))
        _check(st, self._h)
        return lam, info.as_dict()

    def profile(self, enable=-1, reset=False):
        """Per-phase device ms and launch counts since the last reset (gmres_profile)."""
        ms = (C.c_double * len(N.PHASES))()
        nl = (C.c_int64 * len(N.PHASES))()
        _check(N.load().gmres_profile(self._h, int(enable), 1 if reset else 0, ms, nl), self._h)
        return {name: (ms[i], nl[i]) for i, name in enumerate(N.PHASES)}

    def layout(self) -> dict:
        """Device data layout chosen at create (gmres_layout_query)."""
        out = N.gmres_layout()
        _check(N.load().gmres_layout_query(self._h, C.byref(out)), self._h)
        return out.as_dict()

    def adaptive_space(self):
        """(U, T) of the adaptive deflation space left by the last solve: U (n x q,
        orthonormal columns), T = U^T A U (q x q); gmres_adaptive_space."""
        lib = N.load()
        q = C.c_int32()
        _check(lib.gmres_adaptive_space(self._h, C.byref(q), None, 0, None), self._h)
        U = torch.empty((q.value, self.n), dtype=torch.float64, device=self.device)
        T = torch.empty((q.value, q.value), dtype=torch.float64, device=self.device)
        if q.value:
            self._set_stream()
            _check(lib.gmres_adaptive_space(self._h, C.byref(q), U.data_ptr(), self.n,
                                            T.data_ptr()), self._h)
        return U.t(), T

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            N.load().gmres_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_solve(solvers, bs, x0s=None, *, m=30, tol=1e-8, maxit=10000, outs=None,
                stream=None):
    """Solves len(solvers) independent systems in one gmres_batch_solve call."""
    L = N.load()
    cnt = len(solvers)
    outs = outs if outs is not None else [torch.empty_like(b) for b in bs]
    H = (C.c_void_p * cnt)(*[s.handle for s in solvers])
    B = (C.c_void_p * cnt)(*[b.data_ptr() for b in bs])
    X = (C.c_void_p * cnt)(*[x.data_ptr() for x in outs])
    X0 = None
    if x0s is not None:
        X0 = (C.c_void_p * cnt)(*[x.data_ptr() if x is not None else None for x in x0s])
    infos = (N.gmres_info * cnt)()
    st = L.gmres_batch_solve(cnt, H, B, X0, int(m), float(tol), int(maxit), X, infos,
                             _stream_ptr(stream))
    _check(st, None)
    return outs, [i.as_dict() for i in infos], st


def q1_nnz(n: int) -> int:
    return int(N.load().q1_nnz(int(n)))


def q1_assemble(n: int, kappa: torch.Tensor, beta, f: torch.Tensor,
                u: torch.Tensor | None = None, stream=None):
    """Q1 Galerkin system on the device: returns (rowptr, col, val, b)."""
    L = N.load()
    NN = (n + 1) ** 2
    _dev(kappa, torch.float64, "kappa", n * n)
    _dev(f, torch.float64, "f", NN)
    if u is not None:
        _dev(u, torch.float64, "u", NN)
    dev = kappa.device
    nnz = q1_nnz(n)
    rowptr = torch.empty(NN + 1, dtype=torch.int32, device=dev)
    col = torch.empty(nnz, dtype=torch.int32, device=dev)
    val = torch.empty(nnz, dtype=torch.float64, device=dev)
    b = torch.empty(NN, dtype=torch.float64, device=dev)
    st = L.q1_assemble(int(n), kappa.data_ptr(), float(beta[0]), float(beta[1]), f.data_ptr(),
                       u.data_ptr() if u is not None else None, rowptr.data_ptr(),
                       col.data_ptr(), val.data_ptr(), b.data_ptr(), _stream_ptr(stream))
    _check(st, None)
    return rowptr, col, val, b


def q1_kappa_grad(n: int, lam: torch.Tensor, x: torch.Tensor, stream=None) -> torch.Tensor:
    L = N.load()
    NN = (n + 1) ** 2
    _dev(lam, torch.float64, "lam", NN)
    _dev(x, torch.float64, "x", NN)
    grad = torch.empty(n * n, dtype=torch.float64, device=lam.device)
    st = L.q1_kappa_grad(int(n), lam.data_ptr(), x.data_ptr(), grad.data_ptr(),
                         _stream_ptr(stream))
    _check(st, None)
    return grad


def q2_nnz(n: int) -> int:
    return int(N.load().q2_nnz(int(n)))


def q2_bratu_assemble(n: int, lam: float, u: torch.Tensor | None = None, *, device=None,
                      stream=None):
    """Newton system J(u) du = -R(u) of the 3-D Bratu problem on n^3 27-node hexahedra
    (Sec. 3.1) on the device: returns (rowptr, col, val, b)."""
    L = N.load()
    NN = (2 * n + 1) ** 3
    if u is not None:
        _dev(u, torch.float64, "u", NN)
        device = u.device
    dev = torch.device(device) if device is not None else torch.device("cuda")
    nnz = q2_nnz(n)
    rowptr = torch.empty(NN + 1, dtype=torch.int32, device=dev)
    col = torch.empty(nnz, dtype=torch.int32, device=dev)
    val = torch.empty(nnz, dtype=torch.float64, device=dev)
    b = torch.empty(NN, dtype=torch.float64, device=dev)
    st = L.q2_bratu_assemble(int(n), float(lam), u.data_ptr() if u is not None else None,
                             rowptr.data_ptr(), col.data_ptr(), val.data_ptr(), b.data_ptr(),
                             _stream_ptr(stream))
    _check(st, None)
    return rowptr, col, val, b


def bratu_newton(n: int, lam: float, u: torch.Tensor | None = None, *, m=50, tol=1e-8,
                 maxit=20000, newton_tol=1e-10, max_newton=30, agg: torch.Tensor | None = None,
                 r: int = 0, precision=N.FP64, deflation_mode=N.DEFL_ADAPTIVE,
                 mu_mode=N.MU_RITZ_FIRST_CYCLE, mu_user=0.0, rmax=20, ninv=20,
                 ortho=N.ORTHO_CGS2, device=None, stream=None):
    """Newton's method for the 3-D Bratu problem (q2_bratu_newton); u (device, updated in
    place; zeros when None).  Returns (u, info dict)."""
    L = N.load()
    NN = (2 * n + 1) ** 3
    if u is None:
        u = torch.zeros(NN, dtype=torch.float64,
                        device=torch.device(device) if device is not None else "cuda")
    _dev(u, torch.float64, "u", NN)
    opts = N.gmres_opts()
    L.gmres_opts_default(C.byref(opts))
    opts.precision = int(precision)
    opts.deflation_mode = int(deflation_mode)
    opts.mu_mode = int(mu_mode)
    opts.mu_user = float(mu_user)
    opts.rmax = int(rmax)
    opts.ninv = int(ninv)
    opts.ortho = int(ortho)
    defl = None
    if agg is not None and r > 0:
        _dev(agg, torch.int32, "agg", NN)
        defl = N.gmres_defl(int(r), agg.data_ptr(), None)
    info = N.q2_newton_info()
    st = L.q2_bratu_newton(int(n), float(lam), C.byref(opts), C.byref(defl) if defl else None,
                           int(m), float(tol), int(maxit), float(newton_tol), int(max_newton),
                           u.data_ptr(), C.byref(info), _stream_ptr(stream))
    _check(st, None)  # negative: an error; GMRES_NOT_CONVERGED is reported in info
    return u, info.as_dict()
