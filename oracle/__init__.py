"""FP64 CPU oracle for deflated restarted GMRES(m) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product library (``paper_1906_04051_gb300``) never
imports, links or calls it, and the two share no code: the oracle is a plain,
sequential C translation of the paper's steps (arXiv:1906.04051, Sec. 3.1-3.3),
compiled with gcc at ``-O2`` and loaded through ctypes.

Parity status of each routine (what pins it, see tests/test_oracle_*.py):
  q1_assemble      closed-form Q1 stencils, nnz counts, manufactured-solution order 2
  q2_bratu         the paper's Table 1 nnz and CSR bytes, element matrices vs exact 1-D
                   Kronecker forms (sympy), Jacobian vs finite differences of the
                   residual, Newton's quadratic convergence, the z-independence and
                   x/y symmetries of the discrete Bratu solution
  spmv, transpose  scipy.sparse products, <Ax,y> = <x,A^T y>
  lu               numpy.linalg.solve
  hessenberg_eigs  numpy.linalg.eigvals, companion matrices with known roots
  gmres            sparse direct solves, exact termination, monotone residual estimate,
                   estimate = true residual, MGS/CGS2 agreement
  arnoldi          Arnoldi relation and orthonormality checked with dense numpy algebra
  defl (EBP, P)    U^T (A M^-1) U = |mu| I, invariant-subspace eigenvalue shift, P A W = 0
  adaptive         hess_invvec vs numpy eigenvectors (real and complex smallest pairs);
                   adapt_drop vs scipy left eigenvectors and the remaining spectrum;
                   the adaptive solve vs a direct solve, U orthonormal, T = U^T A U
  kappa_grad       dense adjoint (numpy) and central finite differences
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CGS2, MGS = 0, 1
DEFL_NONE, DEFL_EBP, DEFL_PROJECTOR, DEFL_ADAPTIVE = 0, 1, 2, 3
MU_RITZ_FIRST_CYCLE, MU_USER, MU_NORM_INF = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math) into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class Opts(C.Structure):
    _fields_ = [
        ("m", C.c_int32),
        ("tol", C.c_double),
        ("maxit", C.c_int64),
        ("ortho", C.c_int32),
        ("defl_mode", C.c_int32),
        ("mu_mode", C.c_int32),
        ("mu_user", C.c_double),
        ("fixed_iterations", C.c_int32),
        ("r0_norm_ref", C.c_double),
        ("rmax", C.c_int32),
        ("ninv", C.c_int32),
        ("u_out", C.c_void_p),
        ("w_dense", C.c_void_p),
        ("w_cols", C.c_int32),
    ]


class Info(C.Structure):
    _fields_ = [
        ("iters", C.c_int64),
        ("cycles", C.c_int64),
        ("status", C.c_int32),
        ("rel_res_est", C.c_double),
        ("rel_res_true", C.c_double),
        ("mu", C.c_double),
        ("q", C.c_int32),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_P = C.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_q1_nnz.restype = C.c_int64
            L.orc_q1_nnz.argtypes = [C.c_int32]
            L.orc_q1_element.argtypes = [C.c_double, C.c_double, C.c_double, _P, _P, _P]
            L.orc_q1_assemble.argtypes = [C.c_int32, _P, C.c_double, C.c_double, _P, _P,
                                          _P, _P, _P, _P]
            L.orc_q1_kappa_grad.argtypes = [C.c_int32, _P, _P, _P]
            L.orc_spmv.argtypes = [C.c_int32, _P, _P, _P, _P, _P]
            L.orc_transpose.argtypes = [C.c_int32, _P, _P, _P, _P, _P, _P]
            L.orc_lu_factor.argtypes = [C.c_int32, _P, _P]
            L.orc_lu_solve.argtypes = [C.c_int32, _P, _P, _P]
            L.orc_hessenberg_eigs.argtypes = [C.c_int32, _P, _P, _P]
            L.orc_hess_invvec.argtypes = [C.c_int32, _P, C.c_int32, _P, _P]
            L.orc_adapt_drop.argtypes = [C.c_int32, _P, C.c_int32, _P, _P]
            L.orc_q2_nnz.restype = C.c_int64
            L.orc_q2_nnz.argtypes = [C.c_int32]
            L.orc_q2_element.argtypes = [C.c_double, C.c_double, _P, _P, _P]
            L.orc_q2_bratu_assemble.argtypes = [C.c_int32, C.c_double, _P, _P, _P, _P, _P]
            L.orc_defl_create.restype = _P
            L.orc_defl_create.argtypes = [C.c_int32, _P, _P, _P, C.c_int32, _P,
                                          C.POINTER(C.c_int)]
            L.orc_defl_destroy.argtypes = [_P]
            L.orc_defl_T.argtypes = [_P, _P]
            L.orc_defl_apply_Minv.argtypes = [_P, C.c_double, _P, _P]
            L.orc_defl_apply_P.argtypes = [_P, _P, _P]
            L.orc_gmres.argtypes = [C.c_int32, _P, _P, _P, _P, _P, _P, C.POINTER(Opts),
                                    _P, C.POINTER(Info), _P]
            L.orc_arnoldi.argtypes = [C.c_int32, _P, _P, _P, _P, C.c_int32, C.c_double,
                                      C.c_int32, _P, C.c_int32, _P, _P]
            _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


class CSR:
    """Host CSR matrix (int32 rowptr/col, float64 val), columns ascending per row."""

    def __init__(self, rowptr, col, val):
        self.rowptr = _i32(rowptr)
        self.col = _i32(col)
        self.val = _f64(val)
        self.n = len(self.rowptr) - 1

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def matvec(self, x) -> np.ndarray:
        x = _f64(x)
        y = np.empty(self.n)
        lib().orc_spmv(self.n, _p(self.rowptr), _p(self.col), _p(self.val), _p(x), _p(y))
        return y

    def transpose(self) -> "CSR":
        rt = np.empty(self.n + 1, np.int32)
        ct = np.empty(self.nnz, np.int32)
        vt = np.empty(self.nnz)
        lib().orc_transpose(self.n, _p(self.rowptr), _p(self.col), _p(self.val),
                            _p(rt), _p(ct), _p(vt))
        return CSR(rt, ct, vt)


def q1_nnz(n: int) -> int:
    return int(lib().orc_q1_nnz(n))


def q1_element(h: float, bx: float, by: float):
    K1, Cm, M = np.empty(16), np.empty(16), np.empty(16)
    lib().orc_q1_element(h, bx, by, _p(K1), _p(Cm), _p(M))
    return K1.reshape(4, 4), Cm.reshape(4, 4), M.reshape(4, 4)


def q1_assemble(n: int, kappa, beta, f, u=None):
    """Q1 Galerkin system on an n x n mesh: returns (CSR A, b)."""
    kappa = _f64(kappa).reshape(-1)
    f = _f64(f).reshape(-1)
    N = (n + 1) ** 2
    assert kappa.size == n * n and f.size == N
    uu = None if u is None else _f64(u).reshape(-1)
    nnz = q1_nnz(n)
    rowptr = np.empty(N + 1, np.int32)
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz)
    b = np.empty(N)
    lib().orc_q1_assemble(n, _p(kappa), float(beta[0]), float(beta[1]), _p(f), _p(uu),
                          _p(rowptr), _p(col), _p(val), _p(b))
    return CSR(rowptr, col, val), b


def q2_nnz(n: int) -> int:
    return int(lib().orc_q2_nnz(n))


def q2_element(h: float, lam: float, ue=None):
    """Element Jacobian (27 x 27) and residual (27) of the Q2 Bratu element."""
    Je = np.empty(27 * 27)
    Re = np.empty(27)
    uu = None if ue is None else _f64(ue).reshape(-1)
    lib().orc_q2_element(float(h), float(lam), _p(uu), _p(Je), _p(Re))
    return Je.reshape(27, 27), Re


def q2_bratu_assemble(n: int, lam: float, u=None):
    """Newton system of the 3-D Bratu problem on n^3 Q2 elements at u: (CSR J, b = -R)."""
    N = (2 * n + 1) ** 3
    uu = None if u is None else _f64(u).reshape(-1)
    assert uu is None or uu.size == N
    nnz = q2_nnz(n)
    rowptr = np.empty(N + 1, np.int32)
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz)
    b = np.empty(N)
    lib().orc_q2_bratu_assemble(n, float(lam), _p(uu), _p(rowptr), _p(col), _p(val), _p(b))
    return CSR(rowptr, col, val), b


def q1_kappa_grad(n: int, lam, x) -> np.ndarray:
    lam, x = _f64(lam), _f64(x)
    g = np.empty(n * n)
    lib().orc_q1_kappa_grad(n, _p(lam), _p(x), _p(g))
    return g


def lu_factor(a):
    a = _f64(a).copy()
    n = a.shape[0]
    piv = np.empty(n, np.int32)
    info = lib().orc_lu_factor(n, _p(a), _p(piv))
    return a, piv, info


def lu_solve(lu, piv, b) -> np.ndarray:
    b = _f64(b).copy()
    lib().orc_lu_solve(lu.shape[0], _p(lu), _p(piv), _p(b))
    return b


def hessenberg_eigs(h) -> np.ndarray:
    h = _f64(h)
    n = h.shape[0]
    wr, wi = np.empty(n), np.empty(n)
    rc = lib().orc_hessenberg_eigs(n, _p(h), _p(wr), _p(wi))
    if rc != 0:
        raise RuntimeError("Hessenberg QR did not converge")
    return wr + 1j * wi


class Deflation:
    """U = W diag(1/sqrt|agg_p|) for aggregate indicator columns W, T = U^T A U."""

    def __init__(self, A: CSR, agg, r: int):
        self.A = A
        self.agg = _i32(agg)
        self.r = int(r)
        err = C.c_int(0)
        self._h = lib().orc_defl_create(A.n, _p(A.rowptr), _p(A.col), _p(A.val), self.r,
                                        _p(self.agg), C.byref(err))
        if not self._h:
            raise ValueError(f"deflation setup failed (status {err.value})")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_defl_destroy(h)
            self._h = None

    def T(self) -> np.ndarray:
        T = np.empty(self.r * self.r)
        lib().orc_defl_T(self._h, _p(T))
        return T.reshape(self.r, self.r)

    def apply_Minv(self, mu: float, v) -> np.ndarray:
        v = _f64(v)
        z = np.empty_like(v)
        lib().orc_defl_apply_Minv(self._h, float(mu), _p(v), _p(z))
        return z

    def apply_P(self, w) -> np.ndarray:
        w = _f64(w)
        out = np.empty_like(w)
        lib().orc_defl_apply_P(self._h, _p(w), _p(out))
        return out


def gmres(A: CSR, b, x0=None, *, m=30, tol=1e-8, maxit=10000, defl: Deflation | None = None,
          defl_mode=DEFL_EBP, mu_mode=MU_RITZ_FIRST_CYCLE, mu_user=0.0, ortho=CGS2,
          fixed_iterations=False, r0_norm_ref=0.0, history=False, rmax=20, ninv=20,
          return_u=False, w_dense=None):
    """Deflated restarted GMRES(m); returns (x, info dict[, history (steps x 2)][, U]).

    defl_mode=DEFL_ADAPTIVE needs no Deflation object: U starts empty and grows after
    every cycle (Sec. 3.3, Eq. 19), at most rmax columns; return_u appends the final U
    (N x q).  w_dense (N x r): the deflation space as dense columns instead of aggregates
    (U = their orthonormalisation, the EBP preconditioner); a ValueError if a column lies
    in the span of the previous ones."""
    b = _f64(b)
    x0a = None if x0 is None else _f64(x0)
    x = np.empty(A.n)
    adaptive = defl_mode == DEFL_ADAPTIVE
    wd = None
    if w_dense is not None:
        wd = np.asfortranarray(np.asarray(w_dense, dtype=np.float64).reshape(A.n, -1))
    given = wd is not None and not adaptive
    uo = np.zeros(A.n * (wd.shape[1] if given else rmax)) if ((adaptive or given) and return_u) else None
    o = Opts(m, tol, maxit, ortho,
             defl_mode if (defl is not None or adaptive or given) else DEFL_NONE, mu_mode,
             mu_user, 1 if fixed_iterations else 0, r0_norm_ref, rmax, ninv,
             None if uo is None else uo.ctypes.data,
             None if wd is None else wd.ctypes.data, 0 if wd is None else wd.shape[1])
    info = Info()
    hist = np.zeros(2 * maxit) if history else None
    rc = lib().orc_gmres(A.n, _p(A.rowptr), _p(A.col), _p(A.val),
                         None if defl is None else defl._h, _p(b), _p(x0a), C.byref(o), _p(x),
                         C.byref(info), _p(hist))
    if given and rc == -1:
        raise ValueError("w_dense: a column lies in the span of the previous ones")
    out = (x, info.as_dict())
    if history:
        hs = hist.reshape(-1, 2)[: info.iters]
        out = out + (hs,)
    if uo is not None:
        out = out + (uo[: A.n * info.q].reshape(info.q, A.n).T.copy(),)
    return out


def hess_invvec(H, ninv=20):
    """Inverse power method on an upper Hessenberg H (Sec. 3.3): one vector, or two
    spanning a complex pair's invariant subspace."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    k = H.shape[0]
    z = np.zeros(2 * k)
    nv = lib().orc_hess_invvec(k, _p(H), ninv, _p(z), _p(z[k:]))
    return [z[i * k:(i + 1) * k].copy() for i in range(nv)]


def arnoldi(A: CSR, v0, k: int, *, defl: Deflation | None = None, defl_mode=DEFL_NONE,
            mu=0.0, ortho=CGS2):
    """k Arnoldi steps on A M^-1 (EBP), P A (projector) or A; returns (V, H, steps)."""
    v0 = _f64(v0)
    V = np.zeros((k + 1) * A.n)
    H = np.zeros((k + 1) * k)
    done = lib().orc_arnoldi(A.n, _p(A.rowptr), _p(A.col), _p(A.val),
                             None if defl is None else defl._h,
                             defl_mode if defl is not None else DEFL_NONE, float(mu), ortho,
                             _p(v0), k, _p(V), _p(H))
    return V.reshape(k + 1, A.n).T.copy(), H.reshape(k + 1, k), done


def adapt_drop(T):
    """Drop step of the adaptive deflation (Sec. 3.3) on a full space: returns (Qc, Tn,
    p) with Qc (q x (q-p)) an orthonormal basis of the complement of the left
    eigenvector(s) of T's largest-modulus eigenvalue and Tn = Qc^T T Qc."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    q = T.shape[0]
    Qc = np.zeros(q * q)
    Tn = np.zeros(q * q)
    p = lib().orc_adapt_drop(q, _p(T), q, _p(Qc), _p(Tn))
    if p < 0:
        raise RuntimeError("orc_adapt_drop: QR iteration failed")
    nc = q - p
    return Qc[: q * nc].reshape(q, nc).copy(), Tn[: nc * nc].reshape(nc, nc).copy(), p
