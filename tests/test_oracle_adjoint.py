"""Pins for the oracle's adjoint pieces: the transpose solve and dL/dkappa_e.

The element gradient is checked against a dense adjoint whose dA/dkappa_e comes from
re-assembling with kappa + e_e (A is affine in kappa, so that difference is exact up to
rounding), and against central finite differences of L(kappa) = ||x(kappa) - x_t||^2.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W


def _setup(orc, n=16):
    p, kstar = W.workload5(n)
    A, b = orc.q1_assemble(n, p.kappa, p.beta, p.f)
    At, _ = orc.q1_assemble(n, kstar, p.beta, p.f)
    xt = spla.spsolve(At.to_scipy().tocsc(), b)
    return p, A, b, xt


def test_dense_adjoint_gradient(orc):
    n = 16
    p, A, b, xt = _setup(orc, n)
    Ad = A.to_scipy().toarray()
    x = np.linalg.solve(Ad, b)
    lam = np.linalg.solve(Ad.T, 2.0 * (x - xt))
    ref = np.empty(n * n)
    for e in range(n * n):
        kp = p.kappa.copy()
        kp[e] += 1.0
        Ae, be = orc.q1_assemble(n, kp, p.beta, p.f)
        assert np.array_equal(be, b)  # the load does not depend on kappa
        dA = Ae.to_scipy().toarray() - Ad
        ref[e] = -lam @ (dA @ x)
    got = orc.q1_kappa_grad(n, lam, x)
    np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-12 * np.abs(ref).max())


def test_adjoint_gmres_and_finite_differences(orc):
    n = 16
    p, A, b, xt = _setup(orc, n)
    defl = orc.Deflation(A, p.agg, p.r)
    x, info = orc.gmres(A, b, m=50, tol=1e-13, maxit=5000, defl=defl)
    assert info["status"] == 0
    At = A.transpose()
    dT = orc.Deflation(At, p.agg, p.r)
    np.testing.assert_allclose(dT.T(), defl.T().T, rtol=1e-14, atol=1e-15)
    g = 2.0 * (x - xt)
    lam, info_t = orc.gmres(At, g, m=50, tol=1e-13, maxit=5000, defl=dT)
    assert info_t["status"] == 0
    grad = orc.q1_kappa_grad(n, lam, x)
    rng = np.random.default_rng(20)
    elems = rng.choice(n * n, 16, replace=False)
    h = 1e-6

    def loss(kappa):
        Ak, bk = orc.q1_assemble(n, kappa, p.beta, p.f)
        dk = orc.Deflation(Ak, p.agg, p.r)
        xk, ik = orc.gmres(Ak, bk, m=50, tol=1e-13, maxit=5000, defl=dk)
        assert ik["status"] == 0
        return float(np.sum((xk - xt) ** 2))

    for e in elems:
        kp, km = p.kappa.copy(), p.kappa.copy()
        kp[e] += h
        km[e] -= h
        fd = (loss(kp) - loss(km)) / (2 * h)
        assert abs(fd - grad[e]) <= 1e-5 * max(abs(grad[e]), 1e-3 * np.abs(grad).max())
