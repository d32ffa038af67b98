"""Pins of the oracle's adaptive deflation (Sec. 3.3, Eq. 19): the inverse power method
on the Hessenberg matrix against numpy's eigen-decomposition, and the adaptive GMRES
against a direct solve and the EBP identity U^T (A M^-1) U = |mu| I."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as orc
import workloads as W


def _hess(rng, k, diag):
    """Upper Hessenberg with prescribed spectrum: Q^T D Q reduced to Hessenberg form by
    scipy (an independent routine), D given by its diagonal (2x2 blocks allowed)."""
    import scipy.linalg as sla
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    A = Q @ diag @ Q.T
    return sla.hessenberg(A)


def test_invvec_real_smallest_matches_numpy():
    rng = np.random.default_rng(3)
    D = np.diag([0.05, 1.0, 2.0, -3.0, 4.0, 5.5, 7.0, 9.0])
    H = _hess(rng, 8, D)
    (z,) = orc.hess_invvec(H, ninv=30)
    w, V = np.linalg.eig(H)
    i = np.argmin(np.abs(w))
    v = np.real(V[:, i])
    v /= np.linalg.norm(v)
    assert abs(abs(z @ v) - 1.0) < 1e-10
    assert np.linalg.norm(H @ z - w[i].real * z) < 1e-10 * np.linalg.norm(H)
    assert z[np.argmax(np.abs(z))] > 0  # sign convention


def test_invvec_complex_pair_spans_invariant_subspace():
    rng = np.random.default_rng(4)
    D = np.zeros((7, 7))
    D[0:2, 0:2] = [[0.1, 0.3], [-0.3, 0.1]]  # eigenvalues 0.1 +- 0.3i (smallest modulus)
    D[2:, 2:] = np.diag([2.0, 3.0, -4.0, 5.0, 6.0])
    H = _hess(rng, 7, D)
    zs = orc.hess_invvec(H, ninv=30)
    assert len(zs) == 2
    Z = np.stack(zs, axis=1)
    assert np.abs(Z.T @ Z - np.eye(2)).max() < 1e-12
    B = Z.T @ H @ Z
    assert np.linalg.norm(H @ Z - Z @ B) < 1e-8 * np.linalg.norm(H)
    ev = np.sort_complex(np.linalg.eigvals(B))
    assert np.allclose(ev, np.sort_complex(np.array([0.1 - 0.3j, 0.1 + 0.3j])), atol=1e-8)


def test_invvec_one_by_one():
    (z,) = orc.hess_invvec(np.array([[2.5]]), ninv=5)
    assert z.tolist() == [1.0]


def _problem():
    p = W.workload1()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    return p, A, b


def test_adaptive_gmres_converges_to_direct_solution():
    p, A, b = _problem()
    xd = spla.spsolve(A.to_scipy().tocsc(), b)
    x, info, U = orc.gmres(A, b, m=30, tol=1e-11, maxit=20000,
                           defl_mode=orc.DEFL_ADAPTIVE, return_u=True)
    assert info["status"] == 0 and info["rel_res_true"] <= 1e-11
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-8
    # U grows by one or two vectors per cycle and stays orthonormal
    assert 1 <= info["q"] <= min(20, 2 * info["cycles"])
    assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 1e-12


def test_adaptive_deflation_identity_and_fewer_steps():
    p, A, b = _problem()
    x0, i0 = orc.gmres(A, b, m=30, tol=1e-10, maxit=20000, defl=None)
    x, info, U = orc.gmres(A, b, m=30, tol=1e-10, maxit=20000,
                           defl_mode=orc.DEFL_ADAPTIVE, return_u=True)
    assert info["iters"] < i0["iters"]
    # the EBP identity for the final U: U^T (A M^-1) U = |mu| I with T = U^T A U
    Ad = A.to_scipy().toarray()
    T = U.T @ Ad @ U
    mu = abs(info["mu"])
    Minv = np.eye(A.n) + U @ (mu * np.linalg.inv(T) - np.eye(U.shape[1])) @ U.T
    G = U.T @ Ad @ Minv @ U
    assert np.abs(G - mu * np.eye(U.shape[1])).max() <= 1e-9 * mu


def test_adaptive_truncation_at_rmax():
    p, A, b = _problem()
    xd = spla.spsolve(A.to_scipy().tocsc(), b)
    x, info, U = orc.gmres(A, b, m=12, tol=1e-10, maxit=20000,
                           defl_mode=orc.DEFL_ADAPTIVE, rmax=3, return_u=True)
    assert info["status"] == 0 and info["cycles"] > 3
    assert info["q"] == 3 and U.shape == (A.n, 3)
    assert np.abs(U.T @ U - np.eye(3)).max() < 1e-12
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-7


@pytest.mark.parametrize("mu_mode", [orc.MU_USER, orc.MU_NORM_INF])
def test_adaptive_with_given_mu(mu_mode):
    p, A, b = _problem()
    xd = spla.spsolve(A.to_scipy().tocsc(), b)
    x, info = orc.gmres(A, b, m=30, tol=1e-10, maxit=20000, defl_mode=orc.DEFL_ADAPTIVE,
                        mu_mode=mu_mode, mu_user=6.0)
    assert info["status"] == 0
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-7
