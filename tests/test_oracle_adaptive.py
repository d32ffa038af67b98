"""Pins of the oracle's adaptive deflation (Sec. 3.3, Eq. 19): the inverse power method
on the Hessenberg matrix against numpy's eigen-decomposition, the drop step at r_max
against scipy's left eigenvectors and the remaining spectrum, and the adaptive GMRES
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
    q = info["q"]
    assert 1 <= q <= 3 and U.shape == (A.n, q)  # a complex pair leaves two at once
    assert np.abs(U.T @ U - np.eye(q)).max() < 1e-12
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-7


@pytest.mark.parametrize("mu_mode", [orc.MU_USER, orc.MU_NORM_INF])
def test_adaptive_with_given_mu(mu_mode):
    p, A, b = _problem()
    xd = spla.spsolve(A.to_scipy().tocsc(), b)
    x, info = orc.gmres(A, b, m=30, tol=1e-10, maxit=20000, defl_mode=orc.DEFL_ADAPTIVE,
                        mu_mode=mu_mode, mu_user=6.0)
    assert info["status"] == 0
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-7


def _with_spectrum(rng, blocks):
    """A general (nonsymmetric) matrix S D S^-1 with D block diagonal as given."""
    q = sum(b.shape[0] for b in blocks)
    D = np.zeros((q, q))
    i = 0
    for b in blocks:
        k = b.shape[0]
        D[i:i + k, i:i + k] = b
        i += k
    S = rng.standard_normal((q, q)) + 3.0 * np.eye(q)
    return S @ D @ np.linalg.inv(S)


def _check_drop(T, p_expected):
    import scipy.linalg as sla
    q = T.shape[0]
    Qc, Tn, p = orc.adapt_drop(T)
    assert p == p_expected and Qc.shape == (q, q - p) and Tn.shape == (q - p, q - p)
    assert np.abs(Qc.T @ Qc - np.eye(q - p)).max() <= 1e-13
    # orthogonal to the left eigenvector of the largest-modulus eigenvalue (scipy, LAPACK)
    lam, YL = sla.eig(T, left=True, right=False)
    i = int(np.argmax(np.abs(lam)))
    y = YL[:, i] / np.linalg.norm(YL[:, i])
    assert np.abs(y.conj() @ Qc).max() <= 1e-10
    # the complement is T-invariant: T Qc = Qc Tn, and Tn = Qc^T T Qc
    assert np.abs(T @ Qc - Qc @ Tn).max() <= 1e-10 * np.abs(T).max()
    assert np.abs(Tn - Qc.T @ T @ Qc).max() <= 1e-12 * np.abs(T).max()
    # Tn keeps every eigenvalue but the dropped one (pair)
    keep = [j for j in range(q) if abs(abs(lam[j]) - abs(lam[i])) > 1e-9 * abs(lam[i])]
    got = np.sort_complex(np.linalg.eigvals(Tn)) if q > p else np.zeros(0)
    assert np.allclose(got, np.sort_complex(lam[keep]), rtol=1e-8, atol=1e-10)


def test_drop_real_dominant_eigenvalue():
    rng = np.random.default_rng(21)
    T = _with_spectrum(rng, [np.diag([0.01, -0.02, 0.05, 0.3, 0.7]), np.array([[2.5]])])
    _check_drop(T, 1)


def test_drop_complex_dominant_pair():
    rng = np.random.default_rng(22)
    T = _with_spectrum(rng, [np.diag([0.01, 0.04, -0.2, 0.6]),
                             np.array([[1.0, 2.0], [-2.0, 1.0]])])  # 1 +- 2i dominant
    _check_drop(T, 2)


def test_drop_random_nonsymmetric():
    rng = np.random.default_rng(23)
    for q in (2, 5, 12, 20, 32):
        T = rng.standard_normal((q, q))
        lam = np.linalg.eigvals(T)
        i = int(np.argmax(np.abs(lam)))
        _check_drop(T, 2 if abs(lam[i].imag) > 0 else 1)


def test_drop_one_by_one():
    Qc, Tn, p = orc.adapt_drop(np.array([[3.0]]))
    assert p == 1 and Qc.shape == (1, 0) and Tn.shape == (0, 0)
