"""Pins for the oracle's deflated restarted GMRES(m) (Sec. 3.2-3.3, Eqs. 10-18).

Each test fixes a property that the mathematics decides independently of the oracle:
agreement with a sparse direct solve, finite termination, the monotone residual estimate,
estimate = true residual under right preconditioning (Eq. 14), the Arnoldi relation
(Eq. 13) checked with dense numpy algebra, the exact eigenvalue shift of the deflation
preconditioner (Eq. 17), and the projector identity P A W = 0.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W


def _system(orc, n, pe=20.0, sigma=0.4, seed=11, px=2, py=2, f_kind="uniform"):
    p = W.convdiff(n, pe=pe, sigma=sigma, seed=seed, px=px, py=py, f_kind=f_kind)
    A, b = orc.q1_assemble(n, p.kappa, p.beta, p.f)
    return p, A, b


def _dense_U(agg, r):
    N = len(agg)
    U = np.zeros((N, r))
    for p in range(r):
        idx = np.nonzero(agg == p)[0]
        U[idx, p] = 1.0 / np.sqrt(len(idx))
    return U


MODES = [("none", None), ("ebp", 1), ("projector", 2)]


@pytest.mark.parametrize("n", [4, 8, 16])
@pytest.mark.parametrize("mode", ["none", "ebp", "projector"])
@pytest.mark.parametrize("ortho", [0, 1])
def test_gmres_matches_direct_solve(orc, n, mode, ortho):
    p, A, b = _system(orc, n)
    xd = spla.spsolve(A.to_scipy().tocsc(), b)
    defl = None if mode == "none" else orc.Deflation(A, p.agg, p.r)
    dm = {"none": 0, "ebp": 1, "projector": 2}[mode]
    x, info = orc.gmres(A, b, m=10, tol=1e-14, maxit=4000, defl=defl, defl_mode=dm, ortho=ortho)
    assert info["status"] == 0, info
    assert np.linalg.norm(x - xd) <= 1e-11 * np.linalg.norm(xd)
    assert info["rel_res_true"] <= 1e-13


@pytest.mark.parametrize("n", [4, 8])
def test_exact_termination_without_restart(orc, n):
    p, A, b = _system(orc, n)
    N = A.n
    x, info = orc.gmres(A, b, m=N, tol=1e-14, maxit=N)
    assert info["iters"] <= N and info["cycles"] == 1
    assert info["rel_res_true"] <= 1e-10


def test_diagonal_with_k_distinct_eigenvalues(orc):
    rng = np.random.default_rng(3)
    N, k = 60, 5
    d = rng.integers(1, k + 1, N).astype(float)
    assert len(np.unique(d)) == k
    A = orc.CSR(np.arange(N + 1), np.arange(N), d)
    b = rng.standard_normal(N)
    x, info = orc.gmres(A, b, m=20, tol=1e-12, maxit=100)
    assert info["iters"] == k
    np.testing.assert_allclose(x, b / d, rtol=1e-12)


def test_identity_one_step(orc):
    N = 17
    A = orc.CSR(np.arange(N + 1), np.arange(N), np.ones(N))
    b = np.arange(1.0, N + 1)
    x, info = orc.gmres(A, b, m=5, tol=1e-14, maxit=10)
    assert info["iters"] == 1 and info["status"] == 0
    np.testing.assert_allclose(x, b, rtol=1e-15)


def test_zero_rhs_returns_x0(orc):
    p, A, b = _system(orc, 6)
    x, info = orc.gmres(A, np.zeros(A.n), m=5)
    assert info["iters"] == 0 and info["status"] == 0 and not np.any(x)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_residual_estimate_monotone_within_cycles(orc, mode):
    p, A, b = _system(orc, 24, pe=60.0)
    defl = None if mode == 0 else orc.Deflation(A, p.agg, p.r)
    x, info, hist = orc.gmres(A, b, m=15, tol=1e-10, maxit=3000, defl=defl, defl_mode=mode,
                              history=True)
    assert info["status"] == 0
    for t in range(1, len(hist)):
        if hist[t, 0] > 0:  # same cycle as the previous step
            assert hist[t, 1] <= hist[t - 1, 1] * (1 + 1e-13)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_estimate_equals_true_residual(orc, mode):
    # right preconditioning keeps ||b - A x_k|| = |gamma_{k+1}| (Eq. 14)
    p, A, b = _system(orc, 20, pe=30.0)
    defl = None if mode == 0 else orc.Deflation(A, p.agg, p.r)
    for maxit in (7, 23, 61):
        x, info = orc.gmres(A, b, m=10, tol=0.0, maxit=maxit, defl=defl, defl_mode=mode,
                            fixed_iterations=True, mu_mode=1, mu_user=4.0)
        assert abs(info["rel_res_est"] - info["rel_res_true"]) <= 1e-10


@pytest.mark.parametrize("defl_mode", [0, 1, 2])
@pytest.mark.parametrize("ortho", [0, 1])
def test_arnoldi_relation_dense(orc, defl_mode, ortho):
    p, A, b = _system(orc, 12, pe=40.0, px=2, py=3)
    Ad = A.to_scipy().toarray()
    U = _dense_U(p.agg, p.r)
    mu = 5.5
    T = U.T @ Ad @ U
    if defl_mode == 1:
        Op = Ad @ (np.eye(A.n) + U @ (abs(mu) * np.linalg.inv(T) - np.eye(p.r)) @ U.T)
    elif defl_mode == 2:
        Op = (np.eye(A.n) - Ad @ U @ np.linalg.inv(T) @ U.T) @ Ad
    else:
        Op = Ad
    defl = orc.Deflation(A, p.agg, p.r)
    k = 25
    V, H, done = orc.arnoldi(A, b, k, defl=defl, defl_mode=defl_mode, mu=mu, ortho=ortho)
    assert done == k
    scale = np.linalg.norm(Op, 2)
    assert np.linalg.norm(Op @ V[:, :k] - V @ H) <= 1e-13 * scale * np.sqrt(k)
    # CGS2 keeps orthogonality at rounding level; MGS loses it in proportion to the
    # condition number of the Krylov basis, so only a loose bound applies to it
    tol = 1e-13 if ortho == 0 else 1e-7
    assert np.linalg.norm(V.T @ V - np.eye(k + 1)) <= tol
    assert np.allclose(np.tril(H, -2), 0.0)


def test_deflation_T_is_UtAU(orc):
    p, A, b = _system(orc, 10, px=3, py=2)
    U = _dense_U(p.agg, p.r)
    defl = orc.Deflation(A, p.agg, p.r)
    np.testing.assert_allclose(defl.T(), U.T @ A.to_scipy().toarray() @ U, rtol=1e-13,
                               atol=1e-14)


def test_ebp_moves_deflated_eigenvalues_to_mu(orc):
    # U^T (A M^-1) U = |mu| I for any orthonormal U (Eq. 17 with T = U^T A U)
    p, A, b = _system(orc, 10, px=2, py=2)
    defl = orc.Deflation(A, p.agg, p.r)
    U = _dense_U(p.agg, p.r)
    mu = -7.25
    AMU = np.stack([A.matvec(defl.apply_Minv(mu, U[:, q])) for q in range(p.r)], axis=1)
    np.testing.assert_allclose(U.T @ AMU, abs(mu) * np.eye(p.r), atol=1e-13 * abs(mu))


def test_ebp_exact_invariant_subspace(orc):
    # block-diagonal A whose blocks have constant row sums: the aggregate indicators span
    # an invariant subspace, so A M^-1 U = |mu| U and the other eigenvalues are unchanged
    rng = np.random.default_rng(7)
    r, s = 3, 5
    blocks, lam = [], []
    for q in range(r):
        B = rng.standard_normal((s, s)) * 0.3
        B += np.diag(2.0 + q - B.sum(axis=1))  # row sums equal 2 + q
        blocks.append(B)
        lam.append(2.0 + q)
    Ad = sp.block_diag(blocks).toarray()
    S = sp.csr_matrix(Ad)
    S.sort_indices()
    A = orc.CSR(S.indptr, S.indices, S.data)
    agg = np.repeat(np.arange(r), s).astype(np.int32)
    defl = orc.Deflation(A, agg, r)
    mu = 9.0
    Minv = np.stack([defl.apply_Minv(mu, e) for e in np.eye(r * s)], axis=1)
    ev = np.sort_complex(np.linalg.eigvals(Ad @ Minv))
    ref = list(np.linalg.eigvals(Ad))
    for l in lam:  # each block gives up its constant-vector eigenvalue
        j = int(np.argmin([abs(z - l) for z in ref]))
        ref[j] = mu
    np.testing.assert_allclose(np.sort_complex(np.array(ref)), ev, atol=1e-10)


def test_projector_identities(orc):
    p, A, b = _system(orc, 11, px=2, py=3)
    defl = orc.Deflation(A, p.agg, p.r)
    Wm = np.stack([(p.agg == q).astype(float) for q in range(p.r)], axis=1)
    AW = np.stack([A.matvec(Wm[:, q]) for q in range(p.r)], axis=1)
    PAW = np.stack([defl.apply_P(AW[:, q]) for q in range(p.r)], axis=1)
    assert np.linalg.norm(PAW) <= 1e-13 * np.linalg.norm(AW)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(A.n)
    Pv = defl.apply_P(v)
    assert np.linalg.norm(Wm.T @ Pv) <= 1e-12 * np.linalg.norm(v) * np.sqrt(A.n)
    np.testing.assert_allclose(defl.apply_P(Pv), Pv, atol=1e-12 * np.linalg.norm(v))


def test_empty_aggregate_is_rejected(orc):
    p, A, b = _system(orc, 6)
    agg = p.agg.copy()
    agg[agg == 1] = 0  # aggregate 1 now has no node: W has a zero column
    with pytest.raises(ValueError):
        orc.Deflation(A, agg, p.r)


def test_deflation_reduces_steps_on_workload1(orc):
    p = W.workload1()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    defl = orc.Deflation(A, p.agg, p.r)
    _, i_defl = orc.gmres(A, b, m=30, tol=1e-8, maxit=5000, defl=defl)
    _, i_none = orc.gmres(A, b, m=30, tol=1e-8, maxit=5000)
    assert i_defl["status"] == 0 and i_none["status"] == 0
    assert i_defl["iters"] <= i_none["iters"]


def test_mgs_and_cgs2_agree_at_fixed_iterations(orc):
    p, A, b = _system(orc, 32, pe=50.0, px=4, py=4)
    defl = orc.Deflation(A, p.agg, p.r)
    kw = dict(m=20, tol=0.0, maxit=100, defl=defl, fixed_iterations=True, mu_mode=1,
              mu_user=6.0)
    x1, _ = orc.gmres(A, b, ortho=0, **kw)
    x2, _ = orc.gmres(A, b, ortho=1, **kw)
    assert np.linalg.norm(x1 - x2) <= 1e-10 * np.linalg.norm(x1)


def test_ritz_mu_is_spectral_radius_estimate(orc):
    # Ritz values lie in the field of values, so |mu| <= ||A||_2, and with a long first
    # cycle |mu| approaches the spectral radius
    p, A, b = _system(orc, 10, pe=5.0)
    Ad = A.to_scipy().toarray()
    rho = np.abs(np.linalg.eigvals(Ad)).max()
    norm2 = np.linalg.norm(Ad, 2)
    defl = orc.Deflation(A, p.agg, p.r)
    mus = []
    for m in (5, 20, 60):
        _, info = orc.gmres(A, b, m=m, tol=1e-30, maxit=m + 1, defl=defl)
        mus.append(info["mu"])
    assert all(mu <= norm2 * (1 + 1e-12) for mu in mus)
    assert abs(mus[-1] - rho) <= 0.02 * rho


def test_maxit_reports_not_converged(orc):
    p, A, b = _system(orc, 16)
    x, info = orc.gmres(A, b, m=5, tol=1e-14, maxit=12)
    assert info["status"] == 1 and info["iters"] == 12


# ---- a deflation space given as dense columns (Eqs. 16-18 with U = orth(W)) -----------
def _dense_problem(orc):
    p = W.workload1()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    return p, A, b


def test_dense_w_of_aggregate_indicators_equals_ebp(orc):
    p, A, b = _dense_problem(orc)
    Wd = np.zeros((A.n, p.r))
    Wd[np.arange(A.n), p.agg] = 1.0  # indicator columns (unnormalised: the oracle orthonormalises)
    d = orc.Deflation(A, p.agg, p.r)
    x1, i1 = orc.gmres(A, b, m=30, tol=1e-10, maxit=20000, defl=d)
    x2, i2 = orc.gmres(A, b, m=30, tol=1e-10, maxit=20000, w_dense=Wd)
    assert i1["status"] == 0 and i2["status"] == 0
    assert i1["iters"] == i2["iters"]
    assert np.linalg.norm(x1 - x2) <= 1e-10 * np.linalg.norm(x1)
    assert i2["mu"] == pytest.approx(i1["mu"], rel=1e-12)


def test_dense_w_result_depends_only_on_its_span(orc):
    # W and W R (R invertible) span the same space: the same M^-1, the same iterates
    p, A, b = _dense_problem(orc)
    rng = np.random.default_rng(12)
    Wd = rng.standard_normal((A.n, 6))
    R = rng.standard_normal((6, 6)) + 3 * np.eye(6)
    kw = dict(m=20, tol=0.0, maxit=60, fixed_iterations=True, mu_mode=orc.MU_USER, mu_user=4.0)
    x1, i1 = orc.gmres(A, b, w_dense=Wd, **kw)
    x2, i2 = orc.gmres(A, b, w_dense=Wd @ R, **kw)
    assert np.linalg.norm(x1 - x2) <= 1e-9 * np.linalg.norm(x1)
    xd = spla.spsolve(A.to_scipy().tocsc(), b)
    x3, i3 = orc.gmres(A, b, m=30, tol=1e-11, maxit=20000, w_dense=Wd)
    assert i3["status"] == 0 and np.linalg.norm(x3 - xd) <= 1e-8 * np.linalg.norm(xd)


def test_dense_w_identity_and_dependent_columns(orc):
    p, A, b = _dense_problem(orc)
    rng = np.random.default_rng(13)
    Wd = rng.standard_normal((A.n, 4))
    x, info, U = orc.gmres(A, b, m=20, tol=1e-9, maxit=5000, w_dense=Wd, return_u=True)
    assert U.shape == (A.n, 4) and np.abs(U.T @ U - np.eye(4)).max() <= 1e-12
    # U^T (A M^-1) U = |mu| I with M^-1 = I + U (|mu| T^-1 - I) U^T, T = U^T A U (Eq. 17)
    Ad = A.to_scipy().toarray()
    T = U.T @ Ad @ U
    mu = abs(info["mu"])
    Minv = np.eye(A.n) + U @ (mu * np.linalg.inv(T) - np.eye(4)) @ U.T
    assert np.abs(U.T @ Ad @ Minv @ U - mu * np.eye(4)).max() <= 1e-9 * mu
    with pytest.raises(ValueError):
        orc.gmres(A, b, w_dense=np.column_stack([Wd, Wd[:, 0] + 2 * Wd[:, 1]]))


def _random_sparse(seed, N, density):
    """Nonsymmetric sparse matrix with irregular row lengths (including rows holding only
    the diagonal) whose symmetric part is positive definite (diagonal above the mean of
    each row's and column's off-diagonal absolute sums): restarted GMRES(m) then converges
    for every m >= 1 (Elman's bound), while an indefinite matrix may stagnate at small m."""
    rng = np.random.default_rng(seed)
    M = sp.random(N, N, density=density, random_state=rng, format="csr")
    M.data = rng.standard_normal(M.nnz)
    M = (M - sp.diags(M.diagonal())).tocsr()
    absM = abs(M)
    off = 0.5 * (np.asarray(absM.sum(axis=1)).ravel() + np.asarray(absM.sum(axis=0)).ravel())
    M = (M + sp.diags(off + 1.0 + rng.random(N))).tocsr()
    M.sort_indices()
    return M, rng


@pytest.mark.parametrize("N,density,m", [(1, 1.0, 1), (2, 0.5, 1), (5, 0.4, 2), (17, 0.2, 3),
                                         (40, 0.1, 7), (97, 0.05, 10)])
@pytest.mark.parametrize("ortho", [0, 1])
def test_random_sparse_systems_against_dense_solve(orc, N, density, m, ortho):
    # brute force on small irregular systems: short restart lengths force many cycles, and
    # the solution must be numpy's dense solve; an aggregate map with a random assignment
    # (every aggregate non-empty) exercises the EBP and projector paths on the same systems
    M, rng = _random_sparse(1000 + N, N, density)
    A = orc.CSR(M.indptr, M.indices, M.data)
    xt = rng.standard_normal(N)
    b = M @ xt
    xd = np.linalg.solve(M.toarray(), b)
    x, info = orc.gmres(A, b, m=m, tol=1e-13, maxit=20000, ortho=ortho)
    assert info["status"] == 0, info
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    r = max(1, N // 4)
    agg = np.concatenate([np.arange(r), rng.integers(0, r, N - r)]).astype(np.int32)
    rng.shuffle(agg)
    d = orc.Deflation(A, agg, r)
    x2, info2 = orc.gmres(A, b, m=m, tol=1e-13, maxit=20000, defl=d, ortho=ortho,
                          mu_mode=orc.MU_USER, mu_user=3.0)
    assert info2["status"] == 0, info2
    assert np.linalg.norm(x2 - xd) <= 1e-10 * np.linalg.norm(xd)
    x3, info3 = orc.gmres(A, b, m=m, tol=1e-13, maxit=20000, defl=d, ortho=ortho,
                          defl_mode=orc.DEFL_PROJECTOR)
    assert info3["status"] == 0, info3
    assert np.linalg.norm(x3 - xd) <= 1e-10 * np.linalg.norm(xd)
