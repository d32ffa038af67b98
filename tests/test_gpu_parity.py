"""GPU parity: the CUDA library (through the C ABI) against the FP64 CPU oracle.

Bars: CSR index arrays bit-exact; FP64 solutions ||x_gpu - x_cpu|| / ||x_cpu|| <= 1e-9
(both solved to a relative residual of 1e-12, where two correct solvers agree to about
cond(A) * 1e-12); mixed precision: true FP64 relative residual <= 1e-10.
"""
import numpy as np
import pytest

import workloads as W
from helpers import gpu_solver_from_oracle, relerr, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_04051_gb300 as G
    from paper_1906_04051_gb300 import build as B
    B.build()
    return G


# ---------------------------------------------------------------------------------------
# assembly
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 255])
def test_q1_assembly_matches_oracle(G, orc, n):
    p = W.convdiff(n, pe=37.0, sigma=0.6, seed=3 + n, px=2, py=2, f_kind="uniform")
    u = W.uniform(11, 9, (n + 1) ** 2, -1, 1)
    for uu in (None, u):
        rowptr, col, val, b = G.q1_assemble(n, to_dev(p.kappa), p.beta, to_dev(p.f),
                                            None if uu is None else to_dev(uu))
        A, bo = orc.q1_assemble(n, p.kappa, p.beta, p.f, uu)
        assert np.array_equal(rowptr.cpu().numpy(), A.rowptr)
        assert np.array_equal(col.cpu().numpy(), A.col)
        scale = np.abs(A.val).max()
        assert np.abs(val.cpu().numpy() - A.val).max() <= 1e-14 * scale
        bs = max(np.abs(bo).max(), 1e-300)
        assert np.abs(b.cpu().numpy() - bo).max() <= 1e-13 * bs


@pytest.mark.parametrize("n", [1024, 2048])
def test_q1_assembly_indices_full_size(G, orc, n):
    p = W.workload2() if n == 1024 else W.workload3()
    rowptr, col, val, b = G.q1_assemble(n, to_dev(p.kappa), p.beta, to_dev(p.f))
    A, bo = orc.q1_assemble(n, p.kappa, p.beta, p.f)
    assert np.array_equal(rowptr.cpu().numpy(), A.rowptr)
    assert np.array_equal(col.cpu().numpy(), A.col)
    assert np.abs(val.cpu().numpy() - A.val).max() <= 1e-14 * np.abs(A.val).max()
    del rowptr, col, val, b


def test_q1_kappa_grad_matches_oracle(G, orc):
    n = 33
    rng = np.random.default_rng(1)
    lam = rng.standard_normal((n + 1) ** 2)
    x = rng.standard_normal((n + 1) ** 2)
    g = G.q1_kappa_grad(n, to_dev(lam), to_dev(x)).cpu().numpy()
    go = orc.q1_kappa_grad(n, lam, x)
    assert np.abs(g - go).max() <= 1e-13 * np.abs(go).max()


# ---------------------------------------------------------------------------------------
# solves
# ---------------------------------------------------------------------------------------
def _solve_both(G, orc, p, *, m, tol, maxit, mode="ebp", mu_mode=0, mu_user=0.0,
                fixed=False, x0=None):
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    dm = {"ebp": G.DEFL_EBP, "none": G.DEFL_NONE, "proj": G.DEFL_PROJECTOR}[mode]
    s = gpu_solver_from_oracle(G, A, p.agg if mode != "none" else None,
                               p.r if mode != "none" else 0, mu_mode=mu_mode, mu_user=mu_user,
                               fixed_iterations=fixed, deflation_mode=dm)
    xg, ig = s.solve(to_dev(b), None if x0 is None else to_dev(x0), m=m, tol=tol, maxit=maxit)
    d = orc.Deflation(A, p.agg, p.r) if mode != "none" else None
    odm = {"ebp": orc.DEFL_EBP, "none": orc.DEFL_NONE, "proj": orc.DEFL_PROJECTOR}[mode]
    xo, io = orc.gmres(A, b, x0, m=m, tol=tol, maxit=maxit, defl=d, defl_mode=odm,
                       mu_mode=mu_mode, mu_user=mu_user, fixed_iterations=fixed)
    return xg.cpu().numpy(), ig, xo, io, s


# mu enters only the EBP preconditioner: the other modes run with the default rule
@pytest.mark.parametrize("mode,mu_mode", [("ebp", 0), ("ebp", 1), ("ebp", 2), ("none", 0),
                                          ("proj", 0)])
def test_workload1_tight_tolerance(G, orc, mode, mu_mode):
    p = W.workload1()
    xg, ig, xo, io, _ = _solve_both(G, orc, p, m=30, tol=1e-12, maxit=20000, mode=mode,
                                    mu_mode=mu_mode, mu_user=6.0)
    assert ig["status"] == 0 and io["status"] == 0, (ig, io)
    assert relerr(xg, xo) <= 1e-9
    assert ig["rel_res_true"] <= 1e-12
    if mode == "ebp":
        assert ig["mu"] == pytest.approx(io["mu"], rel=1e-10)
    # same method, same arithmetic up to rounding: iteration counts agree closely
    assert abs(ig["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"])


def _permuted(orc, A, b, agg, seed):
    """P A P^T, P b, P agg for a seeded random permutation: the same system with its
    unknowns renumbered, no longer banded (many distinct diagonals)."""
    import scipy.sparse as sp
    n = A.n
    perm = np.random.default_rng(seed).permutation(n)
    P = sp.csr_matrix((np.ones(n), (np.arange(n), perm)), shape=(n, n))
    Ap = (P @ A.to_scipy() @ P.T).tocsr()
    Ap.sort_indices()
    return orc.CSR(Ap.indptr, Ap.indices, Ap.data), b[perm], agg[perm], perm


@pytest.mark.parametrize("mode", ["ebp", "proj", "none"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_general_csr_path_permuted(G, orc, mode, prec):
    # a renumbered (non-banded) matrix takes the CSR kernels instead of the diagonal
    # storage; the solution is the renumbered solution of the banded system
    p = W.convdiff(40, pe=25.0, sigma=0.5, seed=77, px=2, py=3)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    Ap, bp, aggp, perm = _permuted(orc, A, b, p.agg, seed=5)
    dm = {"ebp": G.DEFL_EBP, "none": G.DEFL_NONE, "proj": G.DEFL_PROJECTOR}[mode]
    pr = {"fp64": G.FP64, "fp32": G.FP32_INNER}[prec]
    defl = mode != "none"
    s = gpu_solver_from_oracle(G, Ap, aggp if defl else None, p.r if defl else 0,
                               deflation_mode=dm, precision=pr)
    xg, ig = s.solve(to_dev(bp), m=30, tol=1e-11, maxit=20000)
    d = orc.Deflation(Ap, aggp, p.r) if defl else None
    odm = {"ebp": orc.DEFL_EBP, "none": orc.DEFL_NONE, "proj": orc.DEFL_PROJECTOR}[mode]
    xo, io = orc.gmres(Ap, bp, None, m=30, tol=1e-11, maxit=20000, defl=d, defl_mode=odm)
    assert ig["status"] == 0 and io["status"] == 0, (ig, io)
    assert ig["rel_res_true"] <= 1e-11
    assert relerr(xg.cpu().numpy(), xo) <= 1e-8
    # and against the banded (diagonal storage) solve of the unpermuted system
    s2 = gpu_solver_from_oracle(G, A, p.agg if defl else None, p.r if defl else 0,
                                deflation_mode=dm, precision=pr)
    x2, i2 = s2.solve(to_dev(b), m=30, tol=1e-11, maxit=20000)
    assert relerr(xg.cpu().numpy(), x2.cpu().numpy()[perm]) <= 1e-8
    # the banded system is held in diagonal storage (9 diagonals), the renumbered one not
    lay, lay2 = s.layout(), s2.layout()
    assert lay["ndiag"] == 0 and lay2["ndiag"] == 9
    assert lay["nnz"] == lay2["nnz"] == A.nnz and lay["n"] == A.n
    assert lay["r"] == (p.r if defl else 0)
    if prec == "fp64":
        assert abs(ig["iters"] - i2["iters"]) <= 3


@pytest.mark.parametrize("maxit", [7, 45])
@pytest.mark.parametrize("mode", ["ebp", "proj", "none"])
@pytest.mark.parametrize("ortho", ["cgs2", "mgs_lowsync"])
def test_general_csr_fixed_iterations(G, orc, mode, maxit, ortho):
    # the thread-per-row CSR SpMV (a renumbered, non-banded system) in the fixed-iteration
    # protocol of Sec. 4: the same step count and mu on both sides, every entry of x
    p = W.convdiff(40, pe=25.0, sigma=0.5, seed=78, px=2, py=3)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    Ap, bp, aggp, _ = _permuted(orc, A, b, p.agg, seed=6)
    defl = mode != "none"
    dm = {"ebp": G.DEFL_EBP, "none": G.DEFL_NONE, "proj": G.DEFL_PROJECTOR}[mode]
    go = {"cgs2": G.ORTHO_CGS2, "mgs_lowsync": G.ORTHO_MGS_LOWSYNC}[ortho]
    s = gpu_solver_from_oracle(G, Ap, aggp if defl else None, p.r if defl else 0,
                               deflation_mode=dm, mu_mode=1, mu_user=5.0,
                               fixed_iterations=True, ortho=go)
    lay = s.layout()
    assert lay["ndiag"] == 0 and lay["spmv_lanes"] == 0  # CSR, a thread per row
    xg, ig = s.solve(to_dev(bp), m=10, tol=0.0, maxit=maxit)
    d = orc.Deflation(Ap, aggp, p.r) if defl else None
    odm = {"ebp": orc.DEFL_EBP, "none": orc.DEFL_NONE, "proj": orc.DEFL_PROJECTOR}[mode]
    oo = orc.CGS2 if ortho == "cgs2" else orc.MGS
    xo, io = orc.gmres(Ap, bp, None, m=10, tol=0.0, maxit=maxit, defl=d, defl_mode=odm,
                       mu_mode=1, mu_user=5.0, fixed_iterations=True, ortho=oo)
    assert ig["iters"] == io["iters"] == maxit
    assert relerr(xg.cpu().numpy(), xo) <= 1e-9
    assert ig["rel_res_true"] == pytest.approx(io["rel_res_true"], rel=1e-7, abs=1e-13)


@pytest.mark.parametrize("n", [3, 17, 40])
@pytest.mark.parametrize("maxit", [1, 7, 45])
@pytest.mark.parametrize("mode", ["ebp", "proj"])
def test_fixed_iterations_parity(G, orc, n, maxit, mode):
    # fixed-iteration protocol (Sec. 4): identical step counts, so the iterates agree to
    # rounding amplified by the Krylov process
    p = W.convdiff(n, pe=25.0, sigma=0.5, seed=100 + n, px=2, py=3)
    xg, ig, xo, io, _ = _solve_both(G, orc, p, m=10, tol=0.0, maxit=maxit, mu_mode=1,
                                    mu_user=5.0, fixed=True, mode=mode)
    assert ig["iters"] == io["iters"] == min(maxit, ig["iters"])
    assert relerr(xg, xo) <= 1e-9
    # at a converged iterate the true residual is rounding noise: the two sides form
    # A U y (Eq. 18) in different orders (A W summed per row on the GPU), which moves it
    # by a few hundred ulps of ||b|| at most
    assert ig["rel_res_true"] == pytest.approx(io["rel_res_true"], rel=1e-7, abs=1e-13)


def test_fixed_iterations_ritz_mu(G, orc):
    p = W.convdiff(48, pe=60.0, sigma=0.5, seed=9, px=4, py=2)
    xg, ig, xo, io, _ = _solve_both(G, orc, p, m=20, tol=0.0, maxit=90, fixed=True)
    assert ig["iters"] == io["iters"] == 90
    assert ig["mu"] == pytest.approx(io["mu"], rel=1e-10)
    assert relerr(xg, xo) <= 1e-9


def test_nonzero_initial_guess(G, orc):
    p = W.convdiff(30, pe=15.0, sigma=0.3, seed=21, px=2, py=2)
    x0 = W.uniform(5, 5, p.N, -1, 1)
    xg, ig, xo, io, _ = _solve_both(G, orc, p, m=25, tol=1e-12, maxit=5000, x0=x0)
    assert ig["status"] == 0 and relerr(xg, xo) <= 1e-9


def test_zero_rhs_and_maxit_zero(G, orc):
    p = W.convdiff(8, pe=5.0, sigma=0.0, seed=1, px=2, py=2)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    s = gpu_solver_from_oracle(G, A, p.agg, p.r)
    x, info = s.solve(torch.zeros(A.n, dtype=torch.float64, device="cuda"), m=5)
    assert info["status"] == 0 and info["iters"] == 0 and not torch.any(x)
    x, info = s.solve(to_dev(b), m=5, tol=1e-8, maxit=0)
    assert info["status"] == 1 and info["iters"] == 0


def test_restart_lengths_and_ragged_sizes(G, orc):
    for n, m in [(5, 1), (11, 2), (23, 64), (31, 9)]:
        p = W.convdiff(n, pe=8.0, sigma=0.4, seed=n, px=3, py=2)
        xg, ig, xo, io, _ = _solve_both(G, orc, p, m=m, tol=1e-12, maxit=50000)
        assert ig["status"] == 0, (n, m, ig)
        assert relerr(xg, xo) <= 1e-9, (n, m)


def test_deterministic_bitwise(G, orc):
    p = W.convdiff(64, pe=40.0, sigma=0.5, seed=4, px=4, py=4)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    s = gpu_solver_from_oracle(G, A, p.agg, p.r)
    x1, i1 = s.solve(to_dev(b), m=30, tol=1e-10, maxit=3000)
    x2, i2 = s.solve(to_dev(b), m=30, tol=1e-10, maxit=3000)
    assert i1["iters"] == i2["iters"]
    assert torch.equal(x1, x2)


def test_adjoint_matches_oracle(G, orc):
    p = W.convdiff(40, pe=30.0, sigma=0.5, seed=12, px=2, py=4)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    s = gpu_solver_from_oracle(G, A, p.agg, p.r)
    g = W.uniform(77, 1, A.n, -1, 1)
    lam, info = s.adjoint_solve(to_dev(g), m=30, tol=1e-12, maxit=10000)
    At = A.transpose()
    lo, io = orc.gmres(At, g, m=30, tol=1e-12, maxit=10000, defl=orc.Deflation(At, p.agg, p.r))
    assert info["status"] == 0 and io["status"] == 0
    assert relerr(lam.cpu().numpy(), lo) <= 1e-9
    # <A x, lam> = <x, A^T lam>
    x, _ = s.solve(to_dev(b), m=30, tol=1e-12, maxit=10000)
    xn = x.cpu().numpy()
    assert abs(A.matvec(xn) @ lam.cpu().numpy() - xn @ g) <= 1e-9 * np.abs(xn @ g)


@pytest.mark.parametrize("prec,name", [(1, "fp32"), (2, "bf16")])
@pytest.mark.parametrize("dmode", [0, 1])
def test_mixed_precision_reaches_1e10(G, orc, prec, name, dmode):
    p = W.convdiff(96, pe=50.0, sigma=0.5, seed=33, px=4, py=4)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    s = gpu_solver_from_oracle(G, A, p.agg, p.r, precision=prec, deflation_mode=dmode)
    x, info = s.solve(to_dev(b), m=40, tol=1e-10, maxit=20000)
    assert info["status"] == 0, info
    xn = x.cpu().numpy()
    true_rel = np.linalg.norm(b - A.matvec(xn)) / np.linalg.norm(b)
    assert true_rel <= 1e-10
    xo, io = orc.gmres(A, b, m=40, tol=1e-12, maxit=20000, defl=orc.Deflation(A, p.agg, p.r))
    assert relerr(xn, xo) <= 1e-7  # reported accuracy vs the FP64 oracle


# ---------------------------------------------------------------------------------------
# error paths (host-detected, or device flags read by the host; nothing faults)
# ---------------------------------------------------------------------------------------
def test_invalid_csr_rejected(G, orc):
    A, b = orc.q1_assemble(4, np.ones(16), (1.0, 0.0), np.ones(25))
    col = A.col.copy()
    col[10], col[11] = col[11], col[10]  # unsorted row
    with pytest.raises(G.GmresError) as e:
        G.Solver(to_dev(A.rowptr), to_dev(col), to_dev(A.val))
    assert e.value.status == -1


def test_empty_aggregate_rejected(G, orc):
    p = W.convdiff(6, pe=5.0, sigma=0.0, seed=1, px=2, py=2)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    agg = p.agg.copy()
    agg[agg == 1] = 0
    with pytest.raises(G.GmresError) as e:
        gpu_solver_from_oracle(G, A, agg, p.r)
    assert e.value.status == -4


def test_nan_rhs_reports_nan(G, orc):
    p = W.convdiff(10, pe=5.0, sigma=0.0, seed=1, px=2, py=2)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    b = b.copy()
    b[17] = np.nan
    s = gpu_solver_from_oracle(G, A, p.agg, p.r)
    with pytest.raises(G.GmresError) as e:
        s.solve(to_dev(b), m=10)
    assert e.value.status == -5


def test_bad_restart_length(G, orc):
    A, b = orc.q1_assemble(4, np.ones(16), (1.0, 0.0), np.ones(25))
    s = gpu_solver_from_oracle(G, A)
    for m in (0, 65):
        with pytest.raises(G.GmresError):
            s.solve(to_dev(b), m=m)


def _swapped_band(kl, ku, n, seed):
    """A well-conditioned banded B (kl sub-, ku super-diagonals, diagonal about 8) with
    rows 2i and 2i+1 exchanged: the diagonal of the result holds B's off-diagonal entries,
    so LU with partial pivoting exchanges rows at every step."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    diags, offs = [], []
    for o in range(-kl, ku + 1):
        d = rng.standard_normal(n - abs(o))
        if o == 0:
            d = d + 8.0 * np.sign(d)
        diags.append(d)
        offs.append(o)
    B = sp.diags(diags, offs, shape=(n, n)).tocsr()
    p = np.arange(n)
    p[0:n - 1:2] += 1
    p[1:n:2] -= 1
    A = B[p].tocsr()
    A.sort_indices()
    return A


@pytest.mark.parametrize("kl,ku", [(3, 3), (2, 4)])
def test_band_coarse_inverse_with_row_exchanges(G, orc, kl, ku):
    # every node its own aggregate: T = U^T A U = A, banded with kl + 1 sub- and ku + 1
    # super-diagonals, so gmres_create inverts it by the band LU (Eqs. 17-18), with a row
    # exchange at every step; with U = I the EBP preconditioner is |mu| T^-1, and the
    # solution rests on T^-1 (one GMRES step in exact arithmetic)
    n = 300
    As = _swapped_band(kl, ku, n, seed=7)
    A = orc.CSR(As.indptr, As.indices, As.data)
    b = W.uniform(19, kl, n, -1, 1)
    agg = np.arange(n, dtype=np.int32)
    s = gpu_solver_from_oracle(G, A, agg, n, mu_mode=G.MU_USER, mu_user=1.0)
    assert s.layout()["coarse_band"] == (kl + 1) + (ku + 1) + 1
    xg, ig = s.solve(to_dev(b), m=30, tol=1e-12, maxit=200)
    d = orc.Deflation(A, agg, n)
    xo, io = orc.gmres(A, b, None, m=30, tol=1e-12, maxit=200, defl=d,
                       mu_mode=orc.MU_USER, mu_user=1.0)
    assert ig["status"] == 0 and io["status"] == 0, (ig, io)
    assert relerr(xg.cpu().numpy(), xo) <= 1e-9
    assert np.linalg.norm(As @ xg.cpu().numpy() - b) <= 1e-11 * np.linalg.norm(b)


def test_dense_coarse_matrix_takes_gauss_jordan(G, orc):
    # the 2 x 4 subdomains of the small workloads give a T as wide as it is long: the
    # setup keeps Gauss-Jordan for it
    p = W.convdiff(24, pe=10.0, sigma=0.3, seed=5, px=2, py=4)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    s = gpu_solver_from_oracle(G, A, p.agg, p.r)
    assert s.layout()["coarse_band"] == 0
