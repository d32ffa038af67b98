"""Parity at full size.  The headline system, in the configuration bench.py times:
q1-n1024 (1,050,625 DOF, 9,422,857 nnz), 1024 aggregate deflation vectors, GMRES(50),
the paper's MGS projections in their one-reduction form.  Two restart cycles in the
fixed-iteration protocol against the oracle's MGS GMRES (every entry of x), and the solve
to 1e-8 checked with the oracle's own SpMV (the true residual of the returned x).  The
differentiable-solve system q1-n512: two adjoint GMRES(50) cycles against the oracle."""
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


@pytest.fixture(scope="module")
def system(orc):
    p = W.workload2()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    return p, A, b


@pytest.mark.parametrize("dot", ["fp64", "df32"])
def test_full_size_fixed_iterations_match_oracle_mgs(G, orc, system, dot):
    p, A, b = system
    s = gpu_solver_from_oracle(G, A, p.agg, p.r, ortho=G.ORTHO_MGS_LOWSYNC, mu_mode=1,
                               mu_user=14.0, fixed_iterations=True,
                               dot_arith=G.DOT_DF32 if dot == "df32" else G.DOT_FP64)
    xg, ig = s.solve(to_dev(b), m=50, tol=0.0, maxit=100)
    d = orc.Deflation(A, p.agg, p.r)
    xo, io = orc.gmres(A, b, defl=d, m=50, tol=0.0, maxit=100, mu_mode=1, mu_user=14.0,
                       fixed_iterations=True, ortho=orc.MGS)
    assert ig["iters"] == io["iters"] == 100
    assert relerr(xg.cpu().numpy(), xo) <= 1e-9
    assert ig["rel_res_true"] == pytest.approx(io["rel_res_true"], rel=1e-7)


def test_full_size_solve_true_residual(G, orc, system):
    p, A, b = system
    s = gpu_solver_from_oracle(G, A, p.agg, p.r, ortho=G.ORTHO_MGS_LOWSYNC)
    xg, ig = s.solve(to_dev(b), m=50, tol=1e-8, maxit=20000)
    assert ig["status"] == 0
    x = xg.cpu().numpy()
    r = b - A.matvec(x)  # the oracle's SpMV, in FP64 on the host
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1e-8
    assert rel == pytest.approx(ig["rel_res_true"], rel=1e-6)


def test_full_size_adjoint_fixed_iterations_q1_n512(G, orc):
    # the differentiable-solve workload at its full size (q1-n512: 263,169 DOF,
    # 2,352,137 nnz, 16 x 16 aggregates): two GMRES(50) cycles of the adjoint solve
    # A^T lam = g (transpose built on the device, T^-T) in the fixed-iteration protocol of
    # Sec. 4, every entry of lam against the oracle's GMRES on the explicit transpose
    p, _ = W.workload5(512)
    A, _ = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    g = W.uniform(5120, 1, A.n, -1, 1)
    s = gpu_solver_from_oracle(G, A, p.agg, p.r, mu_mode=1, mu_user=8.0,
                               fixed_iterations=True)
    lam, il = s.adjoint_solve(to_dev(g), m=50, tol=0.0, maxit=100)
    At = A.transpose()
    lo, io = orc.gmres(At, g, m=50, tol=0.0, maxit=100, defl=orc.Deflation(At, p.agg, p.r),
                       mu_mode=1, mu_user=8.0, fixed_iterations=True)
    assert il["iters"] == io["iters"] == 100
    assert relerr(lam.cpu().numpy(), lo) <= 1e-9
    assert il["rel_res_true"] == pytest.approx(io["rel_res_true"], rel=1e-7)
