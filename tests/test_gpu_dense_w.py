"""GPU parity of a deflation space given as dense columns W (Eqs. 16-18 with U the
orthonormalisation of W) against the oracle's same option: aggregate indicators given
densely reproduce the aggregate EBP solve, a random W gives the oracle's iterates and
the oracle's U U^T, and the option's limits."""
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


def _system(orc):
    p = W.workload1()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    return p, A, b


def test_dense_aggregate_indicators_reproduce_ebp(G, orc):
    p, A, b = _system(orc)
    Wd = np.zeros((A.n, p.r))
    Wd[np.arange(A.n), p.agg] = 1.0
    s_d = gpu_solver_from_oracle(G, A, None, 0, w_dense=to_dev(Wd))
    xd, idd = s_d.solve(to_dev(b), m=30, tol=1e-11, maxit=20000)
    s_e = gpu_solver_from_oracle(G, A, p.agg, p.r)
    xe, ie = s_e.solve(to_dev(b), m=30, tol=1e-11, maxit=20000)
    xo, io = orc.gmres(A, b, m=30, tol=1e-11, maxit=20000, w_dense=Wd)
    assert idd["status"] == ie["status"] == io["status"] == 0
    assert abs(idd["iters"] - ie["iters"]) <= 1 and abs(idd["iters"] - io["iters"]) <= 1
    assert relerr(xd.cpu().numpy(), xe.cpu().numpy()) <= 1e-9
    assert relerr(xd.cpu().numpy(), xo) <= 1e-9
    assert s_d.layout()["adapt_q"] == p.r


def test_dense_random_w_fixed_iterations_match_oracle(G, orc):
    p, A, b = _system(orc)
    rng = np.random.default_rng(21)
    Wd = rng.standard_normal((A.n, 6))
    kw = dict(mu_mode=1, mu_user=4.0, fixed_iterations=True)
    s = gpu_solver_from_oracle(G, A, None, 0, w_dense=to_dev(Wd), **kw)
    xg, ig = s.solve(to_dev(b), m=20, tol=0.0, maxit=61)
    Ug, Tg = (t.cpu().numpy() for t in s.adaptive_space())
    xo, io, Uo = orc.gmres(A, b, m=20, tol=0.0, maxit=61, w_dense=Wd, mu_mode=1, mu_user=4.0,
                           fixed_iterations=True, return_u=True)
    assert ig["iters"] == io["iters"] == 61
    assert relerr(xg.cpu().numpy(), xo) <= 1e-9
    assert ig["rel_res_true"] == pytest.approx(io["rel_res_true"], rel=1e-7, abs=1e-13)
    assert Ug.shape == Uo.shape == (A.n, 6)
    assert np.abs(Ug @ Ug.T - Uo @ Uo.T).max() <= 1e-10
    assert np.abs(Tg - Ug.T @ (A.to_scipy() @ Ug)).max() <= 1e-10 * np.abs(Tg).max()


def test_dense_w_limits(G, orc):
    p, A, b = _system(orc)
    rng = np.random.default_rng(22)
    Wd = rng.standard_normal((A.n, 3))
    dep = np.column_stack([Wd, Wd[:, 0] - 0.5 * Wd[:, 2]])
    s = gpu_solver_from_oracle(G, A, None, 0, w_dense=to_dev(dep))
    with pytest.raises(G.GmresError):  # a dependent column, found at the first solve
        s.solve(to_dev(b), m=20, tol=1e-8, maxit=1000)
    with pytest.raises(G.GmresError):  # FP64 only
        gpu_solver_from_oracle(G, A, None, 0, w_dense=to_dev(Wd), precision=G.FP32_INNER)
    with pytest.raises(G.GmresError):  # at most 32 columns
        gpu_solver_from_oracle(G, A, None, 0, w_dense=to_dev(rng.standard_normal((A.n, 33))))
    s2 = gpu_solver_from_oracle(G, A, None, 0, w_dense=to_dev(Wd))
    with pytest.raises(G.GmresError):  # forward solves only
        s2.adjoint_solve(to_dev(b))
    with pytest.raises(G.GmresError):  # single-system solves
        G.batch_solve([s2], [to_dev(b)], m=20, tol=1e-8, maxit=1000)
    with pytest.raises(ValueError):
        gpu_solver_from_oracle(G, A, p.agg, p.r, w_dense=to_dev(Wd))
