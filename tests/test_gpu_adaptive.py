"""GPU parity of the adaptive deflation (Sec. 3.3, Eq. 19) against the oracle: U starts
empty and grows after each restart cycle by the inverse-power eigenvector(s) of H_k
mapped through the basis; solutions, step counts and the size of U agree."""
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


def _both(G, orc, p, *, m, tol, maxit, rmax=20, mu_mode=0, mu_user=0.0, fixed=False):
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    s = gpu_solver_from_oracle(G, A, None, 0, deflation_mode=G.DEFL_ADAPTIVE, rmax=rmax,
                               mu_mode=mu_mode, mu_user=mu_user, fixed_iterations=fixed)
    xg, ig = s.solve(to_dev(b), m=m, tol=tol, maxit=maxit)
    xo, io = orc.gmres(A, b, m=m, tol=tol, maxit=maxit, defl_mode=orc.DEFL_ADAPTIVE,
                       rmax=rmax, mu_mode=mu_mode, mu_user=mu_user, fixed_iterations=fixed)
    return xg.cpu().numpy(), ig, xo, io, s


def test_adaptive_workload1_matches_oracle(G, orc):
    p = W.workload1()
    xg, ig, xo, io, s = _both(G, orc, p, m=30, tol=1e-11, maxit=20000)
    assert ig["status"] == 0 and io["status"] == 0, (ig, io)
    assert ig["rel_res_true"] <= 1e-11
    assert relerr(xg, xo) <= 1e-9
    assert ig["mu"] == pytest.approx(io["mu"], rel=1e-10)
    assert abs(ig["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"])
    # fewer steps than undeflated GMRES(30) on the same system
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    s0 = gpu_solver_from_oracle(G, A, None, 0, deflation_mode=G.DEFL_NONE)
    _, i0 = s0.solve(to_dev(b), m=30, tol=1e-11, maxit=20000)
    assert ig["iters"] < i0["iters"]


@pytest.mark.parametrize("maxit", [31, 95])
def test_adaptive_fixed_iterations_parity(G, orc, maxit):
    # fixed-iteration protocol: the same steps, U updated after each cycle on both sides
    p = W.convdiff(40, pe=25.0, sigma=0.5, seed=140, px=2, py=3)
    xg, ig, xo, io, _ = _both(G, orc, p, m=15, tol=0.0, maxit=maxit, mu_mode=1, mu_user=5.0,
                              fixed=True)
    assert ig["iters"] == io["iters"] == maxit
    assert relerr(xg, xo) <= 1e-9
    assert ig["rel_res_true"] == pytest.approx(io["rel_res_true"], rel=1e-6, abs=1e-13)


def test_adaptive_truncation_at_rmax(G, orc):
    p = W.workload1()
    xg, ig, xo, io, _ = _both(G, orc, p, m=12, tol=1e-10, maxit=20000, rmax=3)
    assert ig["status"] == 0 and io["status"] == 0
    assert ig["cycles"] > 3
    assert relerr(xg, xo) <= 1e-8
    assert abs(ig["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"])


def test_adaptive_options_rejected(G, orc):
    p = W.workload1()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    with pytest.raises(G.GmresError):
        gpu_solver_from_oracle(G, A, p.agg, p.r, deflation_mode=G.DEFL_ADAPTIVE)
    with pytest.raises(G.GmresError):
        gpu_solver_from_oracle(G, A, None, 0, deflation_mode=G.DEFL_ADAPTIVE,
                               precision=G.FP32_INNER)
    with pytest.raises(G.GmresError):
        gpu_solver_from_oracle(G, A, None, 0, deflation_mode=G.DEFL_ADAPTIVE, rmax=0)


def test_adaptive_space_matches_oracle(G, orc):
    # the space itself: U (up to rounding, same signs) and T = U^T A U after 6 cycles
    p = W.convdiff(40, pe=25.0, sigma=0.5, seed=140, px=2, py=3)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    s = gpu_solver_from_oracle(G, A, None, 0, deflation_mode=G.DEFL_ADAPTIVE, rmax=20,
                               mu_mode=1, mu_user=5.0, fixed_iterations=True)
    _, ig = s.solve(to_dev(b), m=15, tol=0.0, maxit=90)
    Ug, Tg = (t.cpu().numpy() for t in s.adaptive_space())
    _, io, Uo = orc.gmres(A, b, m=15, tol=0.0, maxit=90, defl_mode=orc.DEFL_ADAPTIVE, rmax=20,
                          mu_mode=1, mu_user=5.0, fixed_iterations=True, return_u=True)
    assert Ug.shape == Uo.shape and Ug.shape[1] == io["q"] >= 3
    assert s.layout()["adapt_q"] == Ug.shape[1]
    assert np.abs(Ug - Uo).max() <= 1e-8
    As = A.to_scipy()
    assert np.abs(Tg - Uo.T @ (As @ Uo)).max() <= 1e-10 * np.abs(Tg).max()


def test_adaptive_space_invariants(G, orc):
    # Eq. 17 on the returned space: U orthonormal, T = U^T A U, U^T (A M^-1) U = |mu| I
    p = W.workload1()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    s = gpu_solver_from_oracle(G, A, None, 0, deflation_mode=G.DEFL_ADAPTIVE, rmax=4)
    _, ig = s.solve(to_dev(b), m=20, tol=1e-10, maxit=20000)
    assert ig["status"] == 0 and ig["cycles"] > 4
    Ug, Tg = (t.cpu().numpy() for t in s.adaptive_space())
    q = Ug.shape[1]
    assert q == 4  # the space filled up and was truncated, never beyond rmax
    assert np.abs(Ug.T @ Ug - np.eye(q)).max() <= 1e-12
    As = A.to_scipy()
    AU = As @ Ug
    assert np.abs(Tg - Ug.T @ AU).max() <= 1e-12 * np.abs(Tg).max()
    mu = abs(ig["mu"])
    AMU = AU + AU @ (mu * np.linalg.solve(Tg, np.eye(q)) - np.eye(q))  # A M^-1 U
    assert np.abs(Ug.T @ AMU - mu * np.eye(q)).max() <= 1e-9 * mu


def test_adaptive_space_rejected_for_other_modes(G, orc):
    p = W.workload1()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    s = gpu_solver_from_oracle(G, A, p.agg, p.r)
    with pytest.raises(G.GmresError):
        s.adaptive_space()


@pytest.mark.parametrize("rmax", [1, 3, 6])
def test_adaptive_drop_fixed_iterations_parity(G, orc, rmax):
    # many cycles at a full space: every update drops the direction(s) of T's largest
    # eigenvalue first; the solution and the space (as a projector U U^T, which does not
    # depend on the basis chosen inside it) agree with the oracle's
    p = W.convdiff(40, pe=25.0, sigma=0.5, seed=140, px=2, py=3)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    s = gpu_solver_from_oracle(G, A, None, 0, deflation_mode=G.DEFL_ADAPTIVE, rmax=rmax,
                               mu_mode=1, mu_user=5.0, fixed_iterations=True)
    xg, ig = s.solve(to_dev(b), m=10, tol=0.0, maxit=160)
    xg = xg.cpu().numpy()
    Ug, _ = s.adaptive_space()
    Ug = Ug.cpu().numpy()
    xo, io, Uo = orc.gmres(A, b, m=10, tol=0.0, maxit=160, defl_mode=orc.DEFL_ADAPTIVE,
                           rmax=rmax, mu_mode=1, mu_user=5.0, fixed_iterations=True,
                           return_u=True)
    assert ig["iters"] == io["iters"] == 160 and ig["cycles"] == io["cycles"] == 16
    assert Ug.shape == Uo.shape and 1 <= Ug.shape[1] <= rmax
    assert relerr(xg, xo) <= 1e-9
    Pg, Po = Ug @ Ug.T, Uo @ Uo.T
    assert np.abs(Pg - Po).max() <= 1e-8
