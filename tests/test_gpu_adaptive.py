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
