"""Batched solve (one CUDA-graph launch for many systems) against single-system solves
and the FP64 oracle, on the Picard-linearised workload q1-batch256."""
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


def _build(G, orc, probs, **kw):
    solvers, bs, sys = [], [], []
    for p in probs:
        A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
        solvers.append(gpu_solver_from_oracle(G, A, p.agg, p.r, **kw))
        bs.append(to_dev(b))
        sys.append((A, b))
    return solvers, bs, sys


@pytest.mark.parametrize("count,n_min,n_max", [(1, 8, 8), (6, 8, 40), (13, 3, 70)])
def test_batch_matches_single_and_oracle(G, orc, count, n_min, n_max):
    probs = W.workload4(count=count, n_min=n_min, n_max=n_max, seed=1000 + count)
    solvers, bs, sys = _build(G, orc, probs)
    xs, infos, st = G.batch_solve(solvers, bs, m=30, tol=1e-12, maxit=20000)
    assert st == 0, infos
    for x, info, s, b, p, (A, bh) in zip(xs, infos, solvers, bs, probs, sys):
        assert info["status"] == 0 and info["rel_res_true"] <= 1e-12
        x1, i1 = s.solve(b, m=30, tol=1e-12, maxit=20000)
        assert relerr(x.cpu().numpy(), x1.cpu().numpy()) <= 1e-9
        assert abs(info["iters"] - i1["iters"]) <= max(3, 0.05 * i1["iters"])
        xo, _ = orc.gmres(A, bh, m=30, tol=1e-12, maxit=20000, defl=orc.Deflation(A, p.agg, p.r))
        assert relerr(x.cpu().numpy(), xo) <= 1e-9


def test_batch_fixed_iterations_parity(G, orc):
    # fixed-iteration protocol with a given mu: each system's iterate equals the oracle's
    probs = W.workload4(count=5, n_min=6, n_max=30, seed=77)
    solvers, bs, sys = _build(G, orc, probs, mu_mode=1, mu_user=5.0, fixed_iterations=True)
    xs, infos, st = G.batch_solve(solvers, bs, m=10, tol=0.0, maxit=37)
    for x, info, p, (A, b) in zip(xs, infos, probs, sys):
        assert info["iters"] == 37
        xo, io = orc.gmres(A, b, m=10, tol=0.0, maxit=37, defl=orc.Deflation(A, p.agg, p.r),
                           mu_mode=1, mu_user=5.0, fixed_iterations=True)
        assert relerr(x.cpu().numpy(), xo) <= 1e-9


def test_batch_graph_reuse_is_deterministic(G, orc):
    probs = W.workload4(count=4, n_min=10, n_max=50, seed=5)
    solvers, bs, _ = _build(G, orc, probs)
    xs1, _, _ = G.batch_solve(solvers, bs, m=30, tol=1e-10, maxit=20000)
    xs1 = [x.clone() for x in xs1]
    xs2, _, _ = G.batch_solve(solvers, bs, m=30, tol=1e-10, maxit=20000)
    for a, b in zip(xs1, xs2):
        assert torch.equal(a, b)


def test_batch_fp32_inner_reaches_1e10(G, orc):
    probs = W.workload4(count=6, n_min=16, n_max=64, seed=9)
    solvers, bs, sys = _build(G, orc, probs, precision=1)
    xs, infos, st = G.batch_solve(solvers, bs, m=30, tol=1e-10, maxit=50000)
    assert st == 0
    for x, (A, b) in zip(xs, sys):
        xn = x.cpu().numpy()
        assert np.linalg.norm(b - A.matvec(xn)) <= 1e-10 * np.linalg.norm(b)


def test_batch256_full_size(G, orc):
    # the full workload in one graph launch.  EBP deflation with eight subdomain vectors
    # stagnates on a few of the larger convection-dominated systems (a property of the
    # method with this coarse space, reproduced by the oracle); every system must either
    # meet the tolerance (checked on the host in FP64) or report NOT_CONVERGED with the
    # residual it actually has, and sampled converged systems must match the oracle
    probs = W.workload4()
    assert len(probs) == 256
    solvers, bs, sys = _build(G, orc, probs)
    xs, infos, st = G.batch_solve(solvers, bs, m=30, tol=1e-8, maxit=4000)
    assert st in (0, 1)
    converged = []
    for i, (x, info, (A, b)) in enumerate(zip(xs, infos, sys)):
        xn = x.cpu().numpy()
        true_rel = np.linalg.norm(b - A.matvec(xn)) / np.linalg.norm(b)
        if info["status"] == 0:
            assert true_rel <= 1.001e-8
            converged.append(i)
        else:
            assert info["status"] == 1 and info["iters"] == 4000
            assert true_rel == pytest.approx(info["rel_res_true"], rel=1e-6)
    assert len(converged) >= 240
    rng = np.random.default_rng(0)
    for i in rng.choice(converged, 6, replace=False):
        A, b = sys[i]
        p = probs[i]
        xo, io = orc.gmres(A, b, m=30, tol=1e-12, maxit=100000, defl=orc.Deflation(A, p.agg, p.r))
        assert io["status"] == 0
        # both within tol 1e-8 of the same solution: bounded by cond(A) * 1e-8
        assert relerr(xs[i].cpu().numpy(), xo) <= 1e-5


def test_batch_lowsync_fixed_iterations_parity(G, orc):
    # the one-reduction MGS in the batched solve: every system's iterate after 37 fixed
    # steps equals the oracle's MGS GMRES and the single-system one-reduction solve
    probs = W.workload4(count=5, n_min=6, n_max=30, seed=78)
    kw = dict(mu_mode=1, mu_user=5.0, fixed_iterations=True, ortho=G.ORTHO_MGS_LOWSYNC)
    solvers, bs, sys = _build(G, orc, probs, **kw)
    xs, infos, st = G.batch_solve(solvers, bs, m=10, tol=0.0, maxit=37)
    xs = [x.clone() for x in xs]
    for x, info, s, bd, p, (A, b) in zip(xs, infos, solvers, bs, probs, sys):
        assert info["iters"] == 37
        xo, io = orc.gmres(A, b, m=10, tol=0.0, maxit=37, defl=orc.Deflation(A, p.agg, p.r),
                           mu_mode=1, mu_user=5.0, fixed_iterations=True, ortho=orc.MGS)
        assert relerr(x.cpu().numpy(), xo) <= 1e-9
        x1, _ = s.solve(bd, m=10, tol=0.0, maxit=37)
        assert relerr(x.cpu().numpy(), x1.cpu().numpy()) <= 1e-11


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_lowsync_to_tolerance(G, orc, precision):
    probs = W.workload4(count=6, n_min=8, n_max=48, seed=2024)
    solvers, bs, sys = _build(G, orc, probs, ortho=G.ORTHO_MGS_LOWSYNC, precision=precision)
    xs, infos, st = G.batch_solve(solvers, bs, m=30, tol=1e-10, maxit=50000)
    assert st == 0, infos
    xs = [x.clone() for x in xs]
    xs2, _, _ = G.batch_solve(solvers, bs, m=30, tol=1e-10, maxit=50000)
    for x, x2, info, p, (A, b) in zip(xs, xs2, infos, probs, sys):
        xn = x.cpu().numpy()
        assert np.linalg.norm(b - A.matvec(xn)) <= 1e-10 * np.linalg.norm(b)
        assert torch.equal(x, x2)  # deterministic
        xo, _ = orc.gmres(A, b, m=30, tol=1e-12, maxit=50000, defl=orc.Deflation(A, p.agg, p.r))
        assert relerr(xn, xo) <= 1e-7


def test_batch_ortho_limits(G, orc):
    probs = W.workload4(count=2, n_min=6, n_max=10, seed=3)
    s1, b1, _ = _build(G, orc, probs[:1], ortho=G.ORTHO_MGS_LOWSYNC)
    s2, b2, _ = _build(G, orc, probs[1:], ortho=G.ORTHO_CGS2)
    with pytest.raises(G.GmresError):  # one orthogonalisation per batch
        G.batch_solve(s1 + s2, b1 + b2, m=10, tol=1e-8, maxit=100)
