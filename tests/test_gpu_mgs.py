"""GPU parity of the modified Gram-Schmidt orthogonalisation (the paper's, Sec. 3.2,
Eq. 13) against the oracle's MGS GMRES, in both GPU forms: one cooperative kernel per
Arnoldi step (column by column), and the one-reduction inverse compact WY form (the
same projections: (I + L) h = V^T w).  The same steps and solutions in every deflation
mode, bitwise repeatable runs, the same step counts as CGS2, and the options' limits."""
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


@pytest.mark.parametrize("lowsync", [False, True])
@pytest.mark.parametrize("mode", ["ebp", "proj", "none", "adaptive"])
def test_mgs_fixed_iterations_match_oracle(G, orc, mode, lowsync):
    p = W.convdiff(40, pe=25.0, sigma=0.5, seed=140, px=2, py=3)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    gm = {"ebp": G.DEFL_EBP, "proj": G.DEFL_PROJECTOR, "none": G.DEFL_NONE,
          "adaptive": G.DEFL_ADAPTIVE}[mode]
    om = {"ebp": orc.DEFL_EBP, "proj": orc.DEFL_PROJECTOR, "none": orc.DEFL_NONE,
          "adaptive": orc.DEFL_ADAPTIVE}[mode]
    defl = mode in ("ebp", "proj")
    s = gpu_solver_from_oracle(G, A, p.agg if defl else None, p.r if defl else 0,
                               deflation_mode=gm, mu_mode=1, mu_user=5.0,
                               fixed_iterations=True,
                               ortho=G.ORTHO_MGS_LOWSYNC if lowsync else G.ORTHO_MGS)
    xg, ig = s.solve(to_dev(b), m=15, tol=0.0, maxit=47)
    d = orc.Deflation(A, p.agg, p.r) if defl else None
    xo, io = orc.gmres(A, b, defl=d, defl_mode=om, m=15, tol=0.0, maxit=47, mu_mode=1,
                       mu_user=5.0, fixed_iterations=True, ortho=orc.MGS)
    assert ig["iters"] == io["iters"] == 47
    assert relerr(xg.cpu().numpy(), xo) <= 1e-9
    assert ig["rel_res_true"] == pytest.approx(io["rel_res_true"], rel=1e-6, abs=1e-13)
    assert ig["rel_res_est"] == pytest.approx(io["rel_res_est"], rel=1e-6, abs=1e-13)


@pytest.mark.parametrize("lowsync", [False, True])
def test_mgs_to_tolerance_matches_oracle_and_repeats(G, orc, lowsync):
    p = W.workload1()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    s = gpu_solver_from_oracle(G, A, p.agg, p.r,
                               ortho=G.ORTHO_MGS_LOWSYNC if lowsync else G.ORTHO_MGS)
    xg, ig = s.solve(to_dev(b), m=30, tol=1e-11, maxit=20000)
    xg2, ig2 = s.solve(to_dev(b), m=30, tol=1e-11, maxit=20000)
    d = orc.Deflation(A, p.agg, p.r)
    xo, io = orc.gmres(A, b, defl=d, m=30, tol=1e-11, maxit=20000, ortho=orc.MGS)
    assert ig["status"] == 0 and io["status"] == 0
    assert ig["rel_res_true"] <= 1e-11
    assert relerr(xg.cpu().numpy(), xo) <= 1e-9
    assert abs(ig["iters"] - io["iters"]) <= 2
    assert torch.equal(xg, xg2) and ig["iters"] == ig2["iters"]  # deterministic


def test_mgs_and_cgs2_take_the_same_steps(G, orc):
    # the same Krylov space: step counts to 1e-10 agree on a 66k-DOF system
    p = W.workload2(256)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    its = {}
    for name, o in (("cgs2", G.ORTHO_CGS2), ("mgs", G.ORTHO_MGS),
                    ("lowsync", G.ORTHO_MGS_LOWSYNC)):
        s = gpu_solver_from_oracle(G, A, p.agg, p.r, ortho=o)
        x, info = s.solve(to_dev(b), m=50, tol=1e-10, maxit=50000)
        assert info["status"] == 0 and info["rel_res_true"] <= 1e-10
        its[name] = (info["iters"], x.cpu().numpy())
    for name in ("mgs", "lowsync"):
        assert abs(its[name][0] - its["cgs2"][0]) <= max(3, 0.02 * its["cgs2"][0])
        assert relerr(its[name][1], its["cgs2"][1]) <= 1e-7


def test_mgs_bratu_newton(G, orc):
    import scipy.sparse.linalg as spla
    n = 4
    u = np.zeros((2 * n + 1) ** 3)
    for _ in range(30):
        A, b = orc.q2_bratu_assemble(n, 6.8, u)
        du = spla.spsolve(A.to_scipy().tocsc(), b)
        u += du
        if np.abs(du).max() <= 1e-12:
            break
    ug, info = G.bratu_newton(n, 6.8, m=30, tol=1e-11, newton_tol=1e-10,
                              deflation_mode=G.DEFL_ADAPTIVE, ortho=G.ORTHO_MGS)
    assert info["status"] == 0
    assert np.abs(ug.cpu().numpy() - u).max() <= 1e-8


def test_lowsync_fp32_inner_refines_to_fp64(G, orc):
    p = W.convdiff(96, pe=50.0, sigma=0.5, seed=150, px=4, py=4)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    s = gpu_solver_from_oracle(G, A, p.agg, p.r, precision=G.FP32_INNER,
                               ortho=G.ORTHO_MGS_LOWSYNC)
    xg, ig = s.solve(to_dev(b), m=40, tol=1e-10, maxit=50000)
    assert ig["status"] == 0 and ig["rel_res_true"] <= 1e-10
    d = orc.Deflation(A, p.agg, p.r)
    xo, io = orc.gmres(A, b, defl=d, m=40, tol=1e-12, maxit=50000)
    assert relerr(xg.cpu().numpy(), xo) <= 1e-7


def test_mgs_limits(G, orc):
    p = W.workload1()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    with pytest.raises(G.GmresError):  # FP64 only
        gpu_solver_from_oracle(G, A, p.agg, p.r, ortho=G.ORTHO_MGS, precision=G.FP32_INNER)
    with pytest.raises(G.GmresError):
        gpu_solver_from_oracle(G, A, p.agg, p.r, ortho=7)
    with pytest.raises(G.GmresError):  # not with a BF16 basis
        gpu_solver_from_oracle(G, A, p.agg, p.r, ortho=G.ORTHO_MGS_LOWSYNC,
                               precision=G.BF16_BASIS)
    s = gpu_solver_from_oracle(G, A, p.agg, p.r, ortho=G.ORTHO_MGS)
    with pytest.raises(G.GmresError):  # the batched solve orthogonalises by CGS2
        G.batch_solve([s], [to_dev(b)], m=30, tol=1e-8, maxit=1000)


@pytest.mark.parametrize("mode", ["ebp", "none"])
def test_df32_multidot_fixed_iterations_match_oracle(G, orc, mode):
    """The double-FP32 multi-dot (FP32-pipe products and sums, error-free) in the fused
    one-reduction step: the oracle's FP64 MGS solution to 1e-9 after 47 fixed steps, and
    results that differ from the FP64-FMA multi-dot's (it ran) by rounding only."""
    p = W.convdiff(40, pe=25.0, sigma=0.5, seed=140, px=2, py=3)
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    defl = mode == "ebp"
    kw = dict(deflation_mode=G.DEFL_EBP if defl else G.DEFL_NONE, mu_mode=1, mu_user=5.0,
              fixed_iterations=True, ortho=G.ORTHO_MGS_LOWSYNC)
    agg, r = (p.agg, p.r) if defl else (None, 0)
    s = gpu_solver_from_oracle(G, A, agg, r, dot_arith=G.DOT_DF32, **kw)
    xg, ig = s.solve(to_dev(b), m=15, tol=0.0, maxit=47)
    s64 = gpu_solver_from_oracle(G, A, agg, r, **kw)
    x64, _ = s64.solve(to_dev(b), m=15, tol=0.0, maxit=47)
    d = orc.Deflation(A, p.agg, p.r) if defl else None
    xo, io = orc.gmres(A, b, defl=d, defl_mode=orc.DEFL_EBP if defl else orc.DEFL_NONE, m=15,
                       tol=0.0, maxit=47, mu_mode=1, mu_user=5.0, fixed_iterations=True,
                       ortho=orc.MGS)
    assert ig["iters"] == io["iters"] == 47
    assert relerr(xg.cpu().numpy(), xo) <= 1e-9
    assert ig["rel_res_est"] == pytest.approx(io["rel_res_est"], rel=1e-6, abs=1e-13)
    assert not torch.equal(xg, x64)
    assert relerr(xg.cpu().numpy(), x64.cpu().numpy()) <= 1e-10


def test_df32_multidot_to_tolerance_and_repeats(G, orc):
    p = W.workload1()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    s = gpu_solver_from_oracle(G, A, p.agg, p.r, ortho=G.ORTHO_MGS_LOWSYNC,
                               dot_arith=G.DOT_DF32)
    xg, ig = s.solve(to_dev(b), m=30, tol=1e-11, maxit=20000)
    xg2, ig2 = s.solve(to_dev(b), m=30, tol=1e-11, maxit=20000)
    d = orc.Deflation(A, p.agg, p.r)
    xo, io = orc.gmres(A, b, defl=d, m=30, tol=1e-11, maxit=20000, ortho=orc.MGS)
    assert ig["status"] == 0 and ig["rel_res_true"] <= 1e-11
    assert relerr(xg.cpu().numpy(), xo) <= 1e-9
    assert abs(ig["iters"] - io["iters"]) <= 2
    assert torch.equal(xg, xg2) and ig["iters"] == ig2["iters"]  # deterministic


def test_df32_multidot_limits(G, orc):
    p = W.workload1()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    with pytest.raises(G.GmresError):  # the one-reduction MGS only
        gpu_solver_from_oracle(G, A, p.agg, p.r, dot_arith=G.DOT_DF32)
    with pytest.raises(G.GmresError):  # FP64 solves only
        gpu_solver_from_oracle(G, A, p.agg, p.r, ortho=G.ORTHO_MGS_LOWSYNC,
                               precision=G.FP32_INNER, dot_arith=G.DOT_DF32)
    with pytest.raises(G.GmresError):
        gpu_solver_from_oracle(G, A, p.agg, p.r, ortho=G.ORTHO_MGS_LOWSYNC, dot_arith=2)
