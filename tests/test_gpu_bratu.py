"""GPU parity for the paper's benchmark problem, the 3-D Bratu equation on 27-node
hexahedra (Sec. 3.1, Eqs. 2-9): the device assembly against the oracle's (indices bit
for bit, values to rounding), GMRES on the Newton matrices (the lane-per-row CSR SpMV for
long rows) against the oracle's GMRES, and the device Newton iteration against an
oracle Newton iteration with direct solves."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from helpers import gpu_solver_from_oracle, relerr, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
LAM = 6.8  # the paper's lambda (Sec. 3.1)


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_04051_gb300 as G
    from paper_1906_04051_gb300 import build as B
    B.build()
    return G


def _u(n, seed):
    M = 2 * n + 1
    rng = np.random.default_rng(seed)
    u = 0.5 * rng.standard_normal(M ** 3)
    return u


@pytest.mark.parametrize("n,seed", [(1, None), (2, 11), (3, None), (4, 12)])
def test_assembly_matches_oracle(G, orc, n, seed):
    u = None if seed is None else _u(n, seed)
    A, b = orc.q2_bratu_assemble(n, LAM, u)
    rp, cl, vl, bg = G.q2_bratu_assemble(n, LAM, None if u is None else to_dev(u),
                                         device="cuda")
    assert G.q2_nnz(n) == orc.q2_nnz(n) == A.nnz
    assert np.array_equal(rp.cpu().numpy(), A.rowptr)
    assert np.array_equal(cl.cpu().numpy(), A.col)
    scale = np.abs(A.val).max()
    assert np.abs(vl.cpu().numpy() - A.val).max() <= 1e-13 * scale
    assert np.abs(bg.cpu().numpy() - b).max() <= 1e-13 * max(1.0, np.abs(b).max())


def test_assembly_table1_first_row(G, orc):
    # 31^3 nodes (n = 15): the first size of the paper's Table 1, 1,603,945 entries
    u = _u(15, 13) * 0.2
    A, b = orc.q2_bratu_assemble(15, LAM, u)
    rp, cl, vl, bg = G.q2_bratu_assemble(15, LAM, to_dev(u))
    assert int(rp[-1].item()) == 1603945 == A.nnz
    assert np.array_equal(rp.cpu().numpy(), A.rowptr)
    assert np.array_equal(cl.cpu().numpy(), A.col)
    assert np.abs(vl.cpu().numpy() - A.val).max() <= 1e-13 * np.abs(A.val).max()
    assert np.abs(bg.cpu().numpy() - b).max() <= 1e-13 * np.abs(b).max()
    # bitwise deterministic
    rp2, cl2, vl2, bg2 = G.q2_bratu_assemble(15, LAM, to_dev(u))
    assert torch.equal(vl, vl2) and torch.equal(bg, bg2)


def _agg3(n, bs):
    M = 2 * n + 1
    I = np.arange(M)
    nb = (M + bs - 1) // bs
    K, J, Ii = np.meshgrid(I, I, I, indexing="ij")
    agg = ((K // bs) * nb + (J // bs)) * nb + (Ii // bs)
    return agg.reshape(-1).astype(np.int32), nb ** 3


@pytest.mark.parametrize("mode", ["none", "ebp", "adaptive"])
def test_gmres_on_newton_matrix_matches_oracle(G, orc, mode):
    # fixed-iteration protocol on J(u) at a point near the solution: same steps, same x
    n = 3
    A, b = orc.q2_bratu_assemble(n, LAM, _u(n, 5) * 0.1)
    kw, okw = {}, {}
    agg, r = None, 0
    if mode == "none":
        kw["deflation_mode"] = G.DEFL_NONE
        okw["defl_mode"] = orc.DEFL_NONE
    elif mode == "ebp":
        agg, r = _agg3(n, 4)
    else:
        kw.update(deflation_mode=G.DEFL_ADAPTIVE, rmax=4)
        okw.update(defl_mode=orc.DEFL_ADAPTIVE, rmax=4)
    s = gpu_solver_from_oracle(G, A, agg, r, mu_mode=1, mu_user=3.0, fixed_iterations=True, **kw)
    assert s.layout()["spmv_lanes"] == 4  # 27..125 entries per row: lanes per row
    xg, ig = s.solve(to_dev(b), m=12, tol=0.0, maxit=60)
    d = orc.Deflation(A, agg, r) if r else None
    xo, io = orc.gmres(A, b, defl=d, m=12, tol=0.0, maxit=60, mu_mode=1, mu_user=3.0,
                       fixed_iterations=True, **okw)
    assert ig["iters"] == io["iters"] == 60
    assert relerr(xg.cpu().numpy(), xo) <= 1e-9
    assert ig["rel_res_true"] == pytest.approx(io["rel_res_true"], rel=1e-6, abs=1e-13)


def test_fp32_inner_on_newton_matrix(G, orc):
    n = 4
    A, b = orc.q2_bratu_assemble(n, LAM, _u(n, 6) * 0.1)
    s = gpu_solver_from_oracle(G, A, None, 0, deflation_mode=G.DEFL_NONE,
                               precision=G.FP32_INNER)
    xg, ig = s.solve(to_dev(b), m=30, tol=1e-10, maxit=20000)
    assert ig["status"] == 0 and ig["rel_res_true"] <= 1e-10
    xd = spla.spsolve(A.to_scipy().tocsc(), b)
    assert relerr(xg.cpu().numpy(), xd) <= 1e-7


def _oracle_newton(orc, n, tol=1e-12):
    u = np.zeros((2 * n + 1) ** 3)
    its = 0
    for _ in range(30):
        A, b = orc.q2_bratu_assemble(n, LAM, u)
        du = spla.spsolve(A.to_scipy().tocsc(), b)
        u += du
        its += 1
        if np.abs(du).max() <= tol:
            break
    return u, its


@pytest.mark.parametrize("mode", ["adaptive", "none"])
def test_newton_matches_oracle(G, orc, mode):
    n = 4
    uo, its = _oracle_newton(orc, n)
    kw = dict(deflation_mode=G.DEFL_ADAPTIVE) if mode == "adaptive" else dict(
        deflation_mode=G.DEFL_NONE)
    ug, info = G.bratu_newton(n, LAM, m=30, tol=1e-11, newton_tol=1e-10, **kw)
    assert info["status"] == 0, info
    assert abs(info["newton_iters"] - its) <= 1
    assert np.abs(ug.cpu().numpy() - uo).max() <= 1e-8
    assert info["gmres_iters"] == sum(info["step_iters"])
    # the update norms contract quadratically at the end
    du = info["step_du"]
    assert du[-1] <= 1e-10 and du[-2] <= 1e-3


def test_newton_with_subdomain_deflation(G, orc):
    n = 4
    uo, _ = _oracle_newton(orc, n)
    agg, r = _agg3(n, 3)
    ug, info = G.bratu_newton(n, LAM, m=30, tol=1e-11, newton_tol=1e-10,
                              agg=to_dev(agg), r=r, deflation_mode=G.DEFL_EBP)
    assert info["status"] == 0, info
    assert np.abs(ug.cpu().numpy() - uo).max() <= 1e-8


def test_newton_rejects_bad_arguments(G, orc):
    with pytest.raises(G.GmresError):
        G.bratu_newton(0, LAM)
    with pytest.raises(G.GmresError):
        G.q2_bratu_assemble(2, float("nan"), device="cuda")
