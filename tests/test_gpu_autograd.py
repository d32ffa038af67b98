"""GPU parity of the differentiable solve (adjoint GMRES + element gradient) against a
dense adjoint built with numpy from the oracle's assembler, and against central finite
differences of the loss L = ||x(kappa) - x_target||^2 (workload q1-n512 recipe)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from helpers import relerr, to_dev

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


def _setup(G, orc, n, tol=1e-13):
    p, kstar = W.workload5(n)
    A_t, b = orc.q1_assemble(n, kstar, p.beta, p.f)
    x_target = spla.spsolve(A_t.to_scipy().tocsc(), b) if n <= 64 else None
    st = G.Q1Setup(n=n, beta=p.beta, agg=to_dev(p.agg), r=p.r, m=50, tol=tol, maxit=200000)
    return p, kstar, b, x_target, st


def test_gradient_vs_dense_adjoint_16x16(G, orc):
    n = 16
    p, kstar, b, xt, st = _setup(G, orc, n)
    kappa = to_dev(p.kappa).requires_grad_(True)
    bt = to_dev(b).requires_grad_(True)
    x = G.q1_solve(kappa, bt, st)
    loss = ((x - to_dev(xt)) ** 2).sum()
    loss.backward()
    # dense reference: x, lambda by LU; dA/dkappa_e by re-assembly (A is affine in kappa)
    A, _ = orc.q1_assemble(n, p.kappa, p.beta, p.f)
    Ad = A.to_scipy().toarray()
    xd = np.linalg.solve(Ad, b)
    lam = np.linalg.solve(Ad.T, 2.0 * (xd - xt))
    ref = np.empty(n * n)
    for e in range(n * n):
        kp = p.kappa.copy()
        kp[e] += 1.0
        Ae, _ = orc.q1_assemble(n, kp, p.beta, p.f)
        ref[e] = -lam @ ((Ae.to_scipy().toarray() - Ad) @ xd)
    assert relerr(x.detach().cpu().numpy(), xd) <= 1e-10
    assert relerr(kappa.grad.cpu().numpy(), ref) <= 1e-8
    assert relerr(bt.grad.cpu().numpy(), lam) <= 1e-8


def test_gradient_vs_finite_differences_16x16(G, orc):
    n = 16
    p, kstar, b, xt, st = _setup(G, orc, n)
    xt_d, b_d = to_dev(xt), to_dev(b)

    def loss(kap):
        return float(((G.q1_solve(to_dev(kap), b_d, st) - xt_d) ** 2).sum())

    kappa = to_dev(p.kappa).requires_grad_(True)
    ((G.q1_solve(kappa, b_d, st) - xt_d) ** 2).sum().backward()
    g = kappa.grad.cpu().numpy()
    rng = np.random.default_rng(20)
    # central differences: truncation error ~h^2, solver noise ~(tol * |x - x_t| * |x|) / h;
    # h = 1e-4 keeps both well below the 1e-5 relative bound (with h = 1e-6 the noise of
    # two independent 1e-13 solves is of the order of the bound itself)
    h = 1e-4
    for e in rng.choice(n * n, 16, replace=False):
        kp, km = p.kappa.copy(), p.kappa.copy()
        kp[e] += h
        km[e] -= h
        fd = (loss(kp) - loss(km)) / (2 * h)
        assert abs(fd - g[e]) <= 1e-5 * max(abs(g[e]), 1e-3 * np.abs(g).max())


def test_full_size_512_gradient_properties(G, orc):
    # q1-n512: the adjoint solution satisfies A^T lam = dL/dx (checked in FP64 on the
    # host), the element pass matches the oracle's on the same lam and x, and the
    # gradient matches a central-difference directional derivative of GPU solves
    n = 512
    p, kstar, b, _, st = _setup(G, orc, n, tol=1e-12)
    b_d = to_dev(b)
    import paper_1906_04051_gb300 as GG
    zeros = torch.zeros((n + 1) ** 2, dtype=torch.float64, device="cuda")
    r_t, c_t, v_t, _ = GG.q1_assemble(n, to_dev(kstar), p.beta, zeros)
    s_t = GG.Solver(r_t, c_t, v_t, to_dev(p.agg), p.r)
    xt, it = s_t.solve(b_d, m=50, tol=1e-12, maxit=200000)
    assert it["status"] == 0
    kappa = to_dev(p.kappa).requires_grad_(True)
    x = G.q1_solve(kappa, b_d, st)
    gx = 2.0 * (x.detach() - xt)
    ((x - xt) ** 2).sum().backward()
    A, _ = orc.q1_assemble(n, p.kappa, p.beta, p.f)
    At = A.transpose()
    s = GG.Solver(to_dev(A.rowptr), to_dev(A.col), to_dev(A.val), to_dev(p.agg), p.r)
    lam, il = s.adjoint_solve(gx, m=50, tol=1e-12, maxit=200000)
    lam_h, gx_h = lam.cpu().numpy(), gx.cpu().numpy()
    assert np.linalg.norm(At.matvec(lam_h) - gx_h) <= 1e-11 * np.linalg.norm(gx_h)
    g = kappa.grad.cpu().numpy()
    go = orc.q1_kappa_grad(n, lam_h, x.detach().cpu().numpy())
    assert relerr(g, go) <= 1e-9
    # directional derivative along a random perturbation of every kappa_e: its signal
    # sums all elements, so solver-tolerance noise stays far below it
    d = W.normal(77, 3, n * n)
    h = 1e-5
    vals = []
    for sgn in (1, -1):
        kk = p.kappa + sgn * h * d
        vals.append(float(((G.q1_solve(to_dev(kk), b_d, st) - xt) ** 2).sum()))
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd - g @ d) <= 1e-5 * abs(g @ d)
