"""Pins for the oracle's Q1 Galerkin assembly (Sec. 3.1, Eqs. 6-8).

Each pin is fixed by something other than the oracle: hand-derived closed-form stencils
(tests/golden/q1_stencils.txt), a brute-force count of the mesh connectivity, and the
O(h^2) nodal convergence of a manufactured solution solved with scipy's direct solver.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "q1_stencils.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        parts = line.split()
        out[parts[0]] = (parts[1], np.array([int(t) for t in parts[2:]], float).reshape(3, 3))
    return out


def _scale(s, h):
    s = s.replace("h^2", repr(h * h)).replace("h", repr(h))
    num, den = s.split("/")
    return float(eval(num)) / float(den)  # noqa: S307 -- fixed golden file


def _interior_row(A, n, i, j):
    np1 = n + 1
    row = j * np1 + i
    lo, hi = A.rowptr[row], A.rowptr[row + 1]
    assert hi - lo == 9
    out = np.zeros((3, 3))
    for k in range(lo, hi):
        c = A.col[k]
        dj, di = c // np1 - j, c % np1 - i
        out[dj + 1, di + 1] = A.val[k]
    return out


@pytest.mark.parametrize("n", [4, 8, 13])
def test_stencils_match_closed_form(orc, n):
    g = _golden()
    h = 1.0 / n
    N = (n + 1) ** 2
    zero_f = np.zeros(N)
    # diffusion only
    A, _ = orc.q1_assemble(n, np.ones(n * n), (0.0, 0.0), zero_f)
    # convection only (kappa = 0), unit beta_x then unit beta_y
    Ax, _ = orc.q1_assemble(n, np.zeros(n * n), (1.0, 0.0), zero_f)
    Ay, _ = orc.q1_assemble(n, np.zeros(n * n), (0.0, 1.0), zero_f)
    for (i, j) in [(1, 1), (n // 2, n // 2), (n - 1, 1), (2, n - 1)]:
        for mat, key in ((A, "diffusion"), (Ax, "convection_x"), (Ay, "convection_y")):
            s, pat = g[key]
            np.testing.assert_allclose(_interior_row(mat, n, i, j), _scale(s, h) * pat,
                                       rtol=0, atol=1e-15 * max(1.0, abs(_scale(s, h)) * 16))
    # mass: b = M f with f = delta at one interior node reproduces the mass stencil
    s, pat = g["mass"]
    i0, j0 = n // 2, n // 2
    f = np.zeros(N)
    f[j0 * (n + 1) + i0] = 1.0
    _, b = orc.q1_assemble(n, np.ones(n * n), (0.0, 0.0), f)
    got = np.zeros((3, 3))
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            got[dj + 1, di + 1] = b[(j0 + dj) * (n + 1) + i0 + di]
    np.testing.assert_allclose(got, _scale(s, h) * pat, rtol=1e-14, atol=0)
    # b = M 1 gives int(phi_i) = h^2 on interior nodes, 0 on Dirichlet rows
    _, b1 = orc.q1_assemble(n, np.ones(n * n), (0.0, 0.0), np.ones(N))
    B = b1.reshape(n + 1, n + 1)
    np.testing.assert_allclose(B[1:-1, 1:-1], h * h, rtol=1e-13)
    assert np.all(B[0, :] == 0) and np.all(B[-1, :] == 0)
    assert np.all(B[:, 0] == 0) and np.all(B[:, -1] == 0)


def test_element_matrices_exact_rationals(orc):
    # unit element (h = 1): K1 and M in exact rationals from the 1-D tables
    K1, Cm, M = orc.q1_element(1.0, 0.0, 0.0)
    S = [[1, -1], [-1, 1]]
    Mr = [[Fraction(1, 3), Fraction(1, 6)], [Fraction(1, 6), Fraction(1, 3)]]
    for a in range(2):
        for b in range(2):
            for c in range(2):
                for d in range(2):
                    i, j = a + 2 * b, c + 2 * d
                    assert K1[i, j] == pytest.approx(float(S[a][c] * Mr[b][d] + Mr[a][c] * S[b][d]), abs=1e-16)
                    assert M[i, j] == pytest.approx(float(Mr[a][c] * Mr[b][d]), abs=1e-16)
    # each row of the stiffness sums to zero (constants are in its null space)
    np.testing.assert_allclose(K1.sum(axis=1), 0.0, atol=1e-15)
    # the convection matrix annihilates constants: int phi_i beta.grad(1) = 0
    _, Cx, _ = orc.q1_element(0.5, 3.0, -2.0)
    np.testing.assert_allclose(Cx.sum(axis=1), 0.0, atol=1e-15)
    # and it integrates beta.grad(x) = beta_x exactly: sum_j C_ij x_j = beta_x int phi_i
    xs = np.array([0.0, 0.5, 0.0, 0.5])
    np.testing.assert_allclose(Cx @ xs, 3.0 * 0.25 * 0.25, rtol=1e-14)


def _brute_force_pattern(n):
    np1 = n + 1
    rows = [set() for _ in range(np1 * np1)]
    for ej in range(n):
        for ei in range(n):
            nodes = [(ej + b) * np1 + ei + a for b in (0, 1) for a in (0, 1)]
            for p in nodes:
                for q in nodes:
                    rows[p].add(q)
    for j in range(np1):
        for i in range(np1):
            if i in (0, n) or j in (0, n):
                rows[j * np1 + i] = {j * np1 + i}
    return rows


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16])
def test_pattern_is_mesh_connectivity(orc, n):
    rows = _brute_force_pattern(n)
    A, _ = orc.q1_assemble(n, np.ones(n * n), (1.0, 2.0), np.ones((n + 1) ** 2))
    assert A.nnz == sum(len(r) for r in rows) == orc.q1_nnz(n)
    for i, r in enumerate(rows):
        cols = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        assert list(cols) == sorted(r)


def test_nnz_of_workloads(orc):
    # 9 (n-1)^2 interior rows of nine entries + 4n Dirichlet rows of one entry
    expected = {64: 35_977, 1024: 9_422_857, 2048: 37_720_073, 512: 2_352_137, 16: 2_089}
    for n, nnz in expected.items():
        assert orc.q1_nnz(n) == nnz == 9 * (n - 1) ** 2 + 4 * n


def test_manufactured_solution_second_order(orc):
    import scipy.sparse.linalg as spla
    errs = []
    ns = [16, 32, 64, 128]
    for n in ns:
        p = W.workload1(n)
        A, b = orc.q1_assemble(n, p.kappa, p.beta, p.f)
        x = spla.spsolve(A.to_scipy().tocsc(), b)
        errs.append(np.abs(x - W.manufactured_u(n)).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(ns) - 1)]
    for o in orders:
        assert 1.8 <= o <= 2.2, orders


def test_linearised_load_sign(orc):
    # b = M f - K u: with u equal to the exact discrete solution of K u = M f the load
    # vanishes on interior rows
    import scipy.sparse.linalg as spla
    n = 12
    p = W.convdiff(n, pe=30.0, sigma=0.4, seed=99, px=2, py=2, f_kind="uniform")
    A, b = orc.q1_assemble(n, p.kappa, p.beta, p.f)
    u = spla.spsolve(A.to_scipy().tocsc(), b)
    _, b2 = orc.q1_assemble(n, p.kappa, p.beta, p.f, u)
    assert np.abs(b2).max() <= 1e-12 * np.abs(b).max()


def test_transpose_and_spmv(orc):
    rng = np.random.default_rng(0)
    p = W.convdiff(9, pe=40.0, sigma=0.5, seed=5, px=2, py=2)
    A, _ = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    S = A.to_scipy()
    x = rng.standard_normal(A.n)
    y = rng.standard_normal(A.n)
    np.testing.assert_allclose(A.matvec(x), S @ x, rtol=1e-14, atol=1e-14)
    At = A.transpose()
    np.testing.assert_array_equal(At.to_scipy().toarray(), S.T.toarray())
    assert abs(A.matvec(x) @ y - x @ At.matvec(y)) <= 1e-12 * np.abs(S).sum()
    for i in range(At.n):
        c = At.col[At.rowptr[i]:At.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
