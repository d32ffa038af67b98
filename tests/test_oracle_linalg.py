"""Pins for the oracle's dense kernels: LU with partial pivoting and the Francis QR
eigenvalue iteration used for |mu| (Sec. 3.3, Ritz values of H_m)."""
import numpy as np
import pytest


@pytest.mark.parametrize("n", [1, 2, 7, 50])
def test_lu_matches_numpy_solve(orc, n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    lu, piv, info = orc.lu_factor(a)
    assert info == 0
    x = orc.lu_solve(lu, piv, b)
    np.testing.assert_allclose(x, np.linalg.solve(a, b), rtol=1e-11, atol=1e-12)


def test_lu_needs_pivoting_and_reports_singular(orc):
    a = np.array([[0.0, 1.0], [1.0, 1.0]])
    lu, piv, info = orc.lu_factor(a)
    assert info == 0 and list(piv) == [1, 1]
    np.testing.assert_allclose(orc.lu_solve(lu, piv, [1.0, 3.0]), [2.0, 1.0])
    s = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [0.0, 0.0, 1.0]])
    _, _, info = orc.lu_factor(s)
    assert info == 2


def _sorted(ev):
    return np.array(sorted(ev, key=lambda z: (round(z.real, 9), round(z.imag, 9))))


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (10, 3), (30, 4), (51, 5), (64, 6)])
def test_hessenberg_eigs_match_numpy(orc, n, seed):
    rng = np.random.default_rng(seed)
    h = np.triu(rng.standard_normal((n, n)), -1)
    got = orc.hessenberg_eigs(h)
    ref = np.linalg.eigvals(h)
    np.testing.assert_allclose(_sorted(got), _sorted(ref), rtol=0, atol=1e-10 * max(1, np.abs(h).max()))
    assert abs(np.abs(got).max() - np.abs(ref).max()) <= 1e-12 * np.abs(ref).max() * n


def test_hessenberg_eigs_companion_known_roots(orc):
    roots = np.array([0.5, -1.25, 2.0 + 1.0j, 2.0 - 1.0j, 3.0, -0.75 + 2.5j, -0.75 - 2.5j])
    coeffs = np.real(np.poly(roots))  # monic, highest power first
    n = len(roots)
    comp = np.zeros((n, n))
    comp[0, :] = -coeffs[1:]
    comp[1:, :-1] = np.eye(n - 1)  # upper Hessenberg companion form
    got = orc.hessenberg_eigs(comp)
    np.testing.assert_allclose(_sorted(got), _sorted(roots), atol=1e-11)
    assert abs(np.abs(got).max() - np.abs(roots).max()) < 1e-11


def test_hessenberg_eigs_gmres_like_matrix(orc):
    # a Hessenberg matrix with a tiny subdiagonal (near-breakdown) and repeated eigenvalues
    h = np.diag([2.0, 2.0, 2.0, 5.0, 1e-3]) + np.diag([1e-17, 1.0, 1e-12, 2.0], -1)
    h += np.triu(np.ones((5, 5)), 1)
    got = orc.hessenberg_eigs(h)
    ref = np.linalg.eigvals(h)
    np.testing.assert_allclose(np.sort(np.abs(got)), np.sort(np.abs(ref)), rtol=1e-6)
    assert abs(np.abs(got).max() - np.abs(ref).max()) < 1e-12 * 5
