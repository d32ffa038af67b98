"""Algebraic facts the GPU kernels rely on, checked on the CPU with numpy/scipy and the
oracle: the one-reduction form of modified Gram-Schmidt (the product of the rank-1
projectors equals I - V (I + L)^-1 V^T, L the strictly lower part of V^T V), and the
drop step of the adaptive deflation taken in a Householder basis (the same subspace as
the oracle's complement basis Qc)."""
import numpy as np
import pytest

import oracle as orc


def test_mgs_projector_product_is_inverse_compact_wy():
    rng = np.random.default_rng(31)
    n, k = 60, 9
    V, _ = np.linalg.qr(rng.standard_normal((n, k)))
    V += 1e-3 * rng.standard_normal((n, k))  # not exactly orthonormal: the identity is exact
    V /= np.linalg.norm(V, axis=0)
    w = rng.standard_normal(n)
    x = w.copy()
    h_mgs = np.zeros(k)
    for c in range(k):  # modified Gram-Schmidt, one projection after the other
        h_mgs[c] = V[:, c] @ x
        x -= h_mgs[c] * V[:, c]
    L = np.tril(V.T @ V, -1)
    h = np.linalg.solve(np.eye(k) + L, V.T @ w)  # one reduction: V^T w, then (I + L) h = g
    assert np.abs(h - h_mgs).max() <= 1e-12
    assert np.abs((w - V @ h) - x).max() <= 1e-12


@pytest.mark.parametrize("seed,q", [(41, 5), (42, 12), (43, 20), (44, 32)])
def test_householder_drop_spans_the_oracle_complement(seed, q):
    import scipy.linalg as sla
    rng = np.random.default_rng(seed)
    T = rng.standard_normal((q, q))
    Qc, Tn, p = orc.adapt_drop(T)
    lam, YL = sla.eig(T, left=True, right=False)
    i = int(np.argmax(np.abs(lam)))
    Y = np.column_stack([YL[:, i].real, YL[:, i].imag]) if p == 2 else YL[:, i].real[:, None]
    # reflectors that map the columns of Y (after the earlier ones) onto single coordinates
    Q = np.eye(q)
    used = []
    Yw = Y.copy()
    for c in range(p):
        x = Yw[:, c].copy()
        x[used] = 0.0
        j = int(np.argmax(np.abs(x)))
        alpha = -np.linalg.norm(x) if x[j] >= 0 else np.linalg.norm(x)
        v = x.copy()
        v[j] -= alpha
        H = np.eye(q) - 2.0 * np.outer(v, v) / (v @ v)
        Yw = H @ Yw
        Q = Q @ H
        used.append(j)
    keep = [c for c in range(q) if c not in used]
    B = Q[:, keep]  # the kept basis, U B in the GPU's coordinates
    assert np.abs(B.T @ B - np.eye(q - p)).max() <= 1e-12
    # the same subspace as the oracle's complement: projectors agree
    assert np.abs(B @ B.T - Qc @ Qc.T).max() <= 1e-10
    # and the reduced T has the same eigenvalues
    ev1 = np.sort_complex(np.linalg.eigvals(B.T @ T @ B))
    ev2 = np.sort_complex(np.linalg.eigvals(Tn))
    assert np.allclose(ev1, ev2, rtol=1e-8, atol=1e-10)
