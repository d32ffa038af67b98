"""Shared test helpers: move seeded problems to the device and run both sides."""
import numpy as np


def to_dev(a, dtype=None):
    import torch
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a)
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def oracle_system(orc, p):
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f, p.u)
    return A, b


def gpu_solver_from_oracle(G, A, agg=None, r=0, **kw):
    """GPU handle on exactly the oracle's CSR (so only the solvers are compared)."""
    import torch
    rowptr = to_dev(A.rowptr)
    col = to_dev(A.col)
    val = to_dev(A.val)
    a = to_dev(agg.astype(np.int32)) if agg is not None else None
    return G.Solver(rowptr, col, val, a, r, **kw)
