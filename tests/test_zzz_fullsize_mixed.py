"""Parity at the full size of the mixed-precision system, in the configuration bench.py
times: q1-n2048 (4,198,401 DOF, 37,720,073 nnz), 8 x 8 aggregates (r = 64), GMRES(40)
with FP32 (or BF16-basis) inner cycles and FP64 refinement to a true relative residual
of 1e-10.  An oracle solve of this size does not finish in test time, so the check is a
property that holds at any size: the oracle's own FP64 SpMV recomputes b - A x for the
returned x, which must meet the tolerance and match the residual the solver reports.

Collected after every other GPU file (two solves of about 5 s each), so that a run
stopping at the first failure has run the others first."""
import numpy as np
import pytest

import workloads as W
from helpers import gpu_solver_from_oracle, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# b - A x is evaluated twice in FP64 with different summation orders (the oracle row by
# row, the library per diagonal), each with rounding errors of order eps || |A| |x| ||,
# about 300 eps ||b|| on these systems; at a residual of 1e-10 ||b|| that moves the
# computed norm in its last digits only, so a relative slack of 1e-3 is ample.
SLACK = 1e-3


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_04051_gb300 as G
    from paper_1906_04051_gb300 import build as B
    B.build()
    return G


@pytest.fixture(scope="module")
def system(orc):
    p = W.workload3()
    A, b = orc.q1_assemble(p.n, p.kappa, p.beta, p.f)
    return p, A, b


@pytest.mark.parametrize("name", ["fp32_inner", "bf16_basis"])
def test_full_size_mixed_precision_true_residual(G, orc, system, name):
    p, A, b = system
    assert (A.n, A.nnz, p.r, p.m) == (4198401, 37720073, 64, 40)
    prec = {"fp32_inner": G.FP32_INNER, "bf16_basis": G.BF16_BASIS}[name]
    s = gpu_solver_from_oracle(G, A, p.agg, p.r, precision=prec)
    xg, ig = s.solve(to_dev(b), m=p.m, tol=1e-10, maxit=60000)
    s.close()
    assert ig["status"] == 0, ig
    assert ig["refinements"] >= 1
    x = xg.cpu().numpy()
    rel = np.linalg.norm(b - A.matvec(x)) / np.linalg.norm(b)
    assert rel <= 1e-10 * (1 + SLACK)
    assert rel == pytest.approx(ig["rel_res_true"], rel=SLACK)
