"""GB300-native (sm_103a) deflated restarted GMRES(m) -- arXiv:1906.04051, Sec. 3.

The solver lives in a C-ABI CUDA library (include/gmres_gb300.h,
``libgmres_gb300.so``); this package only marshals arguments to it.  Importing the
package does not load the library; the first call does, and fails loudly if the library
has not been built (``python -m paper_1906_04051_gb300.build``).
"""
from ._native import (BF16_BASIS, DEFL_ADAPTIVE, DEFL_EBP, DEFL_NONE, DEFL_PROJECTOR,
                      DOT_DF32, DOT_FP64, FP32_INNER, FP64, MU_NORM_INF, MU_RITZ_FIRST_CYCLE, MU_USER, ORTHO_CGS2,
                      ORTHO_MGS, ORTHO_MGS_LOWSYNC, GmresError)
from .api import (Solver, batch_solve, bratu_newton, q1_assemble, q1_kappa_grad, q1_nnz,
                  q2_bratu_assemble, q2_nnz)

__all__ = [
    "Solver", "batch_solve", "q1_assemble", "q1_kappa_grad", "q1_nnz", "GmresError",
    "q2_bratu_assemble", "q2_nnz", "bratu_newton",
    "FP64", "FP32_INNER", "BF16_BASIS", "DEFL_EBP", "DEFL_PROJECTOR", "DEFL_NONE",
    "DEFL_ADAPTIVE",
    "MU_RITZ_FIRST_CYCLE", "MU_USER", "MU_NORM_INF", "ORTHO_CGS2", "ORTHO_MGS",
    "ORTHO_MGS_LOWSYNC", "DOT_FP64", "DOT_DF32",
]
from .autograd import GmresSolve, Q1Setup, q1_solve  # noqa: E402

__all__ += ["GmresSolve", "Q1Setup", "q1_solve"]
