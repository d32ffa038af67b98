"""Per-phase timing of one deflated GMRES solve (CUDA events from gmres_profile).

  python -m paper_1906_04051_gb300.phases --workload 2 --precision fp64 --steps 100
  python -m paper_1906_04051_gb300.phases --workload 3 --precision fp32 --tol 1e-10

With --steps the solve runs a fixed number of Arnoldi steps (fixed-iteration protocol,
user mu); with --tol it runs to that relative residual (Ritz mu).  The system is one of
the seeded Q1 workloads, assembled on the device.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np
import torch

from . import Solver, q1_assemble
from . import _native as N

PRECISIONS = {"fp64": N.FP64, "fp32": N.FP32_INNER, "bf16": N.BF16_BASIS}
ORTHOS = {"cgs2": N.ORTHO_CGS2, "mgs": N.ORTHO_MGS, "lowsync": N.ORTHO_MGS_LOWSYNC}


def load_workload(num: int, n: int | None = None):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import workloads as W
    fn = {1: W.workload1, 2: W.workload2, 3: W.workload3}[num]
    return fn(n) if n else fn()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--precision", default="fp64", choices=sorted(PRECISIONS))
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--maxit", type=int, default=50000)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--ortho", default="cgs2", choices=sorted(ORTHOS))
    args = ap.parse_args(argv)
    dev = torch.device("cuda")
    p = load_workload(args.workload, args.n)
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt,
                                                    device=dev)
    rowptr, col, val, b = q1_assemble(p.n, t(p.kappa), p.beta, t(p.f))
    fixed = args.steps is not None
    kw = dict(precision=PRECISIONS[args.precision], profile=True, ortho=ORTHOS[args.ortho])
    if fixed:
        kw.update(mu_mode=N.MU_USER, mu_user=50.0, fixed_iterations=True)
    s = Solver(rowptr, col, val, t(p.agg, torch.int32), p.r, **kw)
    for _ in range(args.repeat):
        s.profile(reset=True)
        x, info = s.solve(b, m=p.m, tol=0.0 if fixed else (args.tol or p.tol),
                          maxit=args.steps if fixed else args.maxit)
    prof = s.profile()
    out = {"workload": p.name, "precision": args.precision, "ortho": args.ortho, "m": p.m,
           "info": info,
           "us_per_step": 1e3 * info["ms_total"] / max(info["iters"], 1),
           "phases": {k: {"ms": round(v[0], 4), "launches": v[1],
                          "us_per_launch": round(1e3 * v[0] / v[1], 2) if v[1] else None}
                      for k, v in prof.items() if v[1]}}
    print(json.dumps(out))
    s.close()


if __name__ == "__main__":
    main()
