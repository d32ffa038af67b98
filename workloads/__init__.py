"""Seeded synthetic inputs for the Q1 convection-diffusion systems.

This module is shared by the oracle side and the CUDA side and therefore holds none of
the method's arithmetic: no assembly, no solver step.  It only draws the PROBLEM DATA
that a user would hand to a solver: per-element coefficients kappa_e, the convection
vector beta, nodal load values f_i, nodal linearisation points u_k, and the aggregate
map that defines the deflation space W (one indicator column per aggregate).

Random numbers come from a counter-based SplitMix64 stream: value i of stream s under
seed S is mix(key(S, s) + (i + 1) * 0x9E3779B97F4A7C15), where mix is the SplitMix64
finaliser.  Uniforms take the top 53 bits; normals use the Box-Muller transform.
Default seeds are 1906040510 + workload number.

Workloads (2-D steady  -div(kappa grad u) + beta.grad u = f  on the unit square,
bilinear Q1 elements on an n x n mesh, homogeneous Dirichlet boundary, beta =
Pe (cos theta, sin theta) with theta = 0.3):
  1 "q1-n64"      n=64, kappa=1, Pe=10, manufactured f, 2x4 subdomains (r=8)
  2 "q1-n1024"    n=1024, kappa_e = exp(0.5 xi_e), Pe=100, f_i ~ U[-1,1], 32x32 aggregates
  3 "q1-n2048"    n=2048, kappa as 2, Pe=50, f_i ~ U[-1,1], 8x8 aggregates (r=64)
  4 "q1-batch256" 256 Picard-linearised systems, n_s = round(exp(U[ln 32, ln 256])),
                  Pe_s ~ U[1,200], kappa_e = 1 + (u_k at the element centre)^2,
                  u_k = sum_{p,q<=4} a_pq sin(p pi x) sin(q pi y), a_pq ~ N(0, 1/(p^2+q^2)),
                  load b = M 1 - K(u_k) u_k (f = 1, linearisation point u_k), 2x4 subdomains
  5 "q1-n512"     n=512, kappa_e = exp(0.3 xi_e) (trainable), target kappa*_e from an
                  independent stream, Pe=20, manufactured f, 16x16 aggregates
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1906040510
THETA = 0.3
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_KEYMUL = np.uint64(0xD1B54A32D192ED03)

# stream identifiers
S_KAPPA, S_F, S_KAPPA_STAR, S_SIZES, S_PE, S_UK, S_MISC = 1, 2, 3, 4, 5, 6, 7


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def raw_stream(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """count 64-bit words of stream `stream` under `seed`, starting at index offset."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^
                             (np.uint64(stream) * _KEYMUL)], dtype=np.uint64))[0]
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        return _mix(key + i * _GOLDEN)


def uniform(seed: int, stream: int, count: int, lo=0.0, hi=1.0) -> np.ndarray:
    """Uniform doubles in (lo, hi): (top 53 bits + 1/2) * 2^-53 mapped to [lo, hi]."""
    z = raw_stream(seed, stream, count)
    u = ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    u = uniform(seed, stream, 2 * count)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def node_xy(n: int):
    """Nodal coordinates, node (i, j) -> index j*(n+1)+i, x fastest."""
    t = np.arange(n + 1, dtype=np.float64) / n
    X, Y = np.meshgrid(t, t, indexing="xy")
    return X.reshape(-1), Y.reshape(-1)


def beta_vector(pe: float, theta: float = THETA):
    return (pe * math.cos(theta), pe * math.sin(theta))


def manufactured_u(n: int) -> np.ndarray:
    X, Y = node_xy(n)
    return np.sin(np.pi * X) * np.sin(np.pi * Y)


def manufactured_f(n: int, beta, kappa: float = 1.0) -> np.ndarray:
    """f = -kappa lap(u) + beta.grad(u) for u = sin(pi x) sin(pi y), at the nodes."""
    X, Y = node_xy(n)
    s = np.sin(np.pi * X) * np.sin(np.pi * Y)
    ux = np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
    uy = np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
    return 2.0 * np.pi ** 2 * kappa * s + beta[0] * ux + beta[1] * uy


def partition_agg(n: int, px: int, py: int) -> np.ndarray:
    """Aggregate of node (i,j): (i px)//(n+1) + px ((j py)//(n+1)); all nodes included."""
    i = np.arange(n + 1, dtype=np.int64)
    ax = (i * px) // (n + 1)
    ay = (i * py) // (n + 1)
    agg = ax[None, :] + px * ay[:, None]
    return agg.reshape(-1).astype(np.int32)


@dataclass
class Problem:
    """Data of one system: mesh size n, per-element kappa (n*n, element (ei,ej) at
    ej*n+ei), beta, nodal f, optional nodal linearisation point u, aggregate map."""
    name: str
    n: int
    kappa: np.ndarray
    beta: tuple
    f: np.ndarray
    agg: np.ndarray
    r: int
    u: np.ndarray | None = None
    m: int = 30
    tol: float = 1e-8
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return (self.n + 1) ** 2

    @property
    def nnz(self) -> int:
        return 9 * (self.n - 1) ** 2 + 4 * self.n


def convdiff(n: int, *, pe: float, sigma: float, seed: int, px: int, py: int,
             f_kind: str = "uniform", m: int = 30, tol: float = 1e-8, name=None) -> Problem:
    """Generic seeded Q1 convection-diffusion system (the recipe of workloads 1-3, 5)."""
    beta = beta_vector(pe)
    if sigma > 0.0:
        kappa = np.exp(sigma * normal(seed, S_KAPPA, n * n))
    else:
        kappa = np.ones(n * n)
    if f_kind == "uniform":
        f = uniform(seed, S_F, (n + 1) ** 2, -1.0, 1.0)
    elif f_kind == "manufactured":
        f = manufactured_f(n, beta)
    elif f_kind == "one":
        f = np.ones((n + 1) ** 2)
    else:
        raise ValueError(f_kind)
    return Problem(name or f"q1-n{n}", n, kappa, beta, f, partition_agg(n, px, py), px * py,
                   m=m, tol=tol)


def workload1(n: int = 64) -> Problem:
    return convdiff(n, pe=10.0, sigma=0.0, seed=BASE_SEED + 1, px=2, py=4,
                    f_kind="manufactured", m=30, tol=1e-8, name=f"q1-n{n}")


def workload2(n: int = 1024) -> Problem:
    return convdiff(n, pe=100.0, sigma=0.5, seed=BASE_SEED + 2, px=32, py=32,
                    f_kind="uniform", m=50, tol=1e-8, name=f"q1-n{n}")


def workload3(n: int = 2048) -> Problem:
    p = convdiff(n, pe=50.0, sigma=0.5, seed=BASE_SEED + 3, px=8, py=8, f_kind="uniform",
                 m=40, tol=1e-10, name=f"q1-n{n}")
    return p


def workload5(n: int = 512):
    """Returns (problem with kappa, kappa_star) for the differentiable-solve workload.
    Aggregates of about 32 x 32 nodes (16 x 16 at n = 512): with 2 x 4 subdomains the EBP
    deflated GMRES(50) stagnates at this size (relative residual 0.84 after the first
    cycle, in the oracle and on the GPU alike)."""
    seed = BASE_SEED + 5
    pxy = max(2, n // 32)
    p = convdiff(n, pe=20.0, sigma=0.3, seed=seed, px=pxy, py=pxy, f_kind="manufactured",
                 m=50, tol=1e-10, name=f"q1-n{n}")
    kappa_star = np.exp(0.3 * normal(seed, S_KAPPA_STAR, n * n))
    return p, kappa_star


def uk_field(n: int, coeffs) -> np.ndarray:
    """Smooth linearisation point u_k = sum_{p,q<=4} a_pq sin(p pi x) sin(q pi y), with
    a_pq = coeffs[(q-1)*4 + (p-1)] / sqrt(p^2 + q^2) for standard normal coeffs."""
    X, Y = node_xy(n)
    u = np.zeros_like(X)
    for q in range(1, 5):
        for p in range(1, 5):
            a = coeffs[(q - 1) * 4 + (p - 1)] / math.sqrt(p * p + q * q)
            u += a * np.sin(p * np.pi * X) * np.sin(q * np.pi * Y)
    return u


def workload4(count: int = 256, n_min: int = 32, n_max: int = 256, seed=None) -> list:
    """Batch of Picard-linearised systems -div((1+u_k^2) grad du) + beta.grad du = -R(u_k)."""
    seed = BASE_SEED + 4 if seed is None else seed
    us = uniform(seed, S_SIZES, count, math.log(n_min), math.log(n_max))
    sizes = np.clip(np.rint(np.exp(us)).astype(np.int64), n_min, n_max)
    pes = uniform(seed, S_PE, count, 1.0, 200.0)
    coeffs = normal(seed, S_UK, 16 * count).reshape(count, 16)
    out = []
    for s in range(count):
        n = int(sizes[s])
        uk = uk_field(n, coeffs[s])
        U = uk.reshape(n + 1, n + 1)
        centre = 0.25 * (U[:-1, :-1] + U[:-1, 1:] + U[1:, :-1] + U[1:, 1:])
        kappa = (1.0 + centre ** 2).reshape(-1)
        beta = beta_vector(float(pes[s]))
        out.append(Problem(f"q1-batch[{s}]-n{n}", n, kappa, beta, np.ones((n + 1) ** 2),
                           partition_agg(n, 2, 4), 8, u=uk, m=30, tol=1e-8,
                           extra={"pe": float(pes[s])}))
    return out


WORKLOADS = {1: workload1, 2: workload2, 3: workload3, 5: workload5}
