"""Seeded synthetic inputs for the L0-regularised compressed-sensing solver.

This module is shared by the FP64 oracle (``oracle/``), the tests and the
benchmark.  It holds only the *data* side: the observation model of the
paper's numerical experiments (Section "Numerical experiments", Eq.
observationmodelmatrix) and the run parameters of the standard workloads.  It
contains none of the solver's arithmetic (no local field, no Euler step, no
refit), so the oracle and the CUDA path stay independent of each other.

Every generator draws from NumPy's PCG64 (``numpy.random.default_rng(seed)``)
in a fixed order, so a seed names one instance on every machine.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np

__all__ = [
    "Instance",
    "random_instance",
    "uneven_batch",
    "WORKLOADS",
    "workload",
    "workload_instance",
]


@dataclasses.dataclass
class Instance:
    """One compressed-sensing problem y = A (xi o x0) + w.

    A   : (M, N) float64, row-major
    y   : (M,)   float64
    x0  : (N,)   float64, the source signal with zeros off the true support
    xi  : (N,)   uint8, the true support vector (1 where x0 is nonzero)
    lam : the L0 weight lambda of the objective (Eq. doublel0)
    """

    A: np.ndarray
    y: np.ndarray
    x0: np.ndarray
    xi: np.ndarray
    lam: float

    @property
    def M(self) -> int:
        return int(self.A.shape[0])

    @property
    def N(self) -> int:
        return int(self.A.shape[1])


def random_instance(N: int, M: int, n_nonzero: int, nu: float, lam: float, seed: int) -> Instance:
    """Random-data observation model of the paper (Eq. observationmodelmatrix).

    A has i.i.d. N(0, 1/M) entries, n_nonzero = a*N positions of the support xi are
    drawn uniformly without replacement, the source values there are N(0, 1),
    and the observation noise w is N(0, nu^2).  Draw order: A, support, values,
    noise.
    """
    K = n_nonzero
    if N < 1 or M < 1 or not (0 <= K <= N):
        raise ValueError(f"bad sizes N={N} M={M} n_nonzero={K}")
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, N)) / math.sqrt(M)
    support = np.sort(rng.choice(N, size=K, replace=False))
    x0 = np.zeros(N)
    x0[support] = rng.standard_normal(K)
    xi = np.zeros(N, dtype=np.uint8)
    xi[support] = 1
    w = nu * rng.standard_normal(M) if nu > 0 else np.zeros(M)
    y = A @ x0 + w
    return Instance(A=np.ascontiguousarray(A), y=y, x0=x0, xi=xi, lam=float(lam))


def uneven_batch(n_instances: int, n_min: int, n_max: int, alphas, sparsities,
                 nu: float, lam: float, seed: int) -> List[Instance]:
    """A batch of independent random instances of uneven size.

    N is uniform on [n_min, n_max]; alpha = M/N and a = K/N are drawn uniformly
    from the given lists.  Instance i is ``random_instance`` with seed
    (seed * 1_000_003 + i), so any instance can be regenerated on its own.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        N = int(rng.integers(n_min, n_max + 1))
        alpha = float(alphas[int(rng.integers(len(alphas)))])
        a = float(sparsities[int(rng.integers(len(sparsities)))])
        M = max(1, int(round(alpha * N)))
        K = max(1, int(round(a * N)))
        out.append(random_instance(N, M, K, nu, lam, seed * 1_000_003 + i))
    return out


# Run parameters of the standard workloads.  Keys follow the parameter names of
# the solver (cs_params in include/cs.h); the physics constants are those of the
# paper's random-data experiments where a workload does not set its own.
_COMMON = dict(
    dt=0.01, pump_kind="linear", p0=0.0, p1=1.5, beta=0.2, tau=1.0, K=1.0, j=1.0,
    init_kind="uniform", init_scale=0.01, field="cn", refit="exact",
)

WORKLOADS = {
    # single FP64 instance, N=200, M=120 (alpha=0.6), 20 nonzeros, noise-free
    "single_n200_fp64": dict(
        N=200, M=120, nnz=20, nu=0.0, lam=0.05, seed=0, trials=1,
        n_outer=20, n_steps=1000, precision="fp64", **_COMMON),
    # one N=2000, M=1200 instance with 200 nonzeros, 64 trials in one launch
    "trials64_n2000_fp32": dict(
        N=2000, M=1200, nnz=200, nu=0.01, lam=0.03, seed=0, trials=64,
        n_outer=30, n_steps=2000, precision="fp32", **_COMMON),
}


def workload(name: str, **overrides):
    """Parameters of a named workload with optional overrides."""
    w = dict(WORKLOADS[name])
    w.update(overrides)
    return w


def workload_instance(w) -> Instance:
    """The seeded instance of a workload dict."""
    return random_instance(w["N"], w["M"], w["nnz"], w["nu"], w["lam"], w["seed"])
