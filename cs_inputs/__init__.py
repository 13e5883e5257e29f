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
    "mri_full_instance",
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
    # 128 x 128 Haar-sparse image through a subsampled 2-D DCT (N=16384, M=4915),
    # 8 trials, FP16 storage; K = 0.1 as in the paper's MRI runs
    "mri_n16384_fp16": dict(
        mri_side=128, N=16384, M=4915, nnz=1638, nu=0.0, lam=0.1, seed=0, trials=8,
        n_outer=40, n_steps=3000, precision="fp16", **dict(_COMMON, K=0.1)),
    # the paper's random-data experiments (Numerical experiments): N = 2000,
    # alpha = 0.6, a = 0.2, nu = 0.05; sigmoid pump (Eq. pumprateGACS, p_thr = 1,
    # d = 0.4), dt = 0.02 up to 20 photon lifetimes, eta from 0.8 down to
    # eta_end = 0.18 (0.35 for nu = 0.1) with velo = 51, i.e. 52 outer
    # iterations (Eq. etaSchedulling), damped Jacobi CDP (0.1, 100 sweeps),
    # N(0, 1e-4) initial amplitudes, K = 1; the objective's lambda eta_end^2 / 2
    # the paper's MRI problem on a synthetic 128 x 128 image (mri_full_instance):
    # complex DFT observation (M_obs = 4915 points, compression 0.3), the
    # gamma = 1e-4 second-difference terms, the LASSO solution as the initial R,
    # sigmoid pump d = 0.6, fixed eta (eta_init = eta_end), 11 outer iterations
    # (velo), K = 0.1, the conjugate-gradient CDP; FP16 storage, 8 trials
    "mri_full_n16384": dict(
        mri_side=128, mri_gamma=1e-4, N=16384, M_obs=4915, M=2 * 4915 + 2 * 16384, nnz=1638, nu=0.0,
        lam=0.022 ** 2 / 2, seed=0, trials=8, n_outer=11, n_steps=1000, precision="fp16",
        **dict(_COMMON, dt=0.02, pump_kind="sigmoid", p_thr=1.0, d=0.6, t0=4.0, width=2.0, eta_init=0.022,
               eta_end=0.022, velo=11.0, init_kind="normal", init_scale=0.01, K=0.1, refit="cg",
               init_R="lasso", lasso_lambda=3e-4, lasso_iters=300)),
    "paper_random_n2000": dict(
        N=2000, M=1200, nnz=400, nu=0.05, lam=0.18 ** 2 / 2, seed=0, trials=1,
        n_outer=52, n_steps=1000, precision="fp32",
        **dict(_COMMON, dt=0.02, pump_kind="sigmoid", p_thr=1.0, d=0.4, t0=4.0, width=2.0, eta_init=0.8,
               eta_end=0.18, velo=51.0, init_kind="normal", init_scale=0.01, refit="jacobi", jacobi_dt=0.1,
               jacobi_iters=100)),
}


def workload(name: str, **overrides):
    """Parameters of a named workload with optional overrides."""
    w = dict(WORKLOADS[name])
    w.update(overrides)
    return w


def workload_instance(w) -> Instance:
    """The seeded instance of a workload dict."""
    if "mri_gamma" in w:
        return mri_full_instance(w["mri_side"], w["nnz"] / w["N"], w["M_obs"] / w["N"], w["mri_gamma"], w["lam"],
                                 w["seed"])
    if "mri_side" in w:
        return mri_instance(w["mri_side"], w["nnz"] / w["N"], w["M"] / w["N"], w["lam"], w["seed"])
    return random_instance(w["N"], w["M"], w["nnz"], w["nu"], w["lam"], w["seed"])


def haar_1d_matrix(n: int) -> np.ndarray:
    """Orthonormal multilevel 1-D Haar transform of length n (a power of two), as a
    matrix H1 with coefficients = H1 @ signal: averages and differences of
    neighbouring pairs scaled by 1/sqrt(2), applied again to the averages."""
    if n & (n - 1):
        raise ValueError("n must be a power of two")
    H = np.eye(n)
    m = n
    while m > 1:
        half = m // 2
        step = np.eye(n)
        blk = np.zeros((m, m))
        for k in range(half):
            blk[k, 2 * k] = blk[k, 2 * k + 1] = 1.0 / math.sqrt(2.0)
            blk[half + k, 2 * k] = 1.0 / math.sqrt(2.0)
            blk[half + k, 2 * k + 1] = -1.0 / math.sqrt(2.0)
        step[:m, :m] = blk
        H = step @ H
        m = half
    return H


def dct_1d_matrix(n: int) -> np.ndarray:
    """Orthonormal DCT-II matrix: row u is c_u cos(pi (2x + 1) u / (2n))."""
    x = np.arange(n)
    u = np.arange(n)[:, None]
    D = np.cos(math.pi * (2 * x[None, :] + 1) * u / (2 * n))
    D[0] *= math.sqrt(1.0 / n)
    D[1:] *= math.sqrt(2.0 / n)
    return D


def mri_instance(n_side: int = 128, sparsity: float = 0.1, alpha: float = 0.3, lam: float = 0.01,
                 seed: int = 0) -> Instance:
    """MRI-shaped synthetic problem (stand-in for the paper's brain image, which is
    not available): an n x n image sparse in the 2-D Haar domain, observed through
    a variable-density subsample of its orthonormal 2-D DCT.

    x0: a fraction `sparsity` of the N = n^2 Haar coefficients nonzero, positions
    uniform, values Laplace(0, 1).  The 2-D Haar transform is the separable one
    (the 1-D multilevel transform along each axis), so with image = Haar^T x0 and
    measured frequencies f_i = (u_i, v_i), row i of A = S DCT2 Haar^T is
    kron(H1 phi_u, H1 phi_v), phi_u the u-th DCT basis vector.  M = round(alpha N)
    frequencies are drawn without replacement with density
    p(u, v) ~ max(0.02, (1 - sqrt(u^2 + v^2) / (sqrt(2) n))^2), DC always kept.
    The rows of A are orthonormal; y = A x0 (noise-free).  Draw order: support,
    values, frequencies.
    """
    n = n_side
    N = n * n
    M = int(round(alpha * N))
    rng = np.random.default_rng(seed)
    K = int(round(sparsity * N))
    support = np.sort(rng.choice(N, size=K, replace=False))
    x0 = np.zeros(N)
    x0[support] = rng.laplace(0.0, 1.0, size=K)
    xi = np.zeros(N, dtype=np.uint8)
    xi[support] = 1
    u, v = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    dens = np.maximum(0.02, (1.0 - np.sqrt(u ** 2 + v ** 2) / (math.sqrt(2.0) * n)) ** 2).ravel()
    dens[0] = 0.0
    dens /= dens.sum()
    freq = np.concatenate([[0], rng.choice(N, size=M - 1, replace=False, p=dens)])
    H1 = haar_1d_matrix(n)
    B = H1 @ dct_1d_matrix(n).T  # column u = H1 phi_u
    fu, fv = freq // n, freq % n
    A = np.einsum("mi,mj->mij", B[:, fu].T, B[:, fv].T).reshape(M, N)
    y = A @ x0
    return Instance(A=np.ascontiguousarray(A), y=y, x0=x0, xi=xi, lam=float(lam))

def second_difference_matrix(n: int) -> np.ndarray:
    """Second-order difference along one axis of length n with zero padding outside
    the image: (D v)_i = v_{i-1} - 2 v_i + v_{i+1}, v_{-1} = v_n = 0."""
    return -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)


def mri_full_instance(n_side: int = 128, sparsity: float = 0.1, alpha: float = 0.3, gamma: float = 1e-4,
                      lam: float = 0.01, seed: int = 0) -> Instance:
    """The paper's MRI reconstruction problem (Eq. MRIl0init1 - MRIJMatrix1) on a
    synthetic image, as one real least-squares system the solver takes unchanged.

    The image x = Haar^T r is sparse in the 2-D Haar domain (a fraction `sparsity`
    of the N = n^2 coefficients r nonzero, Laplace(0, 1) values).  It is observed
    through M = round(alpha N) points of its orthonormal complex 2-D DFT, drawn
    without replacement with density ~ max(0.02, (1 - |f| / (sqrt(2) n / 2))^2)
    over the wrapped frequencies |f| = |(min(u, n-u), min(v, n-v))|, DC kept:
    y = S F Haar^T r (noise-free).  The objective 1/2 ||y - S F x||^2
    + gamma/2 ||Delta_v x||^2 + gamma/2 ||Delta_h x||^2 + lambda ||Haar x||_0 has,
    over r, the coupling G = Haar F^H S^T S F Haar^T + gamma Haar Delta_v^T Delta_v
    Haar^T + gamma Haar Delta_h^T Delta_h Haar^T (Eq. MRIJMatrix1; its real part,
    the image being real) and Zeeman term A^T y; both are the Gram data of
    A = [Re(S F Haar^T); Im(S F Haar^T); sqrt(gamma) Delta_v Haar^T;
    sqrt(gamma) Delta_h Haar^T] with y = [Re y; Im y; 0; 0] (2M + 2N rows).
    Delta_v, Delta_h: second differences along the image's rows and columns,
    zero padded.  Draw order: support, values, frequencies."""
    n = n_side
    N = n * n
    M = int(round(alpha * N))
    K = int(round(sparsity * N))
    rng = np.random.default_rng(seed)
    xi = np.zeros(N, dtype=np.uint8)
    xi[rng.choice(N, size=K, replace=False)] = 1
    x0 = np.zeros(N)
    x0[xi == 1] = rng.laplace(0.0, 1.0, size=K)
    u = np.arange(n)
    wu = np.minimum(u, n - u)
    rad = np.sqrt(wu[:, None] ** 2 + wu[None, :] ** 2).reshape(N)
    dens = np.maximum(0.02, (1.0 - rad / (math.sqrt(2.0) * n / 2.0)) ** 2)
    dens[0] = 0.0
    dens /= dens.sum()
    freq = np.concatenate([[0], rng.choice(N, size=M - 1, replace=False, p=dens)])
    H1 = haar_1d_matrix(n)
    F1 = np.exp(-2j * math.pi * np.outer(u, u) / n) / math.sqrt(n)
    B = H1 @ F1.T  # column u = H1 f_u (the DFT basis row f_u through the inverse Haar)
    fu, fv = freq // n, freq % n
    Ac = np.einsum("mi,mj->mij", B[:, fu].T, B[:, fv].T).reshape(M, N)
    D = second_difference_matrix(n)
    DH = D @ H1.T
    sg = math.sqrt(gamma)
    A = np.concatenate([Ac.real, Ac.imag, sg * np.kron(DH, H1.T), sg * np.kron(H1.T, DH)], axis=0)
    yc = Ac @ x0
    y = np.concatenate([yc.real, yc.imag, np.zeros(2 * N)])
    return Instance(A=np.ascontiguousarray(A), y=y, x0=x0, xi=xi, lam=float(lam))
