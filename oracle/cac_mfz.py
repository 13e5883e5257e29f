"""Plain FP64 CPU oracle of CAC-MFZ-CDP (arXiv 2405.00366).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or call
this module.  The product path (the CUDA library and its Python binding) never
routes through it and shares no code with it.

It writes out the alternating minimisation of the paper step by step, in the
paper's order and notation, with NumPy in float64:

* Algorithm 1 (alternating minimisation): for each outer iteration i, draw
  fresh initial amplitudes, integrate the mean-field CIM with chaotic
  amplitude control to a support sigma, refit R on that support, update eta.
* Eq. mfeq1        dc_r/dt = (-1 + p - c_r^2) c_r + K (dc_r/dt)_inj
* Eq. MFZlocalfieldmain  (dc_r/dt)_inj = j e_r (R_r h_r - (eta^2/4) sqrt(tau))
* Eq. GMFZEC5      de_r/dt = -beta (c_r^2 - tau) e_r
* Eq. localfieldMFZ      continuous local field h_r
* Eq. localfieldMFZBN    binarised local field h_r^BN, sigma = H(c)
* Eq. pumprateGACS (sigmoid pump) and a linear pump ramp
* Eq. etaSchedulling (threshold schedule), eta = sqrt(2 lambda) when fixed
* Eq. doublel0     objective E = 1/2 ||y - A(sigma o R)||^2 + lambda ||sigma||_0

Readings where the paper is silent, stated here in full:

* R is defined for every r.  The refit on support S solves the normal
  equations G_SS R_S = (A^T y)_S; off the support R_r is the Jacobi fixed
  point (h^z_r - sum_{r' in S} G_rr' R_r') / G_rr.  The initial R is the same
  formula with an empty support, R = A^T y / diag(G).
* The Euler update is simultaneous: c and e at step n+1 are computed from c
  and e at step n; the pump is evaluated at t_n = n dt.
* H(0) = 0: a spin is on only when its amplitude is strictly positive.
* The linear pump is p(t_n) = p0 + (p1 - p0) n / S over the S steps of one
  CIM run, restarting each outer iteration.
* Initial amplitudes come from a counter-based generator built on the
  SplitMix64 finaliser (Steele, Lea & Flood, OOPSLA 2014), keyed by (seed,
  instance, trial, outer iteration, spin).
* Trials are independent alternating runs; the kept result is the trial of
  lowest energy, ties going to the lower trial index.
* G_SS counts as singular when a Cholesky pivot L_jj^2 is not above
  1e-12 G_jj (for |S| > M the exact pivots are zero and rounding alone would
  decide); it is then solved with a ridge G_SS + eps I,
  eps = 1e-10 * mean(G_rr over S), and flagged.

Pins: tests/test_oracle_pins.py checks this module against the brute-force
minimum over all supports, exact noise-free recovery, the separable case
A orthogonal (hard threshold, both fields), a hand-computed three-spin Euler
step, the symmetry and zero diagonal of J, the published SplitMix64 outputs,
the moments of the initial-amplitude distributions, the pump and eta
schedules at closed-form points, the Gram matrix by brute force, the
recomputed objective, the zero gradient of the exact refit, the ridge on a
singular support, the damped Jacobi refit (two sweeps worked by hand, and its
convergence to the exact refit), the conjugate-gradient refit (two iterations
worked by hand, convergence to the exact refit), the LASSO initial R (three
FISTA iterations worked by hand, the soft threshold of the separable case, the
optimality conditions at convergence), the corrected self-term (hand-worked step,
separable case, brute force against Eq. doublel0) and the best-configuration
readout (against the recorded trajectory scored by objective());
tests/test_oracle_mutations.py plants mistakes in it and checks that a pin
fails for each.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import scipy.linalg

__all__ = [
    "Params", "splitmix64_mix", "counter_uniform", "initial_amplitudes", "gram",
    "coupling_J", "pump", "eta_at", "local_field_cn", "local_field_bn", "injection",
    "euler_step", "self_term_correction", "readout_energy", "cim_run", "refit_exact", "refit_jacobi", "refit_cg",
    "lasso_fista",
    "objective", "rmse",
    "hamming_loss", "solve",
]

_MASK64 = (1 << 64) - 1
# SplitMix64 constants: the golden-ratio increment and the two multipliers of
# the finaliser (Steele, Lea & Flood 2014; Vigna's reference splitmix64.c).
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_MIX1 = 0xBF58476D1CE4E5B9
_MIX2 = 0x94D049BB133111EB


@dataclasses.dataclass
class Params:
    """Run parameters, named as in the paper (Methods, Numerical experiments)."""

    n_outer: int = 20            # outer iterations of Algorithm 1 (velo + 1 in the paper)
    n_steps: int = 1000          # Euler steps per CIM run
    dt: float = 0.01             # Euler step (the paper uses 0.02)
    pump_kind: str = "linear"    # "linear" (p0 -> p1) or "sigmoid" (Eq. pumprateGACS)
    p0: float = 0.0
    p1: float = 1.5
    p_thr: float = 1.0
    d: float = 0.4
    t0: float = 4.0
    width: float = 2.0
    beta: float = 0.2            # CAC feedback rate (Eq. GMFZEC5)
    tau: float = 1.0             # target amplitude
    K: float = 1.0               # feedback strength (Eq. mfeq1)
    j: float = 1.0               # out-coupling rate (Eq. MFZlocalfieldmain)
    eta_init: float = 0.0        # <= 0: fixed eta = sqrt(2 lambda)
    eta_end: float = 0.0
    velo: float = 51.0
    init_kind: str = "uniform"   # "uniform": U(-s, s); "normal": N(0, s^2)
    init_scale: float = 0.01
    field: str = "cn"            # "cn" continuous (Eq. localfieldMFZ), "bn" binarised
    refit: str = "exact"         # "exact" normal equations, "jacobi" damped Jacobi, "cg" conjugate gradient
    jacobi_dt: float = 0.1
    jacobi_iters: int = 100
    cg_iters: int = 10000        # conjugate-gradient refit: at most this many iterations (paper: 10000)
    cg_tol: float = 1e-10        # and until ||h^z_S - G_SS R_S||_2 <= cg_tol ||h^z_S||_2
    init_R: str = "zeeman"       # initial R: "zeeman" h^z / diag(G); "lasso" the LASSO solution (FISTA)
    lasso_lambda: float = 1e-3   # the LASSO's L1 weight
    lasso_iters: int = 500       # FISTA iterations
    seed: int = 0
    self_term: bool = False      # corrected mode: the injection also subtracts (sqrt tau / 4) G_rr R_r^2
    readout: str = "final"       # "final": H(c) at the end of each run; "best": the best configuration visited


# ---------------------------------------------------------------- random numbers
def splitmix64_mix(z):
    """SplitMix64 finaliser on uint64 values (mod 2^64 arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_MIX2)
        z = z ^ (z >> np.uint64(31))
    return z


def _add64(a, k):
    """(a + k) mod 2^64 for uint64 array a and Python int k."""
    with np.errstate(over="ignore"):
        return np.asarray(a, dtype=np.uint64) + np.uint64(k & _MASK64)


def _key(seed: int, inst: int, trial: int, outer: int) -> np.uint64:
    k = splitmix64_mix(np.uint64(seed & _MASK64))
    k = splitmix64_mix(_add64(k, GOLDEN_GAMMA * (inst + 1)))
    k = splitmix64_mix(_add64(k, GOLDEN_GAMMA * (trial + 1)))
    k = splitmix64_mix(_add64(k, GOLDEN_GAMMA * (outer + 1)))
    return k


def counter_uniform(seed: int, inst: int, trial: int, outer: int, r, lane: int = 0):
    """Uniform doubles in [0, 1) for spins r, from 53 high bits of a SplitMix64 word.

    word(r, lane) = mix(key + GAMMA * (2 r + lane + 1)), key chained from
    (seed, inst, trial, outer) by the same finaliser.
    """
    r = np.asarray(r, dtype=np.uint64)
    k = _key(seed, inst, trial, outer)
    with np.errstate(over="ignore"):
        ctr = np.uint64(2) * r + np.uint64(lane + 1)
        z = splitmix64_mix(k + np.uint64(GOLDEN_GAMMA) * ctr)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def initial_amplitudes(seed, inst, trial, outer, N, kind="uniform", scale=0.01):
    """c_r at the start of a CIM run (Algorithm 1; the paper draws N(0, 1e-4)).

    uniform: scale * (2u - 1);  normal: scale * sqrt(-2 ln(1 - u1)) cos(2 pi u2)
    (Box-Muller on two independent counter lanes).
    """
    r = np.arange(N)
    u1 = counter_uniform(seed, inst, trial, outer, r, 0)
    if kind == "uniform":
        return scale * (2.0 * u1 - 1.0)
    if kind == "normal":
        u2 = counter_uniform(seed, inst, trial, outer, r, 1)
        return scale * np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
    raise ValueError(kind)


# ---------------------------------------------------------------- problem data
def gram(A, y):
    """G = A^T A (G_rr' = sum_k A_r^k A_r'^k), A^T y and diag G (Eq. l0Hamiltonian).

    G is built from its upper triangle so that G_rr' and G_r'r are the same
    number, as the definition is symmetric in r, r'.
    """
    A = np.asarray(A, dtype=np.float64)
    G = A.T @ A
    G = np.triu(G) + np.triu(G, 1).T
    hz = A.T @ np.asarray(y, dtype=np.float64)
    g = np.diag(G).copy()
    return G, hz, g


def coupling_J(G, R):
    """The mutual coupling of the continuous field, J_rr' = -1/4 R_r G_rr' R_r' for r != r'.

    Eq. localfieldMFZ times R_r (Eq. MFZlocalfieldmain): the c-dependent part
    of R_r h_r is sum_r' J_rr' c_r'.  J has a zero diagonal.
    """
    Goff = G - np.diag(np.diag(G))
    return -0.25 * (R[:, None] * Goff * R[None, :])


# ---------------------------------------------------------------- schedules
def pump(n: int, prm: Params) -> float:
    """Pump rate at step n of a CIM run, t_n = n dt."""
    if prm.pump_kind == "linear":
        return prm.p0 + (prm.p1 - prm.p0) * n / prm.n_steps
    if prm.pump_kind == "sigmoid":  # Eq. pumprateGACS
        t = n * prm.dt
        return (prm.p_thr - prm.d) + 2.0 * prm.d / (1.0 + math.exp(-(t - prm.t0) / prm.width))
    raise ValueError(prm.pump_kind)


def eta_at(i: int, prm: Params, lam: float) -> float:
    """Threshold eta at outer iteration i (Eq. etaSchedulling); fixed sqrt(2 lambda) otherwise."""
    if prm.eta_init <= 0.0:
        return math.sqrt(2.0 * lam)
    return max(prm.eta_init * (1.0 - i / prm.velo), prm.eta_end)


# ---------------------------------------------------------------- the MFZ-CIM
def local_field_cn(Goff, R, c, hz, tau):
    """Eq. localfieldMFZ: h_r = -sum_{r'!=r} G_rr' R_r' (c_r' + sqrt tau)/4 + (sqrt tau / 2)(A^T y)_r.

    Columns of c (and R) are independent trials.
    """
    st = math.sqrt(tau)
    return -Goff @ (R * (c + st) / 4.0) + (st / 2.0) * hz[:, None]


def local_field_bn(Goff, R, c, hz, tau):
    """Eq. localfieldMFZBN: h_r = -(sqrt tau / 2)(sum_{r'!=r} G_rr' R_r' sigma_r' - (A^T y)_r), sigma = H(c)."""
    st = math.sqrt(tau)
    sigma = (c > 0.0).astype(np.float64)
    return -(st / 2.0) * (Goff @ (R * sigma) - hz[:, None])


def injection(j, e, R, h, eta, tau):
    """Eq. MFZlocalfieldmain: (dc_r/dt)_inj = j e_r (R_r h_r - (eta^2 / 4) sqrt tau)."""
    return j * e * (R * h - (eta * eta / 4.0) * math.sqrt(tau))


def self_term_correction(g, R, tau):
    """(sqrt tau / 4) G_rr R_r^2, subtracted inside the injection in corrected mode.

    The Hamiltonian of Eq. l0Hamiltonian has no self-term 1/2 G_rr R_r^2 sigma_r,
    so with R_r at its Jacobi fixed point the injection switches spin r on when
    G_rr R_r^2 > eta^2 / 2 = lambda, while Eq. doublel0 is lowered by it only
    when 1/2 G_rr R_r^2 > lambda.  Subtracting this term restores the objective's
    own single-spin decision (the discussion of Eq. MFZlocalfieldmain gives the
    field at the stationary amplitudes c = +-sqrt(tau))."""
    return (math.sqrt(tau) / 4.0) * g[:, None] * R * R


def readout_energy(Goff, g, hz, R, sigma, lam):
    """Eq. doublel0 at (R, sigma) less the constant 1/2 y^T y, per trial (columns):
    1/2 x^T G x - (A^T y)^T x + lam |sigma| with x = sigma o R and G = G_off + diag(g)."""
    x = sigma * R
    return 0.5 * np.sum(x * (Goff @ x), axis=0) + 0.5 * np.sum(g[:, None] * x * x, axis=0) \
        - hz @ x + lam * np.sum(sigma, axis=0)


def euler_step(c, e, p, inj, prm: Params):
    """One explicit Euler step of Eq. mfeq1 and Eq. GMFZEC5, both from the old (c, e)."""
    dc = (-1.0 + p - c * c) * c + prm.K * inj
    de = -prm.beta * (c * c - prm.tau) * e
    return c + prm.dt * dc, e + prm.dt * de


def cim_run(Goff, hz, R, eta, prm: Params, outer: int, inst: int = 0,
            record_steps: int = 0, max_steps: Optional[int] = None, g=None):
    """One CIM run (support estimation of Algorithm 1) for all trials (columns of R).

    Returns sigma (N, T) uint8, the final (c, e) and, if record_steps > 0, the
    amplitudes c and e after each of the first record_steps steps
    (shape (record_steps, N, T)).  max_steps stops the run early (a bounded
    sample for tests and timing; the schedules still refer to prm.n_steps).
    g = diag(G) is needed by the corrected mode and the "best" readout: the
    latter (the paper's future-work readout: compare the configurations visited
    rather than take the last) returns, per trial, the first of H(c_1), ...,
    H(c_S) with the lowest readout_energy at lambda = eta^2 / 2.
    """
    N, T = R.shape
    c = np.stack([initial_amplitudes(prm.seed, inst, t, outer, N, prm.init_kind, prm.init_scale)
                  for t in range(T)], axis=1)
    e = np.ones((N, T))
    rec_c = np.zeros((record_steps, N, T)) if record_steps else None
    rec_e = np.zeros((record_steps, N, T)) if record_steps else None
    field = local_field_cn if prm.field == "cn" else local_field_bn
    corr = self_term_correction(g, R, prm.tau) if prm.self_term else None
    best_E = np.full(T, np.inf)
    best_s = np.zeros((N, T), dtype=np.uint8)
    for n in range(prm.n_steps if max_steps is None else min(max_steps, prm.n_steps)):
        p = pump(n, prm)
        h = field(Goff, R, c, hz, prm.tau)
        inj = injection(prm.j, e, R, h, eta, prm.tau)
        if corr is not None:
            inj = inj - prm.j * e * corr
        c, e = euler_step(c, e, p, inj, prm)
        if n < record_steps:
            rec_c[n] = c
            rec_e[n] = e
        if prm.readout == "best":
            s = (c > 0.0).astype(np.uint8)
            E = readout_energy(Goff, g, hz, R, s, eta * eta / 2.0)
            better = E < best_E  # strict: the first configuration of the lowest energy is kept
            best_E = np.where(better, E, best_E)
            best_s[:, better] = s[:, better]
    sigma = (c > 0.0).astype(np.uint8)  # H(c), H(0) = 0
    if prm.readout == "best":
        sigma = best_s
    return sigma, c, e, rec_c, rec_e


# ---------------------------------------------------------------- the CDP refit
PIVOT_TOL = 1e-12


def _cholesky(Gss):
    """Lower Cholesky factor of Gss, or None when a pivot L_jj^2 is not above
    PIVOT_TOL * Gss_jj (numerically singular: e.g. |S| > M, where the exact pivots
    are zero and only rounding decides their sign)."""
    try:
        L = np.linalg.cholesky(Gss)
    except np.linalg.LinAlgError:
        return None
    if not np.all(np.diag(L) ** 2 > PIVOT_TOL * np.diag(Gss)):
        return None
    return L


def refit_exact(G, hz, g, sigma):
    """R minimising 1/2||y - A(sigma o R)||^2 on S = {r : sigma_r = 1}; Jacobi fixed point off S.

    G_SS R_S = hz_S by Cholesky; R_r = (hz_r - sum_{r' in S} G_rr' R_r') / g_r
    for r not in S.  Returns (R, singular) where singular says the ridge was used.
    """
    S = np.flatnonzero(sigma)
    R = np.empty_like(hz)
    singular = False
    if S.size:
        Gss = G[np.ix_(S, S)]
        L = _cholesky(Gss)
        if L is None:
            singular = True
            L = _cholesky(Gss + 1e-10 * np.mean(g[S]) * np.eye(S.size))
            if L is None:
                raise np.linalg.LinAlgError("ridge refit failed")
        z = scipy.linalg.solve_triangular(L, hz[S], lower=True)
        RS = scipy.linalg.solve_triangular(L.T, z, lower=False)
        R[S] = RS
        off = np.ones(hz.size, dtype=bool)
        off[S] = False
        R[off] = (hz[off] - G[np.ix_(off, S)] @ RS) / g[off]
    else:
        R[:] = hz / g
    return R, singular


def refit_jacobi(Goff, hz, g, sigma, R, dtc, iters):
    """Damped Jacobi CDP (paper, random data): R <- R + dtc (R~ - R),
    R~_r = (hz_r - sum_{r'!=r} G_rr' sigma_r' R_r') / g_r, for all r."""
    s = sigma.astype(np.float64)
    for _ in range(iters):
        Rt = (hz - Goff @ (s * R)) / g
        R = R + dtc * (Rt - R)
    return R


def refit_cg(G, hz, g, sigma, R, iters, tol):
    """CDP by conjugate gradient (paper, MRI data): the normal equations of the
    support, G_SS R_S = (A^T y)_S, by conjugate gradient warm started from the
    trial's R_S, at most `iters` iterations and until the residual is at most
    tol ||(A^T y)_S||; off the support R_r is the Jacobi fixed point, as for the
    exact refit."""
    S = np.flatnonzero(sigma)
    R = np.array(R, dtype=np.float64, copy=True)
    if S.size == 0:
        return hz / g
    Gss = G[np.ix_(S, S)]
    b = hz[S]
    x = R[S].copy()
    r = b - Gss @ x
    p = r.copy()
    rr = float(r @ r)
    bnorm = math.sqrt(float(b @ b))
    for _ in range(iters):
        if math.sqrt(rr) <= tol * bnorm:
            break
        q = Gss @ p
        alpha = rr / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(r @ r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    R[S] = x
    off = np.ones(hz.size, dtype=bool)
    off[S] = False
    R[off] = (hz[off] - G[np.ix_(off, S)] @ x) / g[off]
    return R


def lasso_fista(G, hz, lam1, iters):
    """The LASSO solution used as the initial R of the paper's MRI runs:
    argmin 1/2 x^T G x - (A^T y)^T x + lam1 ||x||_1 (= 1/2 ||y - A x||^2 + lam1 ||x||_1
    up to a constant) by FISTA (Beck & Teboulle 2009) from x = 0, `iters`
    iterations, step 1/L with L the largest absolute row sum of G (an upper
    bound of its largest eigenvalue)."""
    L = float(np.max(np.sum(np.abs(G), axis=1)))
    x = np.zeros_like(hz)
    z = x.copy()
    t = 1.0
    for _ in range(iters):
        v = z - (G @ z - hz) / L
        xn = np.sign(v) * np.maximum(np.abs(v) - lam1 / L, 0.0)
        tn = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z = xn + ((t - 1.0) / tn) * (xn - x)
        x, t = xn, tn
    return x


# ---------------------------------------------------------------- metrics
def objective(A, y, x_hat, sigma, lam):
    """Eq. doublel0 at (R, sigma): 1/2 ||y - A x_hat||^2 + lambda |sigma|, x_hat = sigma o R."""
    r = y - A @ x_hat
    return 0.5 * float(r @ r) + lam * float(np.sum(sigma))


def rmse(x_hat, x0):
    """sqrt(1/N sum (R_r sigma_r - x_r xi_r)^2) (Results, ground-state comparison)."""
    d = x_hat - x0
    return math.sqrt(float(d @ d) / d.size)


def hamming_loss(sigma, xi):
    """1/N sum |sigma_r - xi_r| (Discussion, difference in three fields)."""
    return float(np.mean(np.abs(sigma.astype(np.int64) - xi.astype(np.int64))))


# ---------------------------------------------------------------- Algorithm 1
def solve(A, y, lam, prm: Params, trials: int = 1, inst: int = 0,
          record_steps: int = 0, R_init: Optional[np.ndarray] = None,
          max_steps: Optional[int] = None):
    """Alternating minimisation (Algorithm 1) for `trials` independent trials.

    Returns a dict with the kept (lowest-energy) trial's x_hat, sigma, energy and
    index, every trial's R, sigma and energy, per-outer support sizes, every
    trial's sigma and R after each outer iteration (sigma_outer, R_outer:
    n_outer x N x T), a flag for ridge use and, with record_steps, the first
    steps' (c, e) of outer iteration 0.  max_steps truncates every CIM run (bounded samples only).
    """
    A = np.asarray(A, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    G, hz, g = gram(A, y)
    Goff = G - np.diag(g)
    N = G.shape[0]
    if R_init is None and prm.init_R == "lasso":
        R_init = lasso_fista(G, hz, prm.lasso_lambda, prm.lasso_iters)
    if R_init is None:
        R = np.repeat((hz / g)[:, None], trials, axis=1)
    else:
        R = np.repeat(np.asarray(R_init, dtype=np.float64)[:, None], trials, axis=1)
    sigma = np.zeros((N, trials), dtype=np.uint8)
    singular = False
    support_sizes = []
    sigma_outer, R_outer = [], []
    rec = None
    for i in range(prm.n_outer):
        eta = eta_at(i, prm, lam)
        sigma, c, e, rc, re = cim_run(Goff, hz, R, eta, prm, outer=i, inst=inst,
                                      record_steps=record_steps if i == 0 else 0,
                                      max_steps=max_steps, g=g)
        if i == 0 and record_steps:
            rec = (rc, re)
        for t in range(trials):
            if prm.refit == "exact":
                R[:, t], sing = refit_exact(G, hz, g, sigma[:, t])
                singular |= sing
            elif prm.refit == "cg":
                R[:, t] = refit_cg(G, hz, g, sigma[:, t], R[:, t], prm.cg_iters, prm.cg_tol)
            else:
                R[:, t] = refit_jacobi(Goff, hz, g, sigma[:, t], R[:, t],
                                       prm.jacobi_dt, prm.jacobi_iters)
        support_sizes.append(sigma.sum(axis=0).astype(np.int64))
        sigma_outer.append(sigma.copy())
        R_outer.append(R.copy())
    x_hats = sigma * R
    energies = np.array([objective(A, y, x_hats[:, t], sigma[:, t], lam) for t in range(trials)])
    best = int(np.argmin(energies))  # first index among equal minima
    return dict(
        x_hat=x_hats[:, best].copy(), sigma=sigma[:, best].copy(), energy=float(energies[best]),
        best_trial=best, energies=energies, R=R, sigmas=sigma,
        support_sizes=np.array(support_sizes), singular=singular,
        sigma_outer=np.array(sigma_outer), R_outer=np.array(R_outer),
        trajectory=rec, G=G, hz=hz, g=g,
    )
