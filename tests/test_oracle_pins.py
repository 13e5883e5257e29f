"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test checks one part of oracle/cac_mfz.py against something the paper or
the mathematics fixes: published generator outputs, a hand-worked Euler step,
closed forms (the separable case reduces to hard thresholding), brute force over
every support, a library least-squares solver, and algebraic identities.
"""
import dataclasses
import itertools
import math
import os

import numpy as np
import pytest

import cs_inputs
import oracle
from oracle import Params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows[parts[0]] = parts[1:]
    return rows


# ------------------------------------------------------------------ generator
def test_splitmix64_published_outputs():
    rows = _read_golden("splitmix64_state0.txt")
    for k, (hexval,) in rows.items():
        z = (int(k) * 0x9E3779B97F4A7C15) & ((1 << 64) - 1)  # published increment
        assert int(oracle.splitmix64_mix(np.uint64(z))) == int(hexval, 16)


def test_initial_amplitude_distributions():
    N = 200_000
    u = oracle.initial_amplitudes(7, 0, 0, 0, N, "uniform", 0.01)
    assert u.min() >= -0.01 and u.max() < 0.01
    assert abs(u.mean()) < 3 * 0.01 / math.sqrt(3 * N) * 2
    assert abs(u.var() / (0.01 ** 2 / 3) - 1) < 0.02
    n = oracle.initial_amplitudes(7, 0, 0, 0, N, "normal", 0.01)
    assert abs(n.mean()) < 4 * 0.01 / math.sqrt(N)
    assert abs(n.std() / 0.01 - 1) < 0.01
    # fourth moment of a Gaussian is 3 sigma^4
    assert abs(np.mean(n ** 4) / (3 * 0.01 ** 4) - 1) < 0.05
    # different keys give unrelated streams
    a = oracle.initial_amplitudes(7, 0, 0, 0, 1000)
    for key in [(8, 0, 0, 0), (7, 1, 0, 0), (7, 0, 1, 0), (7, 0, 0, 1)]:
        b = oracle.initial_amplitudes(*key, 1000)
        assert abs(np.corrcoef(a, b)[0, 1]) < 0.15


# ------------------------------------------------------------------ problem data
def test_gram_brute_force_and_symmetry():
    inst = cs_inputs.random_instance(7, 5, 2, 0.1, 0.1, seed=3)
    G, hz, g = oracle.gram(inst.A, inst.y)
    M, N = inst.A.shape
    for r in range(N):
        assert hz[r] == pytest.approx(sum(inst.A[k, r] * inst.y[k] for k in range(M)), rel=1e-13, abs=1e-15)
        for rp in range(N):
            ref = sum(inst.A[k, r] * inst.A[k, rp] for k in range(M))
            assert G[r, rp] == pytest.approx(ref, rel=1e-13, abs=1e-15)
    big = cs_inputs.random_instance(300, 180, 30, 0.0, 0.1, seed=1)
    G, _, g = oracle.gram(big.A, big.y)
    assert np.array_equal(G, G.T)
    assert np.array_equal(np.diag(G), g)


def test_coupling_J_symmetric_zero_diagonal():
    inst = cs_inputs.random_instance(150, 90, 15, 0.0, 0.1, seed=2)
    G, hz, g = oracle.gram(inst.A, inst.y)
    R = np.random.default_rng(0).standard_normal(150)
    J = oracle.coupling_J(G, R)
    assert np.all(np.diag(J) == 0.0)
    np.testing.assert_allclose(J, J.T, rtol=4e-16, atol=0)
    # -4 D_R^-1 J D_R^-1 recovers G with its diagonal removed
    back = -4.0 * J / R[:, None] / R[None, :]
    Goff = G - np.diag(g)
    np.testing.assert_allclose(back, Goff, rtol=1e-15, atol=1e-300)
    # J c is the c-dependent part of R o h (Eq. localfieldMFZ times R_r)
    c = np.random.default_rng(1).uniform(-1, 1, 150)
    h1 = oracle.local_field_cn(Goff, R[:, None], c[:, None], hz, 1.0)[:, 0]
    h0 = oracle.local_field_cn(Goff, R[:, None], np.zeros((150, 1)), hz, 1.0)[:, 0]
    np.testing.assert_allclose(R * (h1 - h0), J @ c, rtol=1e-10, atol=1e-12)


# ------------------------------------------------------------------ schedules
def test_pump_and_eta_schedules():
    prm = Params(pump_kind="sigmoid", p_thr=1.0, d=0.4, t0=4.0, width=2.0, dt=0.02, n_steps=1000)
    # Eq. pumprateGACS: p(t0) = p_thr exactly; limits p_thr -/+ d
    assert oracle.pump(200, prm) == 1.0           # t = 200 * 0.02 = 4
    assert oracle.pump(0, prm) == pytest.approx(0.6 + 0.8 / (1 + math.exp(2.0)), rel=1e-15)
    assert oracle.pump(10 ** 6, prm) == pytest.approx(1.4, abs=1e-12)
    lin = Params(pump_kind="linear", p0=0.0, p1=1.5, n_steps=1000)
    assert oracle.pump(0, lin) == 0.0 and oracle.pump(500, lin) == 0.75 and oracle.pump(1000, lin) == 1.5
    # Eq. etaSchedulling with the paper's random-data constants
    sch = Params(eta_init=0.8, eta_end=0.18, velo=51)
    assert oracle.eta_at(0, sch, 0.0) == 0.8
    assert oracle.eta_at(10, sch, 0.0) == pytest.approx(0.8 * 41 / 51, rel=1e-15)
    assert oracle.eta_at(39, sch, 0.0) == pytest.approx(0.8 * 12 / 51, rel=1e-15)  # 0.188 > 0.18
    assert oracle.eta_at(40, sch, 0.0) == 0.18
    assert oracle.eta_at(51, sch, 0.0) == 0.18
    # fixed threshold eta = sqrt(2 lambda)
    assert oracle.eta_at(3, Params(), 0.05) == pytest.approx(math.sqrt(0.1), rel=1e-15)


# ------------------------------------------------------------------ one Euler step
def test_three_spin_hand_worked_step():
    gold = {k: np.array([float(v) for v in vals]) for k, vals in _read_golden("three_spin_step.txt").items()}
    G = np.array([[1.0, 0.5, -0.25], [0.5, 2.0, 0.0], [-0.25, 0.0, 1.5]])
    Goff = G - np.diag(np.diag(G))
    R = np.array([[1.0], [2.0], [-1.0]])
    c = np.array([[0.1], [-0.2], [0.0]])
    e = np.array([[1.0], [1.0], [2.0]])
    hz = np.array([0.5, -1.0, 0.25])
    prm = Params(tau=1.0, K=1.0, j=1.0, beta=0.2, dt=0.1)
    eta, p = 1.0, 0.5
    for field, fn in [("cn", oracle.local_field_cn), ("bn", oracle.local_field_bn)]:
        h = fn(Goff, R, c, hz, 1.0)
        np.testing.assert_allclose(h[:, 0], gold["h_" + field], rtol=0, atol=1e-15)
        inj = oracle.injection(1.0, e, R, h, eta, 1.0)
        np.testing.assert_allclose(inj[:, 0], gold["inj_" + field], rtol=0, atol=1e-15)
        c1, e1 = oracle.euler_step(c, e, p, inj, prm)
        np.testing.assert_allclose(c1[:, 0], gold["c_" + field], rtol=0, atol=1e-15)
        np.testing.assert_allclose(e1[:, 0], gold["e_next"], rtol=0, atol=1e-15)
        # corrected mode: the self-term restored inside the injection
        corr = oracle.self_term_correction(np.diag(G), R, 1.0)
        np.testing.assert_allclose(corr[:, 0], gold["corr"], rtol=0, atol=1e-15)
        inj_c = inj - 1.0 * e * corr
        np.testing.assert_allclose(inj_c[:, 0], gold["inj_" + field + "_corr"], rtol=0, atol=1e-15)
        c2, _ = oracle.euler_step(c, e, p, inj_c, prm)
        np.testing.assert_allclose(c2[:, 0], gold["c_" + field + "_corr"], rtol=0, atol=1e-15)


# ------------------------------------------------------------------ refit
def test_refit_matches_lstsq_and_is_jacobi_fixed_point():
    inst = cs_inputs.random_instance(120, 80, 12, 0.05, 0.1, seed=5)
    G, hz, g = oracle.gram(inst.A, inst.y)
    rng = np.random.default_rng(9)
    for size in [0, 1, 5, 30, 60]:
        sigma = np.zeros(120, dtype=np.uint8)
        sigma[rng.choice(120, size, replace=False)] = 1
        R, singular = oracle.refit_exact(G, hz, g, sigma)
        assert not singular
        S = np.flatnonzero(sigma)
        if size:
            ref, *_ = np.linalg.lstsq(inst.A[:, S], inst.y, rcond=None)
            np.testing.assert_allclose(R[S], ref, rtol=1e-9, atol=1e-11)
            grad = inst.A[:, S].T @ (inst.y - inst.A[:, S] @ R[S])
            assert np.max(np.abs(grad)) <= 1e-10 * np.linalg.norm(hz)
        # every coordinate satisfies g_r R_r + sum_{r' in S, r' != r} G_rr' R_r' = hz_r
        lhs = g * R + (G - np.diag(g)) @ (sigma * R)
        np.testing.assert_allclose(lhs, hz, rtol=1e-10, atol=1e-12)


def test_refit_singular_support_uses_ridge():
    inst = cs_inputs.random_instance(40, 10, 3, 0.0, 0.1, seed=6)
    G, hz, g = oracle.gram(inst.A, inst.y)
    sigma = np.ones(40, dtype=np.uint8)  # |S| = 40 > M = 10: G_SS has rank 10
    R, singular = oracle.refit_exact(G, hz, g, sigma)
    assert singular
    assert np.all(np.isfinite(R))
    # the ridge solution interpolates y (residual ~ 0) like the minimum-norm solution
    assert np.linalg.norm(inst.y - inst.A @ R) < 1e-4 * np.linalg.norm(inst.y)
    mn = np.linalg.pinv(inst.A) @ inst.y
    np.testing.assert_allclose(R, mn, rtol=0, atol=1e-3 * np.abs(mn).max())


def jacobi_golden():
    rows = {}
    with open(os.path.join(GOLDEN, "jacobi_two_sweeps.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#") and not line.startswith("name"):
                name, *vals = line.split()
                rows[name] = np.array([float(v) for v in vals])
    return rows


def test_damped_jacobi_two_sweeps_hand_worked():
    """The damped step R <- R + dtc (R~ - R) and the sweep count, against two sweeps
    worked by hand (tests/golden/jacobi_two_sweeps.txt)."""
    G = np.array([[2.0, 0.5, -0.25], [0.5, 1.0, 0.0], [-0.25, 0.0, 4.0]])
    g = np.diag(G).copy()
    hz = np.array([0.5, -1.0, 0.25])
    sigma = np.array([1, 1, 0], dtype=np.uint8)
    R0 = np.array([1.0, 2.0, -1.0])
    gold = jacobi_golden()
    for iters, key in ((1, "R1"), (2, "R2")):
        R = oracle.refit_jacobi(G - np.diag(g), hz, g, sigma, R0.copy(), 0.1, iters)
        np.testing.assert_allclose(R, gold[key], rtol=0, atol=1e-15)


def test_cg_refit_two_steps_hand_worked():
    """Conjugate gradient on a 2 x 2 support from the trial's R: the first iterate
    and the exact second one (tests/golden/cg_two_steps.txt); spin 3 is off the
    support and takes the Jacobi fixed point."""
    gold = {k: np.array([float(v) for v in vals]) for k, vals in _read_golden("cg_two_steps.txt").items()}
    G = np.array([[4.0, 1.0, 0.5], [1.0, 3.0, -1.0], [0.5, -1.0, 2.0]])
    g = np.diag(G).copy()
    hz = np.array([1.0, 2.0, 0.25])
    sigma = np.array([1, 1, 0], dtype=np.uint8)
    R0 = np.array([2.0, 1.0, 7.0])
    for iters, key in ((1, "x1"), (2, "x2")):
        R = oracle.refit_cg(G, hz, g, sigma, R0, iters, 0.0)
        np.testing.assert_allclose(R[:2], gold[key], rtol=0, atol=1e-15)
        assert R[2] == pytest.approx((0.25 - 0.5 * R[0] + 1.0 * R[1]) / 2.0, abs=1e-15)
    # the iteration stops once the residual meets the tolerance: a third step changes nothing
    R3 = oracle.refit_cg(G, hz, g, sigma, R0, 3, 1e-12)
    np.testing.assert_allclose(R3[:2], gold["x2"], rtol=0, atol=1e-15)


def test_cg_refit_converges_to_exact():
    inst = cs_inputs.random_instance(150, 90, 15, 0.05, 0.1, seed=8)
    G, hz, g = oracle.gram(inst.A, inst.y)
    rng = np.random.default_rng(3)
    for size in (1, 10, 40, 80):
        sigma = np.zeros(150, dtype=np.uint8)
        sigma[rng.choice(150, size, replace=False)] = 1
        exact, _ = oracle.refit_exact(G, hz, g, sigma)
        R = oracle.refit_cg(G, hz, g, sigma, hz / g, 10000, 1e-12)
        np.testing.assert_allclose(R, exact, rtol=0, atol=1e-8 * np.abs(exact).max())


def test_fista_three_steps_hand_worked():
    """Three FISTA iterations of the LASSO on a 2 x 2 problem (tests/golden/fista_three_steps.txt)."""
    gold = {k: np.array([float(v) for v in vals]) for k, vals in _read_golden("fista_three_steps.txt").items()}
    G = np.array([[2.0, 1.0], [1.0, 2.0]])
    hz = np.array([3.0, 1.0])
    for iters, key in ((1, "x1"), (2, "x2"), (3, "x3")):
        np.testing.assert_allclose(oracle.lasso_fista(G, hz, 0.5, iters), gold[key], rtol=0, atol=1e-15)


def test_fista_separable_case_is_the_soft_threshold():
    """G = I: the LASSO solution is the soft threshold of A^T y by lam1, reached
    after one iteration (L = 1) and kept."""
    rng = np.random.default_rng(12)
    hz = rng.standard_normal(40)
    for iters in (1, 5):
        x = oracle.lasso_fista(np.eye(40), hz, 0.3, iters)
        np.testing.assert_allclose(x, np.sign(hz) * np.maximum(np.abs(hz) - 0.3, 0.0), rtol=0, atol=1e-15)


def test_fista_meets_the_lasso_optimality_conditions():
    """At convergence the subgradient conditions hold: (A^T y - G x)_r = lam1 sign(x_r)
    on the support and |(A^T y - G x)_r| <= lam1 off it."""
    inst = cs_inputs.random_instance(120, 80, 12, 0.05, 0.1, seed=13)
    G, hz, g = oracle.gram(inst.A, inst.y)
    lam1 = 0.05
    x = oracle.lasso_fista(G, hz, lam1, 20000)
    grad = hz - G @ x
    on = x != 0
    assert on.any() and (~on).any()
    np.testing.assert_allclose(grad[on], lam1 * np.sign(x[on]), rtol=0, atol=1e-8)
    assert np.abs(grad[~on]).max() <= lam1 + 1e-8


def test_jacobi_refit_converges_to_exact():
    inst = cs_inputs.random_instance(100, 70, 10, 0.05, 0.1, seed=8)
    G, hz, g = oracle.gram(inst.A, inst.y)
    sigma = inst.xi.copy()
    exact, _ = oracle.refit_exact(G, hz, g, sigma)
    R = oracle.refit_jacobi(G - np.diag(g), hz, g, sigma, hz / g, 0.1, 4000)
    np.testing.assert_allclose(R, exact, rtol=0, atol=1e-8)


# ------------------------------------------------------------------ objective
def test_objective_matches_hamiltonian_identity():
    """Eq. doublel0 = 1/2 y^T y + H (Eq. l0Hamiltonian) + 1/2 sum_r G_rr R_r^2 sigma_r."""
    inst = cs_inputs.random_instance(9, 6, 3, 0.1, 0.07, seed=11)
    rng = np.random.default_rng(2)
    R = rng.standard_normal(9)
    sigma = rng.integers(0, 2, 9).astype(np.uint8)
    A, y, lam = inst.A, inst.y, inst.lam
    M, N = A.shape
    H = 0.0
    for r in range(N):
        for rp in range(r + 1, N):
            H += sum(A[k, r] * A[k, rp] for k in range(M)) * R[r] * R[rp] * sigma[r] * sigma[rp]
        H -= sum(y[k] * A[k, r] for k in range(M)) * R[r] * sigma[r]
        H += lam * sigma[r]
    self_term = 0.5 * sum(sum(A[k, r] ** 2 for k in range(M)) * R[r] ** 2 * sigma[r] for r in range(N))
    E = oracle.objective(A, y, sigma * R, sigma, lam)
    assert E == pytest.approx(0.5 * float(y @ y) + H + self_term, rel=1e-12)
    # plain loop form of the objective itself
    res = [y[k] - sum(A[k, r] * sigma[r] * R[r] for r in range(N)) for k in range(M)]
    assert E == pytest.approx(0.5 * sum(v * v for v in res) + lam * sigma.sum(), rel=1e-13)


def test_metrics():
    x0 = np.array([0.0, 1.0, -2.0, 0.0])
    xh = np.array([0.0, 1.5, -2.0, 0.5])
    assert oracle.rmse(xh, x0) == pytest.approx(math.sqrt((0.25 + 0.25) / 4))
    assert oracle.hamming_loss(np.array([0, 1, 1, 1]), np.array([0, 1, 1, 0])) == 0.25


# ------------------------------------------------------------------ whole method
def _separable(N, lam, seed):
    """A orthogonal (M = N): G = I, the spins decouple and R = A^T y."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    thr = math.sqrt(lam)
    mags = np.concatenate([rng.uniform(0.0, thr * 0.85, N // 3),
                           rng.uniform(thr * 1.15, math.sqrt(2 * lam) * 0.97, N // 3),
                           rng.uniform(math.sqrt(2 * lam) * 1.05, 1.5, N - 2 * (N // 3))])
    hz = mags * rng.choice([-1.0, 1.0], N)
    rng.shuffle(hz)
    y = Q @ hz
    return Q, y, hz


@pytest.mark.parametrize("field", ["cn", "bn"])
def test_separable_case_corrected_mode_is_the_objective_threshold(field):
    """Corrected mode (self-term restored): with G = I the support is the hard
    threshold of Eq. doublel0 itself, {r : |(A^T y)_r| > sqrt(2 lambda)} (the L0
    proximal operator), and R = A^T y."""
    lam = 0.05
    A, y, hz = _separable(60, lam, seed=4)
    prm = Params(n_outer=2, n_steps=1000, dt=0.01, field=field, seed=1, self_term=True)
    res = oracle.solve(A, y, lam, prm, trials=2)
    expect = (hz ** 2 > 2 * lam).astype(np.uint8)
    for t in range(2):
        np.testing.assert_array_equal(res["sigmas"][:, t], expect)
        np.testing.assert_allclose(res["R"][:, t], hz, rtol=0, atol=1e-12)


@pytest.mark.parametrize("field", ["cn", "bn"])
def test_separable_case_is_hard_threshold(field):
    """With G = I the dynamics reduce to one scalar ODE per spin whose injection has
    the sign of hz_r^2 - lambda (paper-literal Hamiltonian without the self-term),
    so the final support is the hard threshold {r : |(A^T y)_r| > sqrt(lambda)} and
    R = A^T y (the L0 proximal operator with threshold sqrt(lambda))."""
    lam = 0.05
    A, y, hz = _separable(60, lam, seed=4)
    prm = Params(n_outer=2, n_steps=1000, dt=0.01, field=field, seed=1)
    res = oracle.solve(A, y, lam, prm, trials=2)
    expect = (hz ** 2 > lam).astype(np.uint8)
    for t in range(2):
        np.testing.assert_array_equal(res["sigmas"][:, t], expect)
        np.testing.assert_allclose(res["R"][:, t], hz, rtol=0, atol=1e-12)
    # the set is strictly larger than the minimiser of Eq. doublel0 (threshold sqrt(2 lambda))
    assert expect.sum() > (hz ** 2 > 2 * lam).sum()


def _all_supports_min(A, y, lam_eff):
    """min over every sigma of 1/2 ||y - A_S R_S||^2 + lam_eff |S|, R_S by numpy lstsq."""
    M, N = A.shape
    best, arg = float(0.5 * y @ y), ()
    for size in range(1, N + 1):
        for S in itertools.combinations(range(N), size):
            S = list(S)
            RS, *_ = np.linalg.lstsq(A[:, S], y, rcond=None)
            r = y - A[:, S] @ RS
            E = 0.5 * float(r @ r) + lam_eff * size
            if E < best - 1e-12:
                best, arg = E, tuple(S)
    return best, arg


def brute_force_hits(n_seeds=12, trials=4):
    """Seeds (of n_seeds) on which the kept support is the brute-force minimiser.

    N = 12, M = 8, paper schedules (sigmoid pump, Eq. etaSchedulling from 0.8
    down to sqrt(2 lambda)).  Asserts on every trial that the dynamics never
    beat the brute-force minimum.
    """
    hits = 0
    for seed in range(n_seeds):
        inst = cs_inputs.random_instance(12, 8, 3, 0.05, 0.04, seed=100 + seed)
        prm = Params(n_outer=12, n_steps=1000, dt=0.02, pump_kind="sigmoid", eta_init=0.8,
                     eta_end=math.sqrt(2 * inst.lam), velo=8, seed=seed)
        res = oracle.solve(inst.A, inst.y, inst.lam, prm, trials=trials)
        best, arg = _all_supports_min(inst.A, inst.y, inst.lam / 2)
        for t in range(trials):
            S = np.flatnonzero(res["sigmas"][:, t])
            r = inst.y - inst.A[:, S] @ res["R"][S, t]
            assert 0.5 * float(r @ r) + inst.lam / 2 * len(S) >= best - 1e-10
        hits += tuple(np.flatnonzero(res["sigma"])) == arg
    return hits


def test_brute_force_minimum_over_all_supports():
    """N = 12: the alternating dynamics minimise the paper's Hamiltonian, whose
    single-spin decision equals that of 1/2||y - A(sigma o R)||^2 + (lambda/2)|sigma|.
    Its result can never beat the brute-force minimum, and it reaches it on most
    seeds (8 of 12 with these seeds; planted mistakes in the field or the
    injection drop this to 6 or fewer)."""
    assert brute_force_hits() >= 7


def brute_force_hits_corrected(n_seeds=12, trials=4):
    """As brute_force_hits in corrected mode, against Eq. doublel0 itself (lambda,
    not lambda / 2): never below the minimum; the number of seeds that reach it."""
    hits = 0
    for seed in range(n_seeds):
        inst = cs_inputs.random_instance(12, 8, 3, 0.05, 0.04, seed=100 + seed)
        prm = Params(n_outer=12, n_steps=1000, dt=0.02, pump_kind="sigmoid", eta_init=0.8,
                     eta_end=math.sqrt(2 * inst.lam), velo=8, seed=seed, self_term=True)
        res = oracle.solve(inst.A, inst.y, inst.lam, prm, trials=trials)
        best, arg = _all_supports_min(inst.A, inst.y, inst.lam)
        for t in range(trials):
            S = np.flatnonzero(res["sigmas"][:, t])
            r = inst.y - inst.A[:, S] @ res["R"][S, t]
            assert 0.5 * float(r @ r) + inst.lam * len(S) >= best - 1e-10
        hits += tuple(np.flatnonzero(res["sigma"])) == arg
    return hits


def test_brute_force_minimum_corrected_mode():
    """Corrected mode minimises Eq. doublel0 with the user's lambda: never below the
    brute-force minimum over all 2^12 supports (asserted per trial), and equal to
    it on half of these seeds (6 of 12; the method is a heuristic, and the formula
    of the correction itself is pinned by the three-spin step and the separable
    case)."""
    assert brute_force_hits_corrected() >= 5


@pytest.mark.parametrize("field", ["cn", "bn"])
def test_best_readout_is_the_first_lowest_objective_on_the_trajectory(field):
    """readout = "best": the configuration returned is, per trial, the first of
    H(c_1) .. H(c_S) of lowest objective.  Checked against the recorded trajectory of
    the same run, each configuration scored with objective() from A and y."""
    inst = cs_inputs.random_instance(30, 18, 4, 0.05, 0.03, seed=6)
    G, hz, g = oracle.gram(inst.A, inst.y)
    Goff = G - np.diag(g)
    T, S = 3, 300
    R = np.repeat((hz / g)[:, None], T, axis=1)
    eta = math.sqrt(2 * inst.lam)
    base = Params(n_steps=S, dt=0.02, field=field, seed=2)
    _, _, _, rc, _ = oracle.cim_run(Goff, hz, R, eta, base, outer=0, record_steps=S, g=g)
    best = oracle.cim_run(Goff, hz, R, eta, dataclasses.replace(base, readout="best"), outer=0, g=g)[0]
    yy = 0.5 * float(inst.y @ inst.y)
    for t in range(T):
        E = []
        for n in range(S):
            s = (rc[n][:, t] > 0).astype(np.uint8)
            E.append(oracle.objective(inst.A, inst.y, s * R[:, t], s, inst.lam) - yy)
        n_star = int(np.argmin(E))
        np.testing.assert_array_equal(best[:, t], (rc[n_star][:, t] > 0).astype(np.uint8))
        # and the readout energy is the objective less 1/2 y^T y
        s = best[:, t:t + 1]
        assert oracle.readout_energy(Goff, g, hz, R[:, t:t + 1], s, inst.lam)[0] == pytest.approx(E[n_star],
                                                                                                 abs=1e-12)


def test_noise_free_exact_recovery():
    """y = A x0 with |x0| >= 0.5 on 20 of 200 coordinates, M = 120, small lambda:
    the support is found exactly and the refit returns x0 to rounding."""
    ok = 0
    for seed in range(3):
        inst = cs_inputs.random_instance(200, 120, 20, 0.0, 1e-3, seed=seed)
        x0 = inst.x0.copy()
        S = np.flatnonzero(inst.xi)
        x0[S] = np.sign(x0[S]) * (0.5 + np.abs(x0[S]))
        y = inst.A @ x0
        prm = Params(n_outer=8, n_steps=1000, dt=0.01, seed=seed)
        res = oracle.solve(inst.A, y, inst.lam, prm, trials=1)
        if np.array_equal(res["sigma"], inst.xi):
            np.testing.assert_allclose(res["x_hat"], x0, rtol=0, atol=1e-9)
            ok += 1
    assert ok >= 2, ok


def test_energy_reported_is_recomputed_objective():
    w = cs_inputs.workload("single_n200_fp64", n_outer=3)
    inst = cs_inputs.workload_instance(w)
    prm = Params(n_outer=3, n_steps=w["n_steps"], dt=w["dt"], seed=w["seed"])
    res = oracle.solve(inst.A, inst.y, inst.lam, prm, trials=2)
    for t in range(2):
        x = res["sigmas"][:, t] * res["R"][:, t]
        r = inst.y - inst.A @ x
        E = 0.5 * float(r @ r) + inst.lam * res["sigmas"][:, t].sum()
        assert res["energies"][t] == pytest.approx(E, rel=1e-12)
    assert res["energy"] == res["energies"].min()
    assert res["best_trial"] == int(np.argmin(res["energies"]))
