"""GPU path (libcs.so through its C ABI) against the FP64 oracle, element by element.

Tolerances:
* FP64 solves: trajectories to 1e-10 relative, supports identical, signal to 1e-8.
* FP32 solves: trajectories ||c_gpu - c_ref||_inf / max(||c_ref||_inf, 1e-2) <= 1e-4
  per step over the first 200 steps; final supports identical; RMSE within 1e-3.
"""
import math

import numpy as np
import pytest
import torch

import cs_inputs
import oracle
from paper_2405_00366_gb300 import cs

pytestmark = pytest.mark.gpu

ORACLE_KEYS = {"n_outer", "n_steps", "dt", "pump_kind", "p0", "p1", "p_thr", "d", "t0", "width", "beta", "tau",
               "K", "j", "eta_init", "eta_end", "velo", "init_kind", "init_scale", "field", "refit", "seed"}


def oracle_params(w):
    return oracle.Params(**{k: v for k, v in w.items() if k in ORACLE_KEYS})


def gpu_solve(inst, w, trials, record_steps=0, device_inputs=True):
    prm = cs.params_from_workload(w, record_steps=record_steps)
    if device_inputs:
        A = torch.from_numpy(inst.A).cuda()
        y = torch.from_numpy(inst.y).cuda()
    else:
        A, y = inst.A, inst.y
    h = cs.cs_problem_create(A, y, inst.lam)
    try:
        cs.cs_solve(h, prm, trials)
        x, s, E, st, status = cs.cs_result(h)
        R, sig, Es, ss = cs.cs_result_trials(h, trials, w["n_outer"])
        traj = cs.cs_trajectory(h, min(record_steps, w["n_steps"]), trials) if record_steps else None
        gram = cs.cs_problem_gram(h)
    finally:
        cs.cs_problem_destroy(h)
    return dict(x_hat=x, sigma=s, energy=E, stats=st, status=status, R=R, sigmas=sig, energies=Es,
                support_sizes=ss, trajectory=traj, gram=gram)


def rel_traj_err(c, ref):
    """Per-step ||c - ref||_inf / max(||ref||_inf, 1e-2)."""
    num = np.abs(c - ref).reshape(c.shape[0], -1).max(axis=1)
    den = np.maximum(np.abs(ref).reshape(ref.shape[0], -1).max(axis=1), 1e-2)
    return num / den


# ------------------------------------------------------------------ a1: Gram
@pytest.mark.parametrize("N,M", [(1, 1), (7, 5), (200, 120), (333, 130), (64, 300)])
def test_gram_parity(N, M):
    inst = cs_inputs.random_instance(N, M, max(1, N // 10), 0.01, 0.1, seed=N + M)
    A = torch.from_numpy(inst.A).cuda()
    y = torch.from_numpy(inst.y).cuda()
    h = cs.cs_problem_create(A, y, inst.lam)
    try:
        G, hz, g = cs.cs_problem_gram(h)
    finally:
        cs.cs_problem_destroy(h)
    Gr, hzr, gr = oracle.gram(inst.A, inst.y)
    scale = np.abs(inst.A).max() ** 2 * M
    np.testing.assert_allclose(G, Gr, rtol=0, atol=1e-13 * scale)
    assert np.array_equal(G, G.T)
    np.testing.assert_allclose(hz, hzr, rtol=0, atol=1e-13 * np.abs(inst.A).max() * np.abs(inst.y).sum() + 1e-300)
    np.testing.assert_array_equal(g, np.diag(G))


def test_host_inputs_match_device_inputs():
    w = cs_inputs.workload("single_n200_fp64", n_outer=2, n_steps=300)
    inst = cs_inputs.workload_instance(w)
    a = gpu_solve(inst, w, 1, device_inputs=True)
    b = gpu_solve(inst, w, 1, device_inputs=False)
    np.testing.assert_array_equal(a["x_hat"], b["x_hat"])
    np.testing.assert_array_equal(a["sigma"], b["sigma"])


# ------------------------------------------------------------------ a2-a5: trajectories
def test_trajectory_fp64_single():
    w = cs_inputs.workload("single_n200_fp64", n_outer=1)
    inst = cs_inputs.workload_instance(w)
    g = gpu_solve(inst, w, 1, record_steps=200)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=1, record_steps=200)
    c, e = g["trajectory"]
    assert rel_traj_err(c, r["trajectory"][0]).max() <= 1e-10
    assert rel_traj_err(e, r["trajectory"][1]).max() <= 1e-10


# stats[10] of each tensor_form for FP32 problems with trial blocks of 16 to 64:
# 1 FMA forms (0 or 1), 2 any tensor-core form (2 or 5), 3 mma.sync (2), 4 tcgen05 (5)
FORM_STAT = {1: (0, 1), 2: (2, 5), 3: (2,), 4: (5,)}


@pytest.mark.parametrize("field,form", [("cn", 1), ("bn", 1), ("cn", 4), ("bn", 4), ("cn", 3), ("bn", 3)])
def test_trajectory_fp32_trials64(field, form):
    """The N = 2000, M = 1200, 64-trial workload: the first 200 Euler steps of every
    trial, with FP32 FMAs (tensor_form = 1), on the tcgen05 tensor cores (4: one
    M = 128 MMA per 16-k block on the stacked FP16 splits of G and X, TMEM
    accumulators) and on the mma.sync tensor cores (3: three FP16 MMAs on split
    operands)."""
    w = cs_inputs.workload("trials64_n2000_fp32", n_outer=1, field=field, tensor_form=form)
    inst = cs_inputs.workload_instance(w)
    g = gpu_solve(inst, w, 64, record_steps=200)
    assert g["stats"][10] in FORM_STAT[form]
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=64, record_steps=200, max_steps=200)
    c, e = g["trajectory"]
    err_c = rel_traj_err(c, r["trajectory"][0])
    err_e = rel_traj_err(e, r["trajectory"][1])
    assert err_c.max() <= 1e-4, err_c.max()
    assert err_e.max() <= 1e-4, err_e.max()


# ------------------------------------------------------------------ whole solve
def _compare_solve(g, r, inst, trials, x_tol, fp64):
    np.testing.assert_array_equal(g["support_sizes"], r["support_sizes"])
    np.testing.assert_array_equal(g["sigmas"], r["sigmas"])
    np.testing.assert_array_equal(g["sigma"], r["sigma"])
    assert int(g["stats"][0]) == r["best_trial"]
    np.testing.assert_allclose(g["x_hat"], r["x_hat"], rtol=0, atol=x_tol)
    np.testing.assert_allclose(g["R"], r["R"], rtol=0, atol=x_tol * 10)
    np.testing.assert_allclose(g["energies"], r["energies"], rtol=1e-9 if fp64 else 1e-6)
    assert abs(oracle.rmse(g["x_hat"], inst.x0) - oracle.rmse(r["x_hat"], inst.x0)) <= 1e-3


def test_solve_fp64_single_full():
    """The single FP64 workload at its full size: N=200, M=120, 20 x 1000 steps."""
    w = cs_inputs.workload("single_n200_fp64")
    inst = cs_inputs.workload_instance(w)
    g = gpu_solve(inst, w, 1)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=1)
    _compare_solve(g, r, inst, 1, 1e-9, True)
    assert g["energy"] == pytest.approx(r["energy"], rel=1e-10)
    # the energy is the recomputed objective of the reported signal
    res = inst.y - inst.A @ g["x_hat"]
    assert g["energy"] == pytest.approx(0.5 * res @ res + inst.lam * g["sigma"].sum(), rel=1e-12)


@pytest.mark.parametrize("precision,field", [("fp32", "cn"), ("fp32", "bn"), ("fp64", "bn")])
def test_solve_ragged(precision, field):
    """N = 333 (not a multiple of any tile), 5 trials, both fields."""
    inst = cs_inputs.random_instance(333, 211, 30, 0.01, 0.04, seed=7)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=4, n_steps=600, precision=precision, field=field,
             seed=11)
    g = gpu_solve(inst, w, 5)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=5)
    _compare_solve(g, r, inst, 5, 1e-9 if precision == "fp64" else 1e-5, precision == "fp64")


@pytest.mark.parametrize("trials,cluster,field,form", [(16, 0, "cn", 4), (32, 2, "bn", 4), (64, 1, "cn", 4),
                                                        (64, 8, "bn", 4), (128, 4, "cn", 4), (16, 0, "cn", 3),
                                                        (64, 8, "bn", 3), (32, 0, "cn", 2)])
def test_solve_ragged_fp32_tensor_cores(trials, cluster, field, form):
    """The FP32 tensor-core forms (tcgen05: tensor_form = 4; mma.sync: 3; either: 2) on N = 333
    (ragged row blocks and k ranges; 128 trials: two blocks of 64 in one launch):
    whole solves against the oracle to the FP32 tolerances."""
    inst = cs_inputs.random_instance(333, 211, 30, 0.01, 0.04, seed=7)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=4, n_steps=600, precision="fp32", field=field,
             seed=11, tensor_form=form, cluster_size=cluster)
    g = gpu_solve(inst, w, trials)
    assert g["stats"][10] in FORM_STAT[form]
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=trials)
    _compare_solve(g, r, inst, trials, 1e-5, False)


def test_solve_paper_schedules_fp64():
    """Sigmoid pump (Eq. pumprateGACS), eta schedule (Eq. etaSchedulling), Gaussian initial amplitudes."""
    inst = cs_inputs.random_instance(150, 90, 15, 0.05, 0.0162, seed=21)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=6, n_steps=500, dt=0.02, pump_kind="sigmoid",
             d=0.4, eta_init=0.8, eta_end=0.18, velo=5.0, init_kind="normal", seed=5)
    g = gpu_solve(inst, w, 3)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=3)
    _compare_solve(g, r, inst, 3, 1e-9, True)


@pytest.mark.parametrize("N,M", [(1, 1), (2, 3), (9, 4)])
def test_tiny_sizes(N, M):
    inst = cs_inputs.random_instance(N, M, 1, 0.0, 0.01, seed=N)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=2, n_steps=200)
    g = gpu_solve(inst, w, 2)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=2)
    _compare_solve(g, r, inst, 2, 1e-9, True)


def test_empty_support():
    """lambda so large that every spin ends off: R = A^T y / diag G, x_hat = 0, E = 1/2 ||y||^2."""
    inst = cs_inputs.random_instance(64, 40, 5, 0.0, 50.0, seed=2)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=2, n_steps=300)
    g = gpu_solve(inst, w, 2)
    assert g["sigmas"].sum() == 0
    G, hz, gd = oracle.gram(inst.A, inst.y)
    np.testing.assert_allclose(g["R"], np.repeat((hz / gd)[:, None], 2, axis=1), rtol=1e-13)
    assert g["energy"] == pytest.approx(0.5 * inst.y @ inst.y, rel=1e-13)


def test_singular_support_uses_ridge():
    """lambda = 0 with M < N: the support exceeds M, G_SS is singular and both sides take the ridge."""
    inst = cs_inputs.random_instance(40, 12, 6, 0.1, 0.0, seed=0)
    # supports 9 then 14 > M = 12: the second refit needs the ridge on both sides
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=2, n_steps=400)
    g = gpu_solve(inst, w, 1)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=1)
    assert r["singular"] and g["status"] == cs.CS_ESINGULAR and g["stats"][2] == 1.0
    np.testing.assert_array_equal(g["sigmas"], r["sigmas"])
    assert np.all(np.isfinite(g["R"]))
    # both interpolate y on the support
    assert np.linalg.norm(inst.y - inst.A @ g["x_hat"]) < 1e-4 * np.linalg.norm(inst.y)


@pytest.mark.parametrize("precision,trials", [("fp64", 1), ("fp32", 4)])
def test_jacobi_refit_matches_oracle(precision, trials):
    """refit = damped Jacobi (step 0.1, 100 sweeps from the trial's current R, the paper's
    CDP for random data): supports identical to the oracle's and R, on and off the
    support, to 1e-9 (FP64) / 1e-5 (FP32 Euler)."""
    inst = cs_inputs.random_instance(200, 120, 20, 0.0, 0.05, seed=0)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=5, n_steps=800, precision=precision, refit="jacobi")
    g = gpu_solve(inst, w, trials)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=trials)
    np.testing.assert_array_equal(g["support_sizes"], r["support_sizes"])
    np.testing.assert_array_equal(g["sigmas"], r["sigmas"])
    tol = 1e-9 if precision == "fp64" else 1e-5
    np.testing.assert_allclose(g["R"], r["R"], rtol=0, atol=tol)
    np.testing.assert_allclose(g["energies"], r["energies"], rtol=1e-9 if precision == "fp64" else 1e-6)


def test_large_support_blocked_factor_matches_oracle():
    """Supports of more than about 310 entries do not fit the packed FP32 factor in shared
    memory and take the blocked FP32 factor in global memory with FP64 refinement (FP64
    Cholesky if that does not converge); against the oracle: identical supports, R to 1e-8."""
    inst = cs_inputs.random_instance(900, 760, 420, 0.0, 0.005, seed=4)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=2, n_steps=500, precision="fp64")
    g = gpu_solve(inst, w, 2)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=2)
    assert r["support_sizes"].max() > 320
    np.testing.assert_array_equal(g["sigmas"], r["sigmas"])
    np.testing.assert_allclose(g["R"], r["R"], rtol=0, atol=1e-8)


def test_autotuned_split_matches_oracle():
    """autotune = 1 times the cheapest candidate work splits on the GPU and keeps the
    fastest; whichever it keeps, the solve matches the oracle (FP32 tolerances)."""
    inst = cs_inputs.random_instance(600, 360, 60, 0.01, 0.03, seed=12)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=2, n_steps=400, precision="fp32", seed=5,
             autotune=1)
    g = gpu_solve(inst, w, 8)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=8)
    np.testing.assert_array_equal(g["sigmas"], r["sigmas"])
    np.testing.assert_allclose(g["x_hat"], r["x_hat"], rtol=0, atol=1e-5)


def test_two_trial_blocks_match_oracle():
    """128 trials: two blocks of 64 in one launch (wide split, per-block reductions);
    supports identical to the oracle's, x_hat to 1e-5."""
    inst = cs_inputs.random_instance(300, 180, 30, 0.01, 0.03, seed=21)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=2, n_steps=300, precision="fp32", seed=9)
    g = gpu_solve(inst, w, 128)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=128)
    np.testing.assert_array_equal(g["support_sizes"], r["support_sizes"])
    np.testing.assert_array_equal(g["sigmas"], r["sigmas"])
    np.testing.assert_allclose(g["x_hat"], r["x_hat"], rtol=0, atol=1e-5)


def test_trials64_full_size_properties():
    """The N = 2000, 64-trial workload at full size (30 x 2000 steps), in the launch
    configuration the benchmark times (autotuned work split).  The oracle runs trials 0
    and 1 for the first two outer iterations, and the same launch configuration stopped
    after two outer iterations must give their supports exactly and R to 1e-5; the full
    run is checked by properties that hold at any size."""
    w = cs_inputs.workload("trials64_n2000_fp32", autotune=1)
    inst = cs_inputs.workload_instance(w)
    g = gpu_solve(inst, w, 64)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(dict(w, n_outer=2)), trials=2)
    np.testing.assert_array_equal(g["support_sizes"][:2, :2], r["support_sizes"])
    g2 = gpu_solve(inst, dict(w, n_outer=2), 64)
    np.testing.assert_array_equal(g2["sigmas"][:, :2], r["sigmas"])
    np.testing.assert_allclose(g2["R"][:, :2], r["R"], rtol=0, atol=1e-5)
    G, hz, gd = oracle.gram(inst.A, inst.y)
    for t in range(64):
        s = g["sigmas"][:, t]
        S = np.flatnonzero(s)
        R = g["R"][:, t]
        # the refit is the least-squares solution on S: zero gradient
        grad = inst.A[:, S].T @ (inst.y - inst.A[:, S] @ R[S])
        assert np.abs(grad).max() <= 1e-9 * np.linalg.norm(hz)
        # off the support R is the Jacobi fixed point
        lhs = gd * R + (G - np.diag(gd)) @ (s * R)
        np.testing.assert_allclose(lhs, hz, rtol=0, atol=1e-9)
        res = inst.y - inst.A @ (s * R)
        assert g["energies"][t] == pytest.approx(0.5 * res @ res + inst.lam * s.sum(), rel=1e-10)
    assert int(g["stats"][0]) == int(np.argmin(g["energies"]))
    assert oracle.rmse(g["x_hat"], inst.x0) < 0.05


def test_barrier_timeout_is_reported_and_context_survives():
    """A grid barrier that waits for CTAs that never arrive runs into timeout_ms,
    the solve reports CS_ETIMEOUT, and the next solve on the same problem works."""
    w = cs_inputs.workload("single_n200_fp64", n_outer=1, n_steps=50)
    inst = cs_inputs.workload_instance(w)
    h = cs.cs_problem_create(torch.from_numpy(inst.A).cuda(), torch.from_numpy(inst.y).cuda(), inst.lam)
    try:
        bad = cs.params_from_workload(w, timeout_ms=200, test_phantom_ctas=1)
        cs.cs_solve(h, bad, 1)
        with pytest.raises(cs.CSError) as ei:
            cs.cs_result(h)
        assert ei.value.status == cs.CS_ETIMEOUT
        cs.cs_solve(h, cs.params_from_workload(w), 1)
        x, s, E, st, status = cs.cs_result(h)
        assert status == cs.CS_OK and np.isfinite(E)
    finally:
        cs.cs_problem_destroy(h)
    torch.cuda.synchronize()


# ------------------------------------------------------------------ s2: error against FP64 per result
def test_solve_is_one_graph_launch():
    """cs_solve queues the coupling copy and the initial R directly and every outer
    iteration (Euler launch, refit) plus the objective as one CUDA graph: a second
    solve of the same problem reports two host submissions, the per-phase device
    times come from event nodes inside the graph, the two solves agree bitwise and
    their supports are the oracle's."""
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=3, n_steps=300)
    inst = cs_inputs.workload_instance(w)
    prm = cs.params_from_workload(w)
    h = cs.cs_problem_create(torch.from_numpy(inst.A).cuda(), torch.from_numpy(inst.y).cuda(), inst.lam)
    try:
        cs.cs_solve(h, prm, 2)
        x1, s1, E1, st1, _ = cs.cs_result(h)
        (ms1, n1) = cs.cs_problem_timing(h)
        cs.cs_solve(h, prm, 2)
        x2, s2, E2, st2, _ = cs.cs_result(h)
        (ms2, n2) = cs.cs_problem_timing(h)
    finally:
        cs.cs_problem_destroy(h)
    assert ms1[4] in (2, 3) and ms2[4] == 2
    assert ms2[1] > 0 and ms2[2] > 0 and ms2[3] > 0
    assert n2 >= 2 + 1 + 3 * 2 + 4  # Gram, initial R, per iteration Euler + refit, objective
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(s1, s2)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=2)
    np.testing.assert_array_equal(s2, r["sigma"])
    np.testing.assert_allclose(x2, r["x_hat"], rtol=0, atol=1e-8)


@pytest.mark.parametrize("precision,refit", [("fp64", "exact"), ("fp32", "exact"), ("bf16", "exact"),
                                             ("fp16", "exact"), ("fp32", "jacobi")])
def test_error_against_fp64_is_reported_per_result(precision, refit):
    """stats[11]: relative error of G_off x_hat with G_off in its storage precision
    against FP64; stats[12]: FP64 relative residual of the refit's normal equations on
    the kept support.  Both recomputed here from the returned x_hat (storage rounding
    by the helper pinned in test_storage_rounding_cpu.py)."""
    from storage_rounding import round_to_storage
    inst = cs_inputs.random_instance(300, 180, 30, 0.01, 0.03, seed=17)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=3, n_steps=600, precision=precision, refit=refit)
    g = gpu_solve(inst, w, 4)
    G, hz, gd = oracle.gram(inst.A, inst.y)
    Goff = G - np.diag(gd)
    x = g["x_hat"]
    if precision == "fp64":
        Gs = Goff
    elif precision == "fp32":
        Gs = Goff.astype(np.float32).astype(np.float64)
    else:
        Gs = round_to_storage(Goff, precision)
    U = Goff @ x
    e11 = np.abs((Gs - Goff) @ x).max() / np.abs(U).max()
    S = np.flatnonzero(g["sigma"])
    e12 = np.abs(hz[S] - G[S] @ x).max() / np.abs(hz[S]).max()
    if precision == "fp64":
        assert g["stats"][11] == 0.0
    else:
        assert g["stats"][11] == pytest.approx(e11, rel=1e-6)
        assert 0.0 < g["stats"][11] < {"fp32": 1e-6, "fp16": 1e-2, "bf16": 1e-1}[precision]
    if refit == "exact":
        assert g["stats"][12] <= 1e-12 and e12 <= 1e-12
    else:
        assert g["stats"][12] == pytest.approx(e12, rel=1e-6)


# ------------------------------------------------------------------ f4: corrected self-term, best readout
ORACLE_KEYS_F4 = ORACLE_KEYS | {"self_term", "readout"}


def oracle_params_f4(w):
    return oracle.Params(**{k: v for k, v in w.items() if k in ORACLE_KEYS_F4})


@pytest.mark.parametrize("precision,field", [("fp64", "cn"), ("fp64", "bn"), ("fp32", "cn")])
def test_corrected_self_term_matches_oracle(precision, field):
    """self_term = 1: the injection restores the self-term (the single-spin decision of
    Eq. doublel0); whole solves against the oracle in the same mode."""
    inst = cs_inputs.random_instance(250, 150, 25, 0.01, 0.03, seed=23)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=3, n_steps=700, precision=precision, field=field,
             self_term=True, seed=6)
    g = gpu_solve(inst, w, 4)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params_f4(w), trials=4)
    _compare_solve(g, r, inst, 4, 1e-9 if precision == "fp64" else 1e-5, precision == "fp64")
    # a different dynamics than the paper-literal mode on this instance
    plain = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=4)
    assert not np.array_equal(plain["sigmas"], r["sigmas"])


def test_corrected_self_term_in_a_batch():
    """The batched kernel folds the same correction into its prologue."""
    from test_batch_gpu import run_batch
    insts = [cs_inputs.random_instance(N, int(0.6 * N), N // 10, 0.01, 0.03, seed=40 + N) for N in (120, 77, 200)]
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=2, n_steps=500, precision="fp64", self_term=True)
    out = run_batch(insts, w, 2)
    for i, (inst, res) in enumerate(zip(insts, out)):
        r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params_f4(w), trials=2, inst=i)
        np.testing.assert_array_equal(res["sigmas"], r["sigmas"])
        np.testing.assert_allclose(res["x_hat"], r["x_hat"], rtol=0, atol=1e-9)


@pytest.mark.parametrize("precision,form,cluster", [("fp64", 0, 0), ("fp64", 0, 2), ("fp32", 1, 0), ("fp32", 4, 0)])
def test_best_readout_matches_oracle(precision, form, cluster):
    """readout = best (binarised field): each CIM run returns the first configuration
    of lowest objective among those it visited.  FP64 (two cluster shapes) and FP32
    (FMAs, tcgen05) against the oracle: supports and R per trial."""
    inst = cs_inputs.random_instance(240, 140, 24, 0.01, 0.03, seed=29)
    T = 16 if form == 4 else 4
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=3, n_steps=600, precision=precision, field="bn",
             readout="best", seed=8, tensor_form=form, cluster_size=cluster)
    g = gpu_solve(inst, w, T)
    if form == 4:
        assert g["stats"][10] == 5
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params_f4(w), trials=T)
    _compare_solve(g, r, inst, T, 1e-9 if precision == "fp64" else 1e-5, precision == "fp64")
    final = oracle.solve(inst.A, inst.y, inst.lam, oracle_params_f4(dict(w, readout="final")), trials=T)
    assert r["energy"] <= final["energy"] + 1e-12


def test_best_readout_argument_checks():
    """The best readout needs the binarised field and a single solve."""
    inst = cs_inputs.random_instance(64, 40, 6, 0.0, 0.05, seed=1)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=1, n_steps=10, readout="best")
    h = cs.cs_problem_create(torch.from_numpy(inst.A).cuda(), torch.from_numpy(inst.y).cuda(), inst.lam)
    try:
        with pytest.raises(cs.CSError) as ei:
            cs.cs_solve(h, cs.params_from_workload(w, field="cn"), 2)
        assert ei.value.status == cs.CS_EINVAL
        with pytest.raises(cs.CSError) as ei:
            cs.cs_solve_batch([h], cs.params_from_workload(w, field="bn"), 2)
        assert ei.value.status == cs.CS_EINVAL
    finally:
        cs.cs_problem_destroy(h)


# ------------------------------------------------------------------ f2: conjugate-gradient refit
@pytest.mark.parametrize("precision,trials", [("fp64", 1), ("fp64", 3), ("fp32", 4)])
def test_cg_refit_matches_oracle(precision, trials):
    """refit = cg (the paper's CDP for MRI data): FP64 conjugate gradient on the
    support's normal equations, warm started from each trial's R, against the oracle:
    supports identical, R (on and off the support) to 1e-7 relative to max |R|."""
    inst = cs_inputs.random_instance(300, 180, 30, 0.01, 0.03, seed=19)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=3, n_steps=700, precision=precision, refit="cg",
             cg_iters=10000, cg_tol=1e-10)
    g = gpu_solve(inst, w, trials)
    keys = ORACLE_KEYS | {"cg_iters", "cg_tol"}
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle.Params(**{k: v for k, v in w.items() if k in keys}),
                     trials=trials)
    np.testing.assert_array_equal(g["support_sizes"], r["support_sizes"])
    np.testing.assert_array_equal(g["sigmas"], r["sigmas"])
    np.testing.assert_allclose(g["R"], r["R"], rtol=0, atol=1e-7 * np.abs(r["R"]).max())
    # the refit's FP64 residual is within the tolerance asked for
    assert g["stats"][12] <= 1e-9


def test_cg_refit_mri_shaped():
    """32 x 32 MRI-shaped problem (orthonormal rows of a subsampled 2-D DCT over Haar
    coefficients): the conjugate-gradient refit agrees with the oracle's, and with
    the exact refit's solution (supports identical, x_hat to 1e-7 relative)."""
    w = cs_inputs.workload("mri_n16384_fp16", mri_side=32, N=1024, M=307, nnz=102, n_outer=3, n_steps=800,
                           precision="fp32", refit="cg")
    inst = cs_inputs.workload_instance(w)
    g = gpu_solve(inst, w, 2)
    keys = ORACLE_KEYS | {"cg_iters", "cg_tol"}
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle.Params(**{k: v for k, v in w.items() if k in keys}), trials=2)
    np.testing.assert_array_equal(g["sigmas"], r["sigmas"])
    np.testing.assert_allclose(g["x_hat"], r["x_hat"], rtol=0, atol=1e-7 * np.abs(r["x_hat"]).max())
    e = gpu_solve(inst, dict(w, refit="exact"), 2)
    np.testing.assert_array_equal(g["sigmas"], e["sigmas"])
    np.testing.assert_allclose(g["x_hat"], e["x_hat"], rtol=0, atol=1e-7 * np.abs(e["x_hat"]).max())


# ------------------------------------------------------------------ f1: the paper's random-data schedule
@pytest.mark.parametrize("field", ["cn", "bn"])
def test_paper_schedule_outer_history_matches_oracle(field):
    """The paper's random-data settings (sigmoid pump d = 0.4, dt = 0.02 x 1000,
    eta schedule from 0.8, damped Jacobi CDP, N(0, 1e-4) amplitudes) scaled to
    N = 200, twelve outer iterations (velo = 11), FP64: the support and R of every
    trial after EVERY outer iteration (record_outer, cs_outer_history) equal the
    oracle's, so per-iteration RMSE and Hamming curves are the oracle's too."""
    w = cs_inputs.workload("paper_random_n2000", N=200, M=120, nnz=40, n_outer=12, velo=11.0, precision="fp64",
                           field=field, seed=4)
    inst = cs_inputs.workload_instance(w)
    T = 2
    prm = cs.params_from_workload(w, record_outer=1)
    h = cs.cs_problem_create(torch.from_numpy(inst.A).cuda(), torch.from_numpy(inst.y).cuda(), inst.lam)
    try:
        cs.cs_solve(h, prm, T)
        cs.cs_result(h)
        sig_h, R_h = cs.cs_outer_history(h, w["n_outer"], inst.N, T)
    finally:
        cs.cs_problem_destroy(h)
    keys = ORACLE_KEYS | {"jacobi_dt", "jacobi_iters"}
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle.Params(**{k: v for k, v in w.items() if k in keys}), trials=T)
    np.testing.assert_array_equal(sig_h, r["sigma_outer"])
    np.testing.assert_allclose(R_h, r["R_outer"], rtol=0, atol=1e-9)
    ham = [oracle.hamming_loss(sig_h[i, :, 0], inst.xi) for i in range(w["n_outer"])]
    assert ham[-1] < ham[0]  # the alternation improves the support estimate on this instance


# ------------------------------------------------------------------ f3: the paper's MRI model
ORACLE_KEYS_MRI = ORACLE_KEYS | {"cg_iters", "cg_tol", "init_R", "lasso_lambda", "lasso_iters"}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mri_full_model_matches_oracle(precision):
    """The paper's MRI problem on a synthetic 16 x 16 image: complex-DFT observation
    (real-ified), the gamma-weighted second-difference terms, the LASSO solution
    (FISTA on the GPU) as the initial R, conjugate-gradient CDP, the MRI pump
    (d = 0.6) and fixed eta, against the oracle: supports of every trial after
    every outer iteration identical, x_hat to 1e-7 relative."""
    w = cs_inputs.workload("mri_full_n16384", mri_side=16, N=256, M_obs=77, M=2 * 77 + 2 * 256, nnz=26,
                           n_outer=4, trials=3, precision=precision, mri_gamma=1e-3, lasso_iters=200)
    inst = cs_inputs.workload_instance(w)
    assert inst.A.shape == (w["M"], w["N"])
    T = w["trials"]
    prm = cs.params_from_workload(w, record_outer=1)
    h = cs.cs_problem_create(torch.from_numpy(inst.A).cuda(), torch.from_numpy(inst.y).cuda(), inst.lam)
    try:
        cs.cs_solve(h, prm, T)
        x, s, E, st, status = cs.cs_result(h)
        sig_h, R_h = cs.cs_outer_history(h, w["n_outer"], inst.N, T)
    finally:
        cs.cs_problem_destroy(h)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle.Params(**{k: v for k, v in w.items() if k in ORACLE_KEYS_MRI}),
                     trials=T)
    np.testing.assert_array_equal(sig_h, r["sigma_outer"])
    np.testing.assert_allclose(x, r["x_hat"], rtol=0, atol=1e-7 * max(1.0, np.abs(r["x_hat"]).max()))
    # the LASSO start matters: the first support differs from the plain start's
    plain = oracle.solve(inst.A, inst.y, inst.lam,
                         oracle.Params(**{k: v for k, v in dict(w, init_R="zeeman").items() if k in ORACLE_KEYS_MRI}),
                         trials=T)
    assert not np.array_equal(plain["sigma_outer"][0], r["sigma_outer"][0])
