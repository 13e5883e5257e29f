"""Euler plans that stream G_off tiles from memory every step (for N too large
for the coupling matrix to stay on chip), forced at sizes the oracle can check,
and the MRI-shaped workload (Haar-sparse image through a subsampled 2-D DCT)."""
import numpy as np
import pytest
import torch

import cs_inputs
import oracle
from paper_2405_00366_gb300 import cs
from storage_rounding import round_to_storage

pytestmark = pytest.mark.gpu

ORACLE_KEYS = {"n_outer", "n_steps", "dt", "pump_kind", "p0", "p1", "p_thr", "d", "t0", "width", "beta", "tau",
               "K", "j", "eta_init", "eta_end", "velo", "init_kind", "init_scale", "field", "refit", "seed"}


def oracle_params(w):
    return oracle.Params(**{k: v for k, v in w.items() if k in ORACLE_KEYS})


def solve(inst, w, T, **over):
    prm = cs.params_from_workload(w, **over)
    h = cs.cs_problem_create(torch.from_numpy(inst.A).cuda(), torch.from_numpy(inst.y).cuda(), inst.lam)
    try:
        cs.cs_solve(h, prm, T)
        x, s, E, st, _ = cs.cs_result(h)
        R, sig, Es, ss = cs.cs_result_trials(h, T, w["n_outer"])
    finally:
        cs.cs_problem_destroy(h)
    return dict(x_hat=x, sigma=s, energy=E, stats=st, sigmas=sig, support_sizes=ss)


@pytest.mark.parametrize("field", ["cn", "bn"])
def test_streamed_fp32_matches_oracle(field):
    inst = cs_inputs.random_instance(333, 211, 30, 0.01, 0.04, seed=7)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=3, n_steps=500, precision="fp32", field=field, seed=3)
    g = solve(inst, w, 5, stream_g=1)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=5)
    np.testing.assert_array_equal(g["support_sizes"], r["support_sizes"])
    np.testing.assert_array_equal(g["sigmas"], r["sigmas"])
    np.testing.assert_allclose(g["x_hat"], r["x_hat"], rtol=0, atol=1e-5)


@pytest.mark.parametrize("cluster", [1, 4])
def test_streamed_equals_resident_supports(cluster):
    """The same problem with G_off resident and streamed: identical supports."""
    w = cs_inputs.workload("trials64_n2000_fp32", N=1200, M=720, nnz=120, n_outer=2, n_steps=600, precision="bf16")
    inst = cs_inputs.workload_instance(w)
    a = solve(inst, w, 16, cluster_size=cluster)
    b = solve(inst, w, 16, cluster_size=cluster, stream_g=1)
    np.testing.assert_array_equal(a["sigmas"], b["sigmas"])
    np.testing.assert_allclose(a["x_hat"], b["x_hat"], rtol=0, atol=1e-6)


@pytest.mark.parametrize("precision", ["fp16"])
def test_mri_shaped_small(precision):
    """32 x 32 MRI-shaped problem (N = 1024, M = 307), G_off streamed in FP16: support
    within 1% of the FP64 oracle's and RMSE within 1e-3.  (FP8 storage does not meet
    this gate on the MRI operator: measured Hamming 0.19 on GB300.)"""
    w = cs_inputs.workload("mri_n16384_fp16", mri_side=32, N=1024, M=307, nnz=102, n_outer=3, n_steps=800,
                           precision=precision)
    inst = cs_inputs.workload_instance(w)
    assert np.allclose(inst.A @ inst.A.T, np.eye(inst.M), atol=1e-12)
    g = solve(inst, w, 4, stream_g=1)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=4)
    assert oracle.hamming_loss(g["sigma"], r["sigma"]) <= 0.01
    assert abs(oracle.rmse(g["x_hat"], inst.x0) - oracle.rmse(r["x_hat"], inst.x0)) <= 1e-3


def test_streamed_bf16_autotuned_matches_resident():
    """Streamed G_off with the autotuner choosing among streamed splits: the same
    supports as the resident default on a BF16 problem."""
    w = cs_inputs.workload("trials64_n2000_fp32", N=800, M=480, nnz=80, n_outer=2, n_steps=500, precision="bf16")
    inst = cs_inputs.workload_instance(w)
    a = solve(inst, w, 64)
    b = solve(inst, w, 64, stream_g=1, autotune=1)
    np.testing.assert_array_equal(a["sigmas"], b["sigmas"])
    np.testing.assert_allclose(a["x_hat"], b["x_hat"], rtol=0, atol=1e-6)


# ------------------------------------------------------------ tensor-core form
def rel_traj_err(c, ref):
    """Per-step ||c - ref||_inf / max(||ref||_inf, 1e-2)."""
    num = np.abs(c - ref).reshape(c.shape[0], -1).max(axis=1)
    den = np.maximum(np.abs(ref).reshape(ref.shape[0], -1).max(axis=1), 1e-2)
    return num / den


def solve_traj(inst, w, T, record_steps, y=None, lam=None, **over):
    prm = cs.params_from_workload(w, record_steps=record_steps, **over)
    y = inst.y if y is None else y
    lam = inst.lam if lam is None else lam
    h = cs.cs_problem_create(torch.from_numpy(inst.A).cuda(), torch.from_numpy(y).cuda(), lam)
    try:
        cs.cs_solve(h, prm, T)
        x, s, E, st, status = cs.cs_result(h)
        R, sig, Es, ss = cs.cs_result_trials(h, T, w["n_outer"])
        c, e = cs.cs_trajectory(h, record_steps, T)
    finally:
        cs.cs_problem_destroy(h)
    return dict(x_hat=x, sigma=s, energy=E, stats=st, status=status, sigmas=sig, c=c, e=e)


@pytest.mark.parametrize("precision,field,cluster", [("fp16", "cn", 0), ("fp16", "bn", 1), ("bf16", "cn", 2)])
def test_tensor_core_trajectory_matches_rounded_oracle(precision, field, cluster):
    """Streamed 16-bit G_off with eight trials runs on the tensor cores (stats[10]
    = 2).  N = 333 (ragged: 21 row tiles of 16, a partial last k tile): the first
    200 Euler steps of every trial against the oracle's CIM run on the same G_off
    rounded to the storage type, to the FP32 form's tolerance (1e-4 relative)."""
    inst = cs_inputs.random_instance(333, 211, 30, 0.01, 0.04, seed=7)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=1, n_steps=600, precision=precision, field=field,
             seed=3)
    g = solve_traj(inst, w, 8, 200, stream_g=1, cluster_size=cluster, tensor_form=2)
    assert g["stats"][10] == 2
    op = oracle_params(w)
    G, hz, gd = oracle.gram(inst.A, inst.y)
    Goff = round_to_storage(G - np.diag(gd), precision)
    R = np.repeat((hz / gd)[:, None], 8, axis=1)
    _, _, _, rc, re = oracle.cim_run(Goff, hz, R, oracle.eta_at(0, op, inst.lam), op, outer=0, record_steps=200,
                                     max_steps=200)
    assert rel_traj_err(g["c"], rc).max() <= 1e-4
    assert rel_traj_err(g["e"], re).max() <= 1e-4


def test_tensor_core_power_of_two_scaling_is_exact():
    """(y, lambda, K) -> (2^16 y, 2^32 lambda, 2^-32 K) leaves the dynamics exactly
    unchanged and scales R, x_hat by 2^16 and the energy by 2^32.  With FP16 X the
    unscaled X would overflow (|X| ~ 2^16 |c|); the form's power-of-two scale of X
    makes every trajectory bit-identical to the unscaled problem's."""
    inst = cs_inputs.random_instance(333, 211, 30, 0.01, 0.04, seed=7)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=2, n_steps=400, precision="fp16", seed=3)
    s = 2.0 ** 16
    a = solve_traj(inst, w, 8, 100, stream_g=1, tensor_form=2)
    b = solve_traj(inst, dict(w, K=w["K"] / (s * s)), 8, 100, y=inst.y * s, lam=inst.lam * s * s, stream_g=1,
                   tensor_form=2)
    assert a["stats"][10] == 2 and b["stats"][10] == 2
    np.testing.assert_array_equal(a["c"], b["c"])
    np.testing.assert_array_equal(a["sigmas"], b["sigmas"])
    np.testing.assert_array_equal(a["x_hat"] * s, b["x_hat"])
    assert b["energy"] == pytest.approx(a["energy"] * s * s, rel=1e-14)


def test_mri_shaped_small_tensor_cores():
    """32 x 32 MRI-shaped problem, FP16 G_off streamed, eight trials: the tensor-core
    form (tensor_form = 2) and the FMA forms (tensor_form = 1) each meet the FP16 gate against the
    FP64 oracle (support within 1%, RMSE within 1e-3)."""
    w = cs_inputs.workload("mri_n16384_fp16", mri_side=32, N=1024, M=307, nnz=102, n_outer=3, n_steps=800)
    inst = cs_inputs.workload_instance(w)
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle_params(w), trials=8)
    for tf in (2, 1):
        g = solve(inst, w, 8, stream_g=1, tensor_form=tf)
        assert (g["stats"][10] == 2) == (tf == 2)
        assert oracle.hamming_loss(g["sigma"], r["sigma"]) <= 0.01
        assert abs(oracle.rmse(g["x_hat"], inst.x0) - oracle.rmse(r["x_hat"], inst.x0)) <= 1e-3


def test_tensor_form_2_where_no_tensor_form_applies():
    """tensor_form = 2 asks for the tensor-core form only: FP64 storage, an FP32
    solve with 5 trials (blocks narrower than 16) and a BF16 batch with 4 trials
    have none, and each is refused with CS_EINVAL (no silent fallback)."""
    inst = cs_inputs.random_instance(64, 40, 6, 0.0, 0.05, seed=1)
    w = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=1, n_steps=10)
    h = cs.cs_problem_create(torch.from_numpy(inst.A).cuda(), torch.from_numpy(inst.y).cuda(), inst.lam)
    try:
        for precision, T in (("fp64", 1), ("fp32", 5)):
            with pytest.raises(cs.CSError) as ei:
                cs.cs_solve(h, cs.params_from_workload(w, precision=precision, tensor_form=2), T)
            assert ei.value.status == cs.CS_EINVAL
        with pytest.raises(cs.CSError) as ei:
            cs.cs_solve_batch([h], cs.params_from_workload(w, precision="bf16", tensor_form=2), 4)
        assert ei.value.status == cs.CS_EINVAL
        # the problem stays usable: the same solve with the planner's choice works
        cs.cs_solve(h, cs.params_from_workload(w, precision="fp32"), 5)
        cs.cs_result(h)
    finally:
        cs.cs_problem_destroy(h)


def test_mri_full_size_sampled_steps():
    """The MRI-shaped workload at its full size (128 x 128 image: N = 16384,
    M = 4915, 8 trials, FP16 G_off streamed, the plan the benchmark runs): the
    first three Euler steps of the first CIM run, as the library recorded them,
    against the oracle's own step (local field of Eq. localfieldMFZ, injection,
    explicit Euler step) applied to the recorded state of the step before, on 64
    sampled rows, with those rows of G_off formed from A in FP64 and rounded to
    FP16 as the library stores them (relative 1e-4, the FP32 trajectory bar)."""
    w = cs_inputs.workload("mri_n16384_fp16", n_outer=1)
    inst = cs_inputs.workload_instance(w)
    N, T, K = inst.N, w["trials"], 3
    prm = cs.params_from_workload(w, record_steps=K)
    h = cs.cs_problem_create(torch.from_numpy(inst.A).cuda(), torch.from_numpy(inst.y).cuda(), inst.lam)
    try:
        cs.cs_solve(h, prm, T)
        cs.cs_result(h)
        c_rec, e_rec = cs.cs_trajectory(h, K, T)
    finally:
        cs.cs_problem_destroy(h)
    op = oracle_params(w)
    rows = np.sort(np.random.default_rng(5).choice(N, 64, replace=False))
    A = inst.A
    hz = A.T @ inst.y
    g = np.einsum("ij,ij->j", A, A)
    Goff = A[:, rows].T @ A
    Goff[np.arange(rows.size), rows] = 0.0
    Goff = round_to_storage(Goff, "fp16")
    R = np.repeat((hz / g)[:, None], T, axis=1)
    eta = oracle.eta_at(0, op, inst.lam)
    c = np.stack([oracle.initial_amplitudes(op.seed, 0, t, 0, N, op.init_kind, op.init_scale) for t in range(T)],
                 axis=1)
    e = np.ones((N, T))
    for n in range(K):
        hr = oracle.local_field_cn(Goff, R, c, hz[rows], op.tau)
        inj = oracle.injection(op.j, e[rows], R[rows], hr, eta, op.tau)
        cn, en = oracle.euler_step(c[rows], e[rows], oracle.pump(n, op), inj, op)
        for got, ref in ((c_rec[n][rows], cn), (e_rec[n][rows], en)):
            err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-2)
            assert err <= 1e-4, (n, err)
        c, e = c_rec[n], e_rec[n]
