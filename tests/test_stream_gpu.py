"""Euler plans that stream G_off tiles from memory every step (for N too large
for the coupling matrix to stay on chip), forced at sizes the oracle can check,
and the MRI-shaped workload (Haar-sparse image through a subsampled 2-D DCT)."""
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
