"""cs_objective_static: the objective for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (graph capture, arena-owned device memory,
loops where allocation is not allowed).  cs_objective_static takes every buffer
from the caller and keeps its only scratch in a fixed device array inside the
library.  This file is collected last so that a failure here does not hide the
other GPU tests; it must pass both alone and after them.
"""
import ctypes

import numpy as np
import pytest
import torch

import cs_inputs
import oracle
from paper_2405_00366_gb300 import cs

pytestmark = pytest.mark.gpu


def test_objective_static_matches_solver_energies_twice():
    """Two calls in a row through the C ABI: each equals the solver's own per-trial
    energies (the allocating path) and the FP64 oracle's objective (Eq. doublel0)
    of the same (R, sigma), to 1e-12 relative."""
    w = cs_inputs.workload("trials64_n2000_fp32", n_outer=2, n_steps=400)
    inst = cs_inputs.workload_instance(w)
    T = 8
    A = torch.from_numpy(inst.A).cuda()
    y = torch.from_numpy(inst.y).cuda()
    h = cs.cs_problem_create(A, y, inst.lam)
    try:
        cs.cs_solve(h, cs.params_from_workload(w), T)
        R, sig, ref, _ = cs.cs_result_trials(h, T, w["n_outer"])
    finally:
        cs.cs_problem_destroy(h)
    R_d = torch.from_numpy(R).cuda()
    s_d = torch.from_numpy(sig).cuda()
    for call in range(2):
        out = torch.full((T,), float("nan"), dtype=torch.float64, device="cuda")
        # through the C ABI directly
        P = ctypes.c_void_p
        st = cs.lib().cs_objective_static(P(A.data_ptr()), P(y.data_ptr()), P(s_d.data_ptr()), P(R_d.data_ptr()),
                                          inst.M, inst.N, T, inst.lam, P(out.data_ptr()), None)
        assert st == cs.CS_OK, cs.cs_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
        orc = [oracle.objective(inst.A, inst.y, sig[:, t] * R[:, t], sig[:, t], inst.lam) for t in range(T)]
        np.testing.assert_allclose(got, orc, rtol=1e-12, atol=0)


def test_objective_static_rejects_sizes_beyond_its_scratch():
    A = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    y = torch.zeros(2, dtype=torch.float64, device="cuda")
    P = ctypes.c_void_p
    st = cs.lib().cs_objective_static(P(A.data_ptr()), P(y.data_ptr()), P(A.data_ptr()), P(A.data_ptr()),
                                      2, 200000, 2, 0.1, P(y.data_ptr()), None)
    assert st == cs.CS_EINVAL
    assert "static scratch" in cs.cs_last_error()
