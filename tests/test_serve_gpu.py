"""The continuous-batching server: requests of different shapes admitted by free
slot and HBM budget, overlapping on the GPU, each giving the same result alone
and in the mix, and the FP64 one matching the oracle."""
import ctypes

import numpy as np
import pytest

import cs_inputs
import oracle
from paper_2405_00366_gb300 import cs

ORACLE_KEYS = {"n_outer", "n_steps", "dt", "pump_kind", "p0", "p1", "p_thr", "d", "t0", "width", "beta", "tau",
               "K", "j", "eta_init", "eta_end", "velo", "init_kind", "init_scale", "field", "refit", "seed"}


def _requests():
    base = cs_inputs.WORKLOADS["single_n200_fp64"]
    return [
        (cs_inputs.random_instance(200, 120, 20, 0.0, 0.05, seed=0), dict(base, n_outer=3, n_steps=600), 1),
        (cs_inputs.random_instance(333, 200, 30, 0.01, 0.03, seed=1),
         dict(base, n_outer=2, n_steps=500, precision="fp32"), 4),
        (cs_inputs.random_instance(256, 128, 26, 0.01, 0.03, seed=2),
         dict(base, n_outer=2, n_steps=500, precision="bf16"), 16),
        (cs_inputs.random_instance(150, 90, 15, 0.01, 0.03, seed=3),
         dict(base, n_outer=2, n_steps=400, precision="fp32", field="bn"), 2),
    ]


def _serve(reqs, slots=3, budget=8 << 30):
    sv = cs.cs_server_create(budget, slots)
    try:
        tickets = [cs.cs_server_submit_host(sv, inst.A, inst.y, inst.lam, cs.params_from_workload(w), T)
                   for inst, w, T in reqs]
        out = []
        for (inst, w, T), t in zip(reqs, tickets):
            cs.cs_server_wait(sv, t)
            assert cs.cs_server_poll(sv, t)
            out.append(cs.cs_server_result(sv, t, inst.N))
    finally:
        cs.cs_server_destroy(sv)
    return out


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix():
    reqs = _requests()
    mixed = _serve(reqs)
    for k, req in enumerate(reqs):
        alone = _serve([req])[0]
        np.testing.assert_array_equal(alone[0], mixed[k][0])  # x_hat, bit for bit
        np.testing.assert_array_equal(alone[1], mixed[k][1])
        assert alone[2] == mixed[k][2]
    # the FP64 request against the oracle
    inst, w, T = reqs[0]
    r = oracle.solve(inst.A, inst.y, inst.lam, oracle.Params(**{k: v for k, v in w.items() if k in ORACLE_KEYS}),
                     trials=T)
    np.testing.assert_array_equal(mixed[0][1], r["sigma"])
    np.testing.assert_allclose(mixed[0][0], r["x_hat"], rtol=0, atol=1e-9)


@pytest.mark.gpu
def test_budget_admission_and_ticket_lifecycle():
    reqs = [_requests()[1]] * 3  # about 6.5 MB of device memory each
    # room for one request at a time: each starts after the previous finished
    sv = cs.cs_server_create(10 << 20, 3)
    try:
        with pytest.raises(cs.CSError) as ei:  # can never fit
            big = cs_inputs.random_instance(4000, 100, 10, 0.0, 0.1, seed=9)
            cs.cs_server_submit_host(sv, big.A, big.y, big.lam, cs.cs_params_default(), 64)
        assert ei.value.status == cs.CS_ENOMEM
        tickets = [cs.cs_server_submit_host(sv, i.A, i.y, i.lam, cs.params_from_workload(w), T) for i, w, T in reqs]
        times = []
        for (inst, w, T), t in zip(reqs, tickets):
            cs.cs_server_wait(sv, t)
            res = cs.cs_server_result(sv, t, inst.N)
            times.append(res[4])
            with pytest.raises(cs.CSError):  # the ticket is gone once its result is read
                cs.cs_server_result(sv, t, inst.N)
        for a, b in zip(times, times[1:]):
            assert b[1] >= a[2] - 1e-3  # admitted only after the previous one finished
    finally:
        cs.cs_server_destroy(sv)


def test_server_argument_checks_need_no_gpu():
    h = ctypes.c_void_p()
    assert cs.lib().cs_server_create(0, 2, ctypes.byref(h)) == cs.CS_EINVAL
    assert cs.lib().cs_server_create(1 << 30, 0, ctypes.byref(h)) == cs.CS_EINVAL
    d = ctypes.c_int32()
    assert cs.lib().cs_server_poll(None, 1, ctypes.byref(d)) == cs.CS_EINVAL
    t = ctypes.c_uint64()
    p = cs.cs_params_default()
    assert cs.lib().cs_server_submit(None, None, ctypes.byref(p), 1, ctypes.byref(t)) == cs.CS_EINVAL


@pytest.mark.gpu
def test_small_requests_backfill_beside_a_large_one():
    """A large request leaves a few SMs; small requests submitted after it start
    while it runs, and a second large request waits until the first has
    finished (one large request at a time)."""
    base = cs_inputs.WORKLOADS["single_n200_fp64"]
    big = (cs_inputs.random_instance(2000, 1200, 200, 0.01, 0.03, seed=5),
           dict(cs_inputs.WORKLOADS["trials64_n2000_fp32"], n_outer=2, n_steps=1500), 64)
    # FP32 small requests: 2-CTA grids, so both fit in the SMs the large one leaves
    small = (cs_inputs.random_instance(200, 120, 20, 0.0, 0.05, seed=6),
             dict(base, n_outer=2, n_steps=300, precision="fp32"), 1)
    sv = cs.cs_server_create(8 << 30, 8)
    try:
        order = [big, small, small, big]
        tickets = [cs.cs_server_submit_host(sv, i.A, i.y, i.lam, cs.params_from_workload(w), T) for i, w, T in order]
        times = []
        for (inst, w, T), t in zip(order, tickets):
            cs.cs_server_wait(sv, t)
            times.append(cs.cs_server_result(sv, t, inst.N)[4])
    finally:
        cs.cs_server_destroy(sv)
    b1, s1, s2, b2 = times
    assert s1[1] < b1[2] and s2[1] < b1[2]  # the small ones started before the first large one finished
    assert b2[1] >= b1[2]                   # the second large one waited for the first


@pytest.mark.gpu
def test_requests_on_a_cached_problem():
    """cs_server_submit on a problem made once by cs_problem_create: two requests
    with different seeds (and a third with more trials) reuse its Gram, run one
    after the other on it, and each matches the oracle with its own parameters;
    afterwards the problem is back on its own stream and solves directly."""
    import torch
    inst = cs_inputs.random_instance(200, 120, 20, 0.0, 0.05, seed=0)
    base = dict(cs_inputs.WORKLOADS["single_n200_fp64"], n_outer=2, n_steps=500)
    h = cs.cs_problem_create(torch.from_numpy(inst.A).cuda(), torch.from_numpy(inst.y).cuda(), inst.lam)
    G0 = cs.cs_problem_gram(h)[0]
    sv = cs.cs_server_create(8 << 30, 4)
    reqs = [(dict(base, seed=1), 1), (dict(base, seed=2), 1), (dict(base, seed=3), 3)]
    try:
        tickets = [cs.cs_server_submit(sv, h, cs.params_from_workload(w), T) for w, T in reqs]
        results = []
        for t in tickets:
            cs.cs_server_wait(sv, t)
            results.append(cs.cs_server_result(sv, t, inst.N))
    finally:
        cs.cs_server_destroy(sv)
    try:
        for (w, T), res in zip(reqs, results):
            r = oracle.solve(inst.A, inst.y, inst.lam,
                             oracle.Params(**{k: v for k, v in w.items() if k in ORACLE_KEYS}), trials=T)
            np.testing.assert_array_equal(res[1], r["sigma"])
            np.testing.assert_allclose(res[0], r["x_hat"], rtol=0, atol=1e-9)
            assert res[5] == cs.CS_OK
        # the requests ran one after the other on the one problem
        times = [res[4] for res in results]
        assert times[1][1] >= times[0][2] - 1e-3 and times[2][1] >= times[1][2] - 1e-3
        # its Gram is untouched and it is usable directly again
        np.testing.assert_array_equal(cs.cs_problem_gram(h)[0], G0)
        cs.cs_solve(h, cs.params_from_workload(reqs[0][0]), 1)
        x, s, E, st, status = cs.cs_result(h)
        np.testing.assert_allclose(x, results[0][0], rtol=0, atol=1e-9)
    finally:
        cs.cs_problem_destroy(h)


@pytest.mark.gpu
def test_large_request_runs_with_the_planner_split():
    """A request whose grid would take more than half the GPU (N = 2000, 64 trials)
    runs with the planner's own work split over all SMs but 8, beside small
    requests in the SMs it leaves: its result and plan are those of a plain
    cs_solve of the same problem with max_ctas = SMs - 8."""
    import torch

    base = cs_inputs.WORKLOADS["single_n200_fp64"]
    small = [(cs_inputs.random_instance(200, 120, 20, 0.0, 0.05, seed=40 + k), dict(base, n_outer=2, n_steps=400), 1)
             for k in range(3)]
    big = cs_inputs.random_instance(2000, 1200, 200, 0.01, 0.03, seed=7)
    wbig = dict(cs_inputs.WORKLOADS["trials64_n2000_fp32"], n_outer=2, n_steps=300)
    reqs = small[:2] + [(big, wbig, 64)] + small[2:]
    res = _serve(reqs, slots=4, budget=64 << 30)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    h = cs.cs_problem_create(torch.from_numpy(big.A).cuda(), torch.from_numpy(big.y).cuda(), big.lam)
    try:
        cs.cs_solve(h, cs.params_from_workload(wbig, max_ctas=sms - 8), 64)
        x, s, E, st, _ = cs.cs_result(h)
    finally:
        cs.cs_problem_destroy(h)
    assert res[2][3][8] == st[8] and res[2][3][9] == st[9] and res[2][3][10] == st[10]
    np.testing.assert_array_equal(res[2][0], x)
    np.testing.assert_array_equal(res[2][1], s)
