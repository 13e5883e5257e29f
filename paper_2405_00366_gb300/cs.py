"""Thin ctypes binding of libcs.so (include/cs.h), with the same names.

Only argument marshalling happens here: every step of the solve runs in the
library's CUDA kernels.  PyTorch tensors may be passed for A and y (host or
CUDA); their data pointer is handed to the library, and a torch stream may be
given as the work queue.  If libcs.so is missing this module raises at first
use: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcs.so")

CS_OK, CS_EINVAL, CS_ENOMEM, CS_ECUDA, CS_ETIMEOUT, CS_ENOTREADY, CS_ESINGULAR = range(7)
STATUS_NAMES = {0: "CS_OK", 1: "CS_EINVAL", 2: "CS_ENOMEM", 3: "CS_ECUDA", 4: "CS_ETIMEOUT",
                5: "CS_ENOTREADY", 6: "CS_ESINGULAR"}
CS_FIELD_CN, CS_FIELD_BN = 0, 1
CS_REFIT_EXACT, CS_REFIT_JACOBI, CS_REFIT_CG = 0, 1, 2
CS_PUMP_LINEAR, CS_PUMP_SIGMOID = 0, 1
CS_INIT_UNIFORM, CS_INIT_NORMAL = 0, 1
CS_P_FP64, CS_P_FP32, CS_P_BF16, CS_P_FP16, CS_P_FP8 = 0, 1, 2, 3, 4
CS_STATS_LEN = 13

PRECISIONS = {"fp64": CS_P_FP64, "fp32": CS_P_FP32, "bf16": CS_P_BF16, "fp16": CS_P_FP16, "fp8": CS_P_FP8}
FIELDS = {"cn": CS_FIELD_CN, "bn": CS_FIELD_BN}
PUMPS = {"linear": CS_PUMP_LINEAR, "sigmoid": CS_PUMP_SIGMOID}
INITS = {"uniform": CS_INIT_UNIFORM, "normal": CS_INIT_NORMAL}
REFITS = {"exact": CS_REFIT_EXACT, "jacobi": CS_REFIT_JACOBI, "cg": CS_REFIT_CG}
CS_READOUT_FINAL, CS_READOUT_BEST = 0, 1
READOUTS = {"final": CS_READOUT_FINAL, "best": CS_READOUT_BEST}
CS_INIT_R_ZEEMAN, CS_INIT_R_LASSO = 0, 1
INIT_RS = {"zeeman": CS_INIT_R_ZEEMAN, "lasso": CS_INIT_R_LASSO}


class cs_params(ctypes.Structure):
    """Mirror of the C struct cs_params (field order and types must match cs.h)."""

    _fields_ = [
        ("n_outer", ctypes.c_int32), ("n_steps", ctypes.c_int32), ("dt", ctypes.c_double),
        ("pump_kind", ctypes.c_int32), ("p0", ctypes.c_double), ("p1", ctypes.c_double),
        ("p_thr", ctypes.c_double), ("d", ctypes.c_double), ("t0", ctypes.c_double), ("width", ctypes.c_double),
        ("beta", ctypes.c_double), ("tau", ctypes.c_double), ("K", ctypes.c_double), ("j", ctypes.c_double),
        ("eta_init", ctypes.c_double), ("eta_end", ctypes.c_double), ("velo", ctypes.c_double),
        ("init_kind", ctypes.c_int32), ("init_scale", ctypes.c_double),
        ("field", ctypes.c_int32), ("refit", ctypes.c_int32), ("jacobi_dt", ctypes.c_double),
        ("jacobi_iters", ctypes.c_int32), ("precision", ctypes.c_int32), ("seed", ctypes.c_uint64),
        ("instance", ctypes.c_int32), ("record_steps", ctypes.c_int32), ("timeout_ms", ctypes.c_int64),
        ("test_phantom_ctas", ctypes.c_int32), ("cluster_size", ctypes.c_int32), ("max_ctas", ctypes.c_int32),
        ("stream_g", ctypes.c_int32), ("autotune", ctypes.c_int32), ("tensor_form", ctypes.c_int32),
        ("self_term", ctypes.c_int32), ("readout", ctypes.c_int32),
        ("cg_iters", ctypes.c_int32), ("cg_tol", ctypes.c_double), ("record_outer", ctypes.c_int32),
        ("init_R", ctypes.c_int32), ("lasso_iters", ctypes.c_int32), ("lasso_lambda", ctypes.c_double),
    ]


class CSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """The loaded libcs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        L.cs_params_default.argtypes = [ctypes.POINTER(cs_params)]
        L.cs_params_default.restype = None
        L.cs_problem_create.argtypes = [P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_int, P,
                                        ctypes.POINTER(P)]
        L.cs_solve.argtypes = [P, ctypes.POINTER(cs_params), ctypes.c_int32]
        L.cs_solve_batch.argtypes = [ctypes.POINTER(P), ctypes.POINTER(ctypes.POINTER(cs_params)),
                                     ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]
        L.cs_result.argtypes = [P, P, P, P, P]
        L.cs_result_trials.argtypes = [P, P, P, P, P]
        L.cs_trajectory.argtypes = [P, P, P]
        L.cs_problem_gram.argtypes = [P, P, P, P]
        L.cs_outer_history.argtypes = [P, P, P]
        L.cs_problem_timing.argtypes = [P, P, ctypes.POINTER(ctypes.c_int64)]
        L.cs_objective_static.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_double, P, P]
        L.cs_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(P)]
        L.cs_server_submit.argtypes = [P, P, ctypes.POINTER(cs_params), ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_uint64)]
        L.cs_server_submit_host.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                            ctypes.POINTER(cs_params), ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]
        L.cs_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32)]
        L.cs_server_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_int64]
        L.cs_server_result.argtypes = [P, ctypes.c_uint64, P, P, P, P, P]
        L.cs_server_destroy.argtypes = [P]
        L.cs_server_destroy.restype = None
        L.cs_problem_shape.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.cs_tune_info.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), P,
                                   ctypes.c_int64]
        L.cs_problem_destroy.argtypes = [P]
        L.cs_problem_destroy.restype = None
        L.cs_last_error.argtypes = []
        L.cs_last_error.restype = ctypes.c_char_p
        for name in ["cs_problem_create", "cs_solve", "cs_solve_batch", "cs_result", "cs_result_trials", "cs_trajectory",
                     "cs_outer_history",
                     "cs_problem_gram", "cs_problem_shape", "cs_problem_timing", "cs_objective_static",
                     "cs_server_create", "cs_server_submit", "cs_server_submit_host", "cs_server_poll",
                     "cs_server_wait", "cs_server_result", "cs_tune_info"]:
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def cs_last_error() -> str:
    return lib().cs_last_error().decode()


def _check(status: int, allow=(CS_OK,)) -> int:
    if status not in allow:
        raise CSError(status, cs_last_error())
    return status


def cs_params_default(**overrides) -> cs_params:
    """cs_params filled by the library's defaults, then `overrides` (names as in cs.h;
    the string forms 'fp32', 'cn', 'linear', 'uniform', 'exact', 'best' are accepted)."""
    p = cs_params()
    lib().cs_params_default(ctypes.byref(p))
    maps = {"precision": PRECISIONS, "field": FIELDS, "pump_kind": PUMPS, "init_kind": INITS, "refit": REFITS,
            "readout": READOUTS, "init_R": INIT_RS}
    for k, v in overrides.items():
        if k in maps and isinstance(v, str):
            v = maps[k][v]
        if isinstance(v, bool):
            v = int(v)
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr_and_kind(x):
    """(pointer, on_device, keepalive) of a float64 host/device buffer."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.float64 or not x.is_contiguous():
                x = x.to(torch.float64).contiguous()
            return x.data_ptr(), 1 if x.is_cuda else 0, x
    except ImportError:  # pragma: no cover
        pass
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a.ctypes.data, 0, a


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


def cs_problem_create(A, y, lam: float, stream=None):
    """Handle of a new problem (see cs.h).  A: (M, N), y: (M,), host or CUDA float64."""
    pa, da, ka = _ptr_and_kind(A)
    py, dy, ky = _ptr_and_kind(y)
    if da != dy:
        raise ValueError("A and y must both be on the host or both on the device")
    M, N = (int(s) for s in A.shape)
    h = ctypes.c_void_p()
    _check(lib().cs_problem_create(pa, py, M, N, float(lam), da, _stream_ptr(stream), ctypes.byref(h)))
    del ka, ky
    return h


def cs_solve(problem, params: cs_params, trials: int) -> None:
    _check(lib().cs_solve(problem, ctypes.byref(params), int(trials)))


def cs_solve_batch(problems, params, trials) -> None:
    """Queue one batched solve of several problems (same stream).  `params` is one
    cs_params for every problem or a sequence with one per problem; `trials` is one
    int or a sequence with one per problem."""
    n = len(problems)
    arr = (ctypes.c_void_p * n)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in problems])
    plist = list(params) if isinstance(params, (list, tuple)) else [params] * n
    tlist = list(trials) if isinstance(trials, (list, tuple, np.ndarray)) else [trials] * n
    if len(plist) != n or len(tlist) != n:
        raise ValueError("one params and one trial count per problem")
    pp = (ctypes.POINTER(cs_params) * n)(*[ctypes.pointer(q) for q in plist])
    tt = (ctypes.c_int32 * n)(*[int(t) for t in tlist])
    _check(lib().cs_solve_batch(arr, pp, tt, n))


def cs_result(problem):
    """(x_hat (N,), sigma_hat (N,) uint8, energy, stats (CS_STATS_LEN,), status)."""
    M, N = cs_problem_shape(problem)
    x = np.empty(N)
    s = np.empty(N, dtype=np.uint8)
    e = ctypes.c_double()
    st = np.empty(CS_STATS_LEN)
    status = _check(lib().cs_result(problem, x.ctypes.data, s.ctypes.data, ctypes.addressof(e), st.ctypes.data),
                    allow=(CS_OK, CS_ESINGULAR))
    return x, s, e.value, st, status


def cs_result_trials(problem, trials: int, n_outer: int):
    """(R (N, T), sigma (N, T) uint8, energies (T,), support sizes (n_outer, T))."""
    M, N = cs_problem_shape(problem)
    R = np.empty((N, trials))
    s = np.empty((N, trials), dtype=np.uint8)
    e = np.empty(trials)
    ss = np.empty((n_outer, trials), dtype=np.int32)
    _check(lib().cs_result_trials(problem, R.ctypes.data, s.ctypes.data, e.ctypes.data, ss.ctypes.data),
           allow=(CS_OK, CS_ESINGULAR))
    return R, s, e, ss


def cs_trajectory(problem, record_steps: int, trials: int):
    """(c, e) of the first record_steps Euler steps of outer iteration 0, shape (k, N, T)."""
    M, N = cs_problem_shape(problem)
    c = np.empty((record_steps, N, trials))
    e = np.empty((record_steps, N, trials))
    _check(lib().cs_trajectory(problem, c.ctypes.data, e.ctypes.data), allow=(CS_OK, CS_ESINGULAR))
    return c, e


def cs_problem_gram(problem):
    """(G (N, N), hz (N,), g (N,)) as formed on the GPU in FP64."""
    M, N = cs_problem_shape(problem)
    G = np.empty((N, N))
    hz = np.empty(N)
    g = np.empty(N)
    _check(lib().cs_problem_gram(problem, G.ctypes.data, hz.ctypes.data, g.ctypes.data))
    return G, hz, g


CS_TIMING_LEN = 5


def cs_problem_timing(problem):
    """(ms per group [gram, euler, refit, other] followed by the count of host
    submissions of the last solve, kernel launches) of the last create + solve."""
    ms = np.zeros(CS_TIMING_LEN)
    n = ctypes.c_int64()
    _check(lib().cs_problem_timing(problem, ms.ctypes.data, ctypes.byref(n)))
    return ms, n.value


def cs_objective_static(A, y, sigma, R, lam: float, energy, stream=None) -> None:
    """Per-trial objective into `energy` without any device allocation (see cs.h).
    A (M, N), y (M,), R (N, T) float64, sigma (N, T) uint8 and energy (T,) float64
    must be contiguous CUDA tensors; the work is queued on `stream`."""
    M, N = (int(d) for d in A.shape)
    T = int(R.shape[1])
    for t in (A, y, sigma, R, energy):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("cs_objective_static takes contiguous CUDA tensors")
    _check(lib().cs_objective_static(A.data_ptr(), y.data_ptr(), sigma.data_ptr(), R.data_ptr(), M, N, T,
                                     float(lam), energy.data_ptr(), _stream_ptr(stream)))


def cs_server_create(hbm_budget_bytes: int, max_slots: int):
    h = ctypes.c_void_p()
    _check(lib().cs_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)))
    return h


def cs_server_submit(server, problem, params: cs_params, trials: int) -> int:
    """Queue one request on a problem made by cs_problem_create (its Gram is reused);
    returns its ticket."""
    t = ctypes.c_uint64()
    _check(lib().cs_server_submit(server, problem, ctypes.byref(params), int(trials), ctypes.byref(t)))
    return t.value


def cs_server_submit_host(server, A, y, lam: float, params: cs_params, trials: int) -> int:
    """Queue one request from host arrays (the server forms the problem); returns its ticket."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    t = ctypes.c_uint64()
    _check(lib().cs_server_submit_host(server, A.ctypes.data, y.ctypes.data, A.shape[0], A.shape[1], float(lam),
                                       ctypes.byref(params), int(trials), ctypes.byref(t)))
    return t.value


def cs_server_poll(server, ticket: int) -> bool:
    d = ctypes.c_int32()
    _check(lib().cs_server_poll(server, ticket, ctypes.byref(d)))
    return bool(d.value)


def cs_server_wait(server, ticket: int, timeout_ms: int = 600000) -> None:
    _check(lib().cs_server_wait(server, ticket, int(timeout_ms)))


def cs_server_result(server, ticket: int, N: int):
    """(x_hat, sigma_hat, energy, stats, times[submit, start, done], status) of a finished request."""
    x = np.empty(N)
    s = np.empty(N, dtype=np.uint8)
    e = ctypes.c_double()
    st = np.empty(CS_STATS_LEN)
    tm = np.empty(3)
    status = _check(lib().cs_server_result(server, ticket, x.ctypes.data, s.ctypes.data, ctypes.addressof(e),
                                           st.ctypes.data, tm.ctypes.data), allow=(CS_OK, CS_ESINGULAR))
    return x, s, e.value, st, tm, status


def cs_server_destroy(server) -> None:
    if server:
        lib().cs_server_destroy(server)


def cs_outer_history(problem, n_outer: int, N: int, trials: int):
    """(sigma, R) after each outer iteration of the last solve (record_outer = 1):
    arrays of shape (n_outer, N, trials), uint8 and float64."""
    s = np.empty((n_outer, N, trials), dtype=np.uint8)
    R = np.empty((n_outer, N, trials))
    _check(lib().cs_outer_history(problem, s.ctypes.data, R.ctypes.data), allow=(CS_OK, CS_ESINGULAR))
    return s, R


def cs_tune_info():
    """(timed tunings, choices read from the tuning cache file, that file's path)."""
    t = ctypes.c_int64()
    h = ctypes.c_int64()
    buf = ctypes.create_string_buffer(4096)
    _check(lib().cs_tune_info(ctypes.byref(t), ctypes.byref(h), buf, len(buf)))
    return t.value, h.value, buf.value.decode()


def cs_problem_shape(problem):
    M = ctypes.c_int64()
    N = ctypes.c_int64()
    _check(lib().cs_problem_shape(problem, ctypes.byref(M), ctypes.byref(N)))
    return M.value, N.value


def cs_problem_destroy(problem) -> None:
    if problem:
        lib().cs_problem_destroy(problem)


def params_from_workload(w: dict, **overrides) -> cs_params:
    """cs_params for a workload dict of cs_inputs (names shared with cs.h)."""
    keys = {f for f, _ in cs_params._fields_}
    kw = {k: v for k, v in w.items() if k in keys}
    kw["precision"] = w.get("precision", "fp32")
    kw.update(overrides)
    return cs_params_default(**kw)
