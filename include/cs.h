/*
 * cs.h -- C ABI of the GB300 (sm_103a) solver for L0-regularised compressed
 * sensing by the mean-field coherent Ising machine with chaotic amplitude
 * control and a classical refit (CAC-MFZ-CDP, arXiv 2405.00366).
 *
 * The solver minimises  E(R, sigma) = 1/2 ||y - A (sigma o R)||^2 + lambda ||sigma||_0
 * (Eq. doublel0) by the alternating loop of Algorithm 1: for each outer
 * iteration it integrates the mean-field CIM amplitude equations (Eq. mfeq1,
 * Eq. MFZlocalfieldmain, Eq. GMFZEC5 with the local field of Eq. localfieldMFZ
 * or Eq. localfieldMFZBN) by explicit Euler steps, reads the support
 * sigma = H(c) off the final amplitudes, and refits R on that support.
 *
 * Conventions for every call:
 *  - Every call returns a cs_status; none aborts the process and no kernel
 *    traps.  On failure cs_last_error() gives a message (thread-local).
 *  - The caller keeps ownership of every pointer it passes.  Host buffers are
 *    read or written before the call returns unless stated otherwise.
 *  - The library owns all device memory it allocates; it is released by
 *    cs_problem_destroy.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is queued on it in order.
 *  - Threads: calls on different problems (and servers) may be made from
 *    different host threads at the same time; calls on one problem must not
 *    overlap each other.
 *  - Matrices are row-major.  Per-trial arrays are laid out [r][t]: element
 *    (r, t) of an N x T array is at r * T + t.
 */
#ifndef CS_H
#define CS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CS_OK = 0,
  CS_EINVAL = 1,      /* bad argument (sizes, NaN input, parameters) */
  CS_ENOMEM = 2,      /* device allocation failed or HBM budget exceeded */
  CS_ECUDA = 3,       /* a CUDA runtime call failed; see cs_last_error() */
  CS_ETIMEOUT = 4,    /* a device-side wait exceeded params.timeout_ms; results invalid */
  CS_ENOTREADY = 5,   /* no solve has completed on this problem yet */
  CS_ESINGULAR = 6    /* warning: a refit needed the ridge; results are valid */
} cs_status;

enum { CS_FIELD_CN = 0, CS_FIELD_BN = 1 };          /* Eq. localfieldMFZ / Eq. localfieldMFZBN */
enum { CS_REFIT_EXACT = 0, CS_REFIT_JACOBI = 1, CS_REFIT_CG = 2 }; /* normal equations / damped Jacobi /
                                                                       conjugate gradient */
enum { CS_PUMP_LINEAR = 0, CS_PUMP_SIGMOID = 1 };   /* p0 -> p1 ramp / Eq. pumprateGACS */
enum { CS_INIT_UNIFORM = 0, CS_INIT_NORMAL = 1 };   /* U(-s, s) / N(0, s^2) */
enum { CS_READOUT_FINAL = 0, CS_READOUT_BEST = 1 }; /* sigma of a CIM run: last / best visited */
enum { CS_INIT_R_ZEEMAN = 0, CS_INIT_R_LASSO = 1 }; /* initial R: h^z / diag G / the LASSO solution */
/* Storage precision of the coupling matrix G and arithmetic of the Euler loop:
 * FP64 keeps G and the amplitudes in double; the others accumulate in float.
 * FP8 is E4M3 with one FP32 scale per row of G_off (its largest magnitude / 448). */
enum { CS_P_FP64 = 0, CS_P_FP32 = 1, CS_P_BF16 = 2, CS_P_FP16 = 3, CS_P_FP8 = 4 };

/* Run parameters (Methods and Numerical experiments of the paper).
 * Fill with cs_params_default() and override. */
typedef struct {
  int32_t n_outer;      /* outer iterations of Algorithm 1 (>= 1) */
  int32_t n_steps;      /* Euler steps per CIM run (>= 1) */
  double dt;            /* Euler step (> 0) */
  int32_t pump_kind;    /* CS_PUMP_* */
  double p0, p1;        /* linear pump: p(t_n) = p0 + (p1 - p0) n / n_steps */
  double p_thr, d, t0, width; /* sigmoid pump: (p_thr - d) + 2d / (1 + exp(-(t - t0)/width)) */
  double beta;          /* CAC feedback rate, Eq. GMFZEC5 */
  double tau;           /* target amplitude (> 0) */
  double K;             /* feedback strength, Eq. mfeq1 */
  double j;             /* out-coupling rate, Eq. MFZlocalfieldmain */
  double eta_init;      /* <= 0: fixed eta = sqrt(2 lambda); else Eq. etaSchedulling */
  double eta_end, velo;
  int32_t init_kind;    /* CS_INIT_*: initial amplitudes of each CIM run */
  double init_scale;
  int32_t field;        /* CS_FIELD_* */
  int32_t refit;        /* CS_REFIT_* */
  double jacobi_dt;     /* damped Jacobi step (paper: 0.1) */
  int32_t jacobi_iters; /* damped Jacobi sweeps per outer iteration (paper: 100) */
  int32_t precision;    /* CS_P_* */
  uint64_t seed;        /* key of the counter-based initial-amplitude generator */
  int32_t instance;     /* instance number mixed into that key */
  int32_t record_steps; /* record c, e after each of the first k steps of outer iteration 0 */
  int64_t timeout_ms;   /* bound on every device-side wait (grid barrier) */
  int32_t test_phantom_ctas; /* test hook: the grid barrier also waits for this many CTAs that
                                do not exist, so it runs into timeout_ms; in a batch, > 0 makes
                                each CTA's first ring copy never issued, so the waits on it
                                run into timeout_ms; 0 in normal use */
  int32_t cluster_size; /* CTAs per thread-block cluster of the Euler kernel: 0 = chosen by the
                           library's planner, or 1, 2, 4, 8; in a batch, the first problem of a
                           group fixes the batched kernel's cluster size this way */
  int32_t max_ctas;     /* at most this many CTAs (SMs) per Euler launch, 0 = all; lets solves
                           on different streams share the GPU */
  int32_t stream_g;     /* 0: keep G_off on chip when it fits, else stream its tiles from memory
                           every step; 1: always stream (FP32/BF16/FP16/FP8 only) */
  int32_t autotune;     /* 0: the planner's cost model picks the Euler work split (deterministic);
                           1: the first solve of a shape in this process times the cost model's
                           four cheapest splits on this GPU (48 steps each, synchronising the
                           problem's stream) and keeps the fastest for later solves; in a batch,
                           the first batch of a shape times the batched kernel's cluster sizes
                           and ring shapes (48 steps of every problem each).  Choices persist
                           across processes in the tuning cache file (cs_tune_info) */
  int32_t tensor_form;  /* the product G_off X on the tensor cores.  FP32 problems with trial
                           blocks of 16, 32 or 64: G_off and X each split into two FP16 parts
                           (FP32-level accuracy), either on the tcgen05 tensor cores (one
                           M = 128 MMA per 16 k on the stacked parts, TMEM accumulators;
                           resident G_off, at most 64 rows per cluster) or on the mma.sync
                           path (three MMAs per tile); streamed FP16 / BF16 G_off with exactly
                           8 trials (mma.sync), and batches of FP16 / BF16 problems with 8 or
                           16 trials (tcgen05 or mma.sync: the stored G_off times X in two
                           16-bit parts).  X is
                           scaled by a power of two from max |R|, so |X| <= |c| and FP16 X
                           overflows only on runs whose explicit Euler steps already diverge.
                           0: the planner chooses among every form; 1: FMA forms only;
                           2: tensor-core forms only; 3: mma.sync tensor-core forms only;
                           4: the tcgen05 forms only (single solves: resident FP32 G_off;
                           batches: BF16 / FP16 G_off with 8 or 16 trials, one M = 128 MMA
                           per 128-row tile and 16 k, TMEM accumulators, the batched default
                           where it applies).  2, 3 and 4 make the solve fail with CS_EINVAL
                           where no such form applies */
  int32_t self_term;    /* 0: the injection of Eq. MFZlocalfieldmain as written (its Hamiltonian,
                           Eq. l0Hamiltonian, has no self-term, so a spin at its refit value turns
                           on when G_rr R_r^2 > lambda); 1: corrected mode, the injection also
                           subtracts (sqrt tau / 4) G_rr R_r^2, so that it turns on when
                           1/2 G_rr R_r^2 > lambda, the single-spin decision of Eq. doublel0 */
  int32_t readout;      /* CS_READOUT_FINAL: sigma = H(c) at the end of each CIM run (the paper);
                           CS_READOUT_BEST: the first configuration H(c_n), n = 1 .. n_steps, of
                           lowest objective (Eq. doublel0 at the run's R, lambda = eta^2 / 2), the
                           readout the paper's discussion proposes.  BEST needs the binarised field
                           (its product is the configuration's coupling term) and single solves;
                           each run then keeps a history of (n_steps + 1) x N x trials bytes and
                           (n_steps + 1) x CTAs x trials doubles on the device */
  int32_t cg_iters;     /* CS_REFIT_CG (the paper's CDP for MRI data): conjugate gradient on
                           G_SS R_S = (A^T y)_S in FP64, warm started from the trial's R, at most
                           cg_iters iterations (paper: 10000) ... */
  double cg_tol;        /* ... and until ||(A^T y)_S - G_SS R_S||_2 <= cg_tol ||(A^T y)_S||_2; off
                           the support R is the Jacobi fixed point, as for the exact refit */
  int32_t record_outer; /* 1: keep sigma and R after every outer iteration (single solves; read
                           with cs_outer_history): n_outer x N x trials bytes and doubles */
  int32_t init_R;       /* R before the first CIM run: CS_INIT_R_ZEEMAN, h^z / diag G (the refit of
                           the empty support); CS_INIT_R_LASSO, the LASSO solution (the paper's
                           initial condition for its MRI runs), argmin 1/2 ||y - A x||^2 +
                           lasso_lambda ||x||_1 by lasso_iters FISTA iterations from 0 in FP64
                           (step 1 / the largest absolute row sum of G); single solves */
  int32_t lasso_iters;
  double lasso_lambda;
} cs_params;

typedef struct cs_problem cs_problem;

/* Defaults: 20 x 1000 steps, dt 0.01, linear pump 0 -> 1.5, beta 0.2, tau 1,
 * K = j = 1, fixed eta, U(-0.01, 0.01) initial amplitudes, continuous field,
 * exact refit (damped Jacobi: step 0.1, 100 sweeps; conjugate gradient: 10000
 * iterations, tolerance 1e-10), FP32, seed 0, no recording, 10 s timeout. */
void cs_params_default(cs_params* p);

/* Create a problem from A (M x N, row-major, float64) and y (M, float64) and
 * form, on the GPU, G = A^T A (FP64), h^z = A^T y and g = diag G
 * (Eq. l0Hamiltonian and the Zeeman term of Eq. localfieldMFZ).  G is then
 * kept resident for every solve on this problem.
 *  on_device = 0: A, y are host pointers (copied to the device);
 *  on_device = 1: A, y are device pointers, read on `stream` before return.
 * Errors: CS_EINVAL for M, N < 1, lambda < 0 or NULL pointers; CS_ENOMEM;
 * CS_ECUDA.  A and y are checked for finite values on the device. */
cs_status cs_problem_create(const double* A, const double* y, int64_t M, int64_t N,
                            double lambda, int on_device, void* stream, cs_problem** out);

/* Queue one full solve (Algorithm 1, every outer iteration) of `trials`
 * independent trials on the problem's stream; returns without waiting.
 * Trial t draws its initial amplitudes from key (seed, instance, t, outer).
 * The exact refit returns the FP64 least-squares solution on the support: an
 * FP32 Cholesky factor (in shared memory, or blocked in global memory for
 * large supports) with FP64 iterative refinement, else an FP64 Cholesky, with
 * the ridge for numerically singular G_SS (CS_ESINGULAR).  With autotune = 1
 * the first solve of a shape synchronises the stream while it times splits.
 * Errors: CS_EINVAL for bad parameters or trials < 1; CS_ENOMEM; CS_ECUDA. */
cs_status cs_solve(cs_problem* p, const cs_params* prm, int32_t trials);

/* Queue one full solve (Algorithm 1) of every problem ps[0..n) as a batch:
 * problem i with its own parameters *prm[i] and trials[i] (<= 64) trials.
 * Problems that share a storage precision, a trial count and the tensor-core
 * decision form a group; each outer iteration of a group is one persistent
 * launch of thread-block clusters that take problems from a device work queue
 * (largest N first) and stream each problem's G_off tiles from memory: a
 * large problem (at least two 128-row tiles per CTA) is run by a whole
 * cluster, the CTAs splitting its row tiles and meeting at the cluster barrier
 * after every Euler step, a small one by one CTA alone.  The cluster size
 * (1, 2, 4, 8) is the group's first problem's cluster_size when that is not
 * 0; otherwise, and for the ring shape, the batch autotuner chooses when a
 * problem of the group sets autotune = 1, else clusters of one CTA.  Then
 * one refit launch covers every (problem, trial) of the group.  A problem
 * leaves the batch after its own n_outer iterations.  All outer iterations and
 * the objective are captured into one CUDA graph, submitted to the problems'
 * stream as a single launch.  Problem i draws its initial amplitudes with
 * instance number i (prm[i]->instance is not used).  All problems must have
 * been created on the same device and stream and appear once each.  Results
 * are read per problem with cs_result / cs_result_trials.
 * ps, prm and trials are host arrays of n entries.
 * Errors: CS_EINVAL (parameters, trials > 64, record_steps != 0, mixed
 * streams, a problem given twice, tensor_form >= 2 without a batched
 * tensor-core form), CS_ENOMEM, CS_ECUDA. */
cs_status cs_solve_batch(cs_problem* const* ps, const cs_params* const* prm, const int32_t* trials, int32_t n);

/* The autotuners' record: *tunings = timed tuning runs in this process,
 * *disk_hits = choices taken from the tuning cache file instead, and path
 * (path_len bytes, NUL-terminated, may be NULL) = that file: $CS_TUNE_CACHE if
 * set (empty: no file), else $XDG_CACHE_HOME/paper_2405_00366_gb300/tune.txt,
 * else $HOME/.cache/paper_2405_00366_gb300/tune.txt.  Host only; never fails. */
cs_status cs_tune_info(int64_t* tunings, int64_t* disk_hits, char* path, int64_t path_len);

/* Wait for the last solve and copy out the kept trial (lowest energy, ties to
 * the lower trial index): x_hat = sigma o R (N doubles), sigma_hat (N bytes,
 * 0/1) and its energy (Eq. doublel0 with the problem's lambda, recomputed from
 * A and y in FP64).  Any output pointer may be NULL.  stats, if not NULL,
 * receives CS_STATS_LEN doubles:
 *   [0] kept trial index  [1] |sigma_hat|  [2] 1 if a refit used the ridge
 *   [3] device error word (0 = none)       [4] trials  [5] N  [6] M
 *   [7] energy of the kept trial  [8] cluster size (batched: CTAs that ran the problem) and [9] CTAs of the Euler kernel
 *   [10] form of the Euler kernel: 0 FP32/FP64 FMAs (narrow split), 1 packed FP32
 *        FMAs (wide split), 2 tensor cores (mma.sync), 3 batched (one problem per CTA),
 *        4 batched on tensor cores (mma.sync), 5 tensor cores (tcgen05, TMEM),
 *        6 batched on tensor cores (tcgen05, TMEM)
 *   [11] error of the coupling against FP64: max_r |(G_off^s x_hat)_r - (G_off x_hat)_r|
 *        / max_r |(G_off x_hat)_r|, G_off^s being G_off rounded to the storage precision
 *        the Euler kernels used (0 for FP64), both products formed in FP64
 *   [12] FP64 residual of the refit: max over the support of |h^z_r - (G x_hat)_r| /
 *        max over the support of |h^z_r| (the normal equations G_SS R_S = h^z_S of
 *        Algorithm 1's refit; about 1e-15 for the exact refit, larger with the ridge
 *        or the damped Jacobi refit)
 * Host pointers.  Returns CS_ETIMEOUT if a device wait timed out,
 * CS_ESINGULAR (with valid outputs) if the ridge was needed. */
#define CS_STATS_LEN 13
cs_status cs_result(cs_problem* p, double* x_hat, uint8_t* sigma_hat, double* energy,
                    double* stats);

/* Per-trial results of the last solve (host pointers, any may be NULL):
 * R (N x trials, [r][t]), sigma (N x trials bytes), energy (trials),
 * support_sizes (n_outer x trials int32: |sigma| after each outer iteration). */
cs_status cs_result_trials(cs_problem* p, double* R, uint8_t* sigma, double* energy,
                           int32_t* support_sizes);

/* The recorded amplitudes of the last solve: c and e after each of the first
 * params.record_steps Euler steps of outer iteration 0, as doubles laid out
 * [step][r][t] (record_steps x N x trials).  Host pointers. */
cs_status cs_trajectory(cs_problem* p, double* c, double* e);

/* sigma and R of every trial after each outer iteration of the last solve
 * (params.record_outer = 1), laid out [outer][r][t]: n_outer x N x trials bytes
 * and doubles.  Host pointers, either may be NULL.  CS_EINVAL if the solve did
 * not record them. */
cs_status cs_outer_history(cs_problem* p, uint8_t* sigma, double* R);

/* Copy the FP64 Gram data formed by cs_problem_create to host buffers
 * (any may be NULL): G (N x N), h^z = A^T y (N), g = diag G (N). */
cs_status cs_problem_gram(cs_problem* p, double* G, double* hz, double* g);

/* Device time of the work queued by the last cs_problem_create and the last
 * cs_solve on this problem (for the first problem of a cs_solve_batch: the
 * whole batch's Euler launches, refits and objective), from CUDA events recorded on the problem's stream
 * around each group of launches (event-record nodes inside the solve's graph),
 * summed per group into ms[0..3]:
 *   [0] Gram formation  [1] Euler kernels (all outer iterations)
 *   [2] refits          [3] the rest (coupling copy, initial R, objective, selection)
 *   [4] (a count, not a time) host submissions of the last cs_solve's device
 *       work: the kernels it queued directly (coupling copy, initial R) plus
 *       one CUDA graph launch that holds every outer iteration and the objective
 * and, in *launches, how many kernels the library launched for them, inside
 * the graph or not.  Waits for the stream.  Host pointers, either may be NULL. */
#define CS_TIMING_LEN 5
cs_status cs_problem_timing(cs_problem* p, double* ms, int64_t* launches);

/* Per-trial objective E_t = 1/2 ||y - A (sigma_t o R_t)||^2 + lambda |sigma_t| in
 * FP64, for callers that cannot allocate device memory.  The paper has no
 * counterpart: this entry point exists for callers that may not call
 * cudaMalloc or any allocating routine, such as code running during CUDA graph
 * capture, hosts that own all device memory through their own arena, or
 * loops where an allocation is not allowed.  It allocates nothing.
 *  A (M x N row-major), y (M), sigma (N x trials bytes, [r][t]), R (N x trials,
 *  [r][t]) and energy (trials) are DEVICE pointers owned by the caller; the
 *  kernel is queued on `stream` and the call returns without waiting.
 *  Scratch: a fixed device array of 262144 int32 entries (1 MiB) inside the
 *  library, held by every GPU that loads the library until exit; N * trials
 *  must not exceed 262144 (CS_EINVAL otherwise).  Every call shares that array
 *  and it keeps the last call's contents (each call writes every entry it
 *  reads), so calls whose kernels overlap on the GPU (for example on two
 *  streams) race and give wrong results; serialise them.
 *  The first call on a device looks up the array's device address with that
 *  device current; make that first call before any stream capture.
 * Errors: CS_EINVAL (NULL pointer, sizes, lambda), CS_ECUDA (lookup or launch). */
cs_status cs_objective_static(const double* A, const double* y, const uint8_t* sigma, const double* R, int64_t M,
                              int64_t N, int32_t trials, double lambda, double* energy, void* stream);

/* Sizes of a problem. */
cs_status cs_problem_shape(const cs_problem* p, int64_t* M, int64_t* N);

/* Release everything the problem owns.  NULL is ignored. */
void cs_problem_destroy(cs_problem* p);

/* ---- Serving: a continuous-batching request loop over the solver.
 * A server owns `max_slots` CUDA streams on the current device and a worker
 * thread.  A small request gets an Euler grid sized to its work (unless
 * params.max_ctas is set): one CTA per 26e6 coupling FMAs per step (N^2 x
 * trials) and per 150 KB of G_off in its storage precision, at least 2 (8 for
 * FP64), run as cooperative launches with clusters of one.  A request whose
 * grid would take more than half the SMs is large: it runs with the planner's
 * own work split (clusters) over all SMs but 8 (or the caller's cluster_size
 * and max_ctas), one large request at a time, and small requests run beside it
 * in the SMs it leaves.  Submitted requests are scanned in arrival order; each
 * is admitted when a slot is free, its device-memory estimate fits what is left
 * of `hbm_budget_bytes` and its grid fits the SMs not held by running requests
 * (a small request that does not fit yet does not hold back smaller ones behind
 * it; a large one at the head waits, admitting nothing behind it, until no
 * other large request runs and the small ones fit in its reserve).  An admitted
 * request takes its problem (the caller's, or one it forms from host data) and
 * queues its solve on its slot's stream, so the solves of several requests
 * overlap on the GPU.
 * When a solve finishes, the worker copies its result to host memory and
 * releases its device memory, SMs and slot at once.  A result is the same
 * whether the request ran alone or among others (same work split, fixed
 * summation order). */
typedef struct cs_server cs_server;

/* Errors: CS_EINVAL (max_slots outside [1, 256], zero budget), CS_ECUDA. */
cs_status cs_server_create(size_t hbm_budget_bytes, int32_t max_slots, cs_server** out);

/* Queue one reconstruction of the caller's problem p (made by
 * cs_problem_create): its G, h^z and g, formed once at creation, serve every
 * request on it, so a problem solved again (another seed, lambda schedule or
 * trial count) costs no new Gram.  params and trials as for cs_solve (for a
 * small request the server sets cluster_size = 1 and, if 0, max_ctas as above;
 * a large one keeps them, max_ctas 0 becoming all SMs but 8).  While the request runs
 * the problem is the server's: its work moves to one of the server's streams
 * (ordered after what was already queued on the problem's own stream) and
 * returns to the problem's stream when the request finishes; requests on the
 * same problem run one after the other.  The caller must not use or destroy p
 * until the request has finished.  *ticket names the request.
 * Errors: CS_EINVAL (NULL arguments, trials < 1), CS_ENOMEM if the request can
 * never fit the budget. */
cs_status cs_server_submit(cs_server* sv, cs_problem* p, const cs_params* prm, int32_t trials, uint64_t* ticket);

/* Queue one reconstruction from host data: A (M x N row-major) and y (M) are
 * HOST pointers, copied before the call returns; the server forms the problem
 * (its Gram) when it admits the request and frees it when the request ends.
 * Otherwise as cs_server_submit. */
cs_status cs_server_submit_host(cs_server* sv, const double* A, const double* y, int64_t M, int64_t N, double lambda,
                                const cs_params* prm, int32_t trials, uint64_t* ticket);

/* Non-blocking: *done = 1 once the request has finished (or failed). */
cs_status cs_server_poll(cs_server* sv, uint64_t ticket, int32_t* done);

/* Block until the request has finished, at most timeout_ms (CS_ENOTREADY after). */
cs_status cs_server_wait(cs_server* sv, uint64_t ticket, int64_t timeout_ms);

/* Copy a finished request's result (host pointers, any may be NULL) and forget
 * the ticket: x_hat (N), sigma_hat (N), energy, stats (CS_STATS_LEN, as for
 * cs_result) and times[3] = submit, start (admission) and finish instants in
 * seconds of a monotonic clock.  Returns the solve's status (CS_OK,
 * CS_ESINGULAR or its error), CS_ENOTREADY if it has not finished. */
cs_status cs_server_result(cs_server* sv, uint64_t ticket, double* x_hat, uint8_t* sigma_hat, double* energy,
                           double* stats, double* times);

/* Finish running requests, drop queued ones, release everything. */
void cs_server_destroy(cs_server* sv);

/* Message for the last failing call on this thread ("" if none). */
const char* cs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CS_H */
