// Host-side declarations shared by the translation units of libcs.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/cs.h"

namespace cs {

void set_last_error(const std::string& msg);

// Stream-ordered device memory from the device's default pool, which keeps
// freed blocks for reuse (no release threshold), so creating and destroying
// problems in a loop does not go back to the driver each time.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// Launch accounting of the last create + solve on a problem: CUDA events
// around each group of launches on the problem's stream, and a launch count.
enum { TM_GRAM = 0, TM_EULER = 1, TM_REFIT = 2, TM_OTHER = 3, TM_COUNT = 4 };

// Rows of G_off are padded to this multiple (k quads of the Euler kernels and
// the 32-column tiles of the streamed layout).
constexpr int64_t kPadN = 32;

// Largest grid of the persistent Euler kernel (one CTA per SM at most).
constexpr int kMaxEulerCtas = 1024;

// Device buffers of one problem (all owned by the library).
struct ProblemDev {
  int64_t M = 0, N = 0, Npad = 0;  // Npad: N rounded up to a multiple of kPadN
  double lambda = 0.0;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  double* A = nullptr;    // M x N
  double* y = nullptr;    // M
  double* G = nullptr;    // N x N, FP64 Gram (full, symmetric)
  double* hz = nullptr;   // N, A^T y
  double* g = nullptr;    // N, diag G
  void* Gs = nullptr;     // Npad x Npad, G in storage precision with zero diagonal and zero padding
  int gs_prec = -1;       // precision held in Gs
  void* Gt = nullptr;     // G_off in storage precision, tiled for streaming (batched solves)
  int gt_prec = -1, gt_frag = 0;
  float* gscale = nullptr; // N row scales of G_off for FP8 storage (largest |G_off[r][k]| / 448)
  void* Gt2 = nullptr;    // G_off tiles of a streaming Euler plan (see euler.cu)
  int gt2_prec = -1, gt2_rpc = 0, gt2_rpcpad = 0, gt2_nc = 0, gt2_frag = 0;
  int* flag = nullptr;    // device word: nonzero if A or y had a non-finite value
  int64_t launches = 0;   // kernels launched by the last create + solve
};

// What the refit, objective and selection kernels need of one problem.
struct RefitJob {
  const double* G;
  const double* hz;
  const double* g;
  const double* A;
  const double* y;
  const uint8_t* sigma;  // N x T
  double* R;             // N x T
  int* sidx;             // T x N support index lists
  int* lead;             // T: trial whose refit this trial copies (itself if none)
  int32_t* ssize;        // n_outer x T support sizes
  double* energy;        // T
  double* x_hat;         // N
  uint8_t* sigma_hat;    // N
  double* stats;         // CS_STATS_LEN
  int N, M, T;
  double lambda;
  int* singular;
  int* err;
  int refit;             // CS_REFIT_EXACT or CS_REFIT_JACOBI
  int jacobi_iters;      // damped Jacobi sweeps per outer iteration
  double jacobi_dt;      // damped Jacobi step
  int cg_iters;          // conjugate-gradient refit: most iterations
  double cg_tol;         // and relative residual
  int precision;         // CS_P_*: storage precision of G_off in the Euler kernels
  const float* gscale;   // FP8 row scales of G_off (NULL unless FP8)
};

// Per-solve device state, sized by (N, trials).
struct SolveDev {
  size_t x_bytes = 0;   // bytes of each of X0, X1
  int trials = 0, n_outer = 0, record_steps = 0, precision = -1, cap_trials = 0, cap_outer = 0,
      cap_record = 0, cap_prec = -1;
  double* R = nullptr;          // N x T (FP64), refit signal
  void* X0 = nullptr;           // Npad x round4(T) coupling operand (blocks of 64 trials), two buffers
  void* X1 = nullptr;
  void* state = nullptr;        // 3 x N x T amplitudes, feedback, injection constant (streamed kernel)
  uint8_t* sigma = nullptr;     // N x T support
  double* energy = nullptr;     // T
  int32_t* ssize = nullptr;     // n_outer x T support sizes
  int32_t* sidx = nullptr;      // T x N support index lists
  int32_t* lead = nullptr;      // T
  double* work = nullptr;       // refit workspace pool
  size_t work_stride = 0;       // doubles per pool block
  int work_blocks = 0;
  double* rec_c = nullptr;      // record_steps x N x T
  double* rec_e = nullptr;
  double* x_hat = nullptr;      // N, kept trial
  uint8_t* sigma_hat = nullptr; // N
  double* stats = nullptr;      // CS_STATS_LEN
  unsigned* bar = nullptr;      // Euler kernel: per-CTA X publication flags (kMaxEulerCtas + 1 words)
  int* err = nullptr;           // device error word
  int* singular = nullptr;      // set when a refit used the ridge
  double* err4 = nullptr;       // 4 doubles: scratch of the error against FP64 (launch_finish)
  uint8_t* sig_outer = nullptr; // record_outer: n_outer x N x T supports after each outer iteration
  double* R_outer = nullptr;    // and n_outer x N x T signals
  bool has_outer = false;       // the last solve recorded them
  double* e_hist = nullptr;     // best-configuration readout: (n_steps + 1) x CTAs x T energy partials
  uint8_t* s_hist = nullptr;    // and (n_steps + 1) x N x T configurations
  size_t cap_e_hist = 0, cap_s_hist = 0;
  RefitJob* job = nullptr;      // this problem's refit job (device copy)
  bool done = false;
  int plan_cluster = 0, plan_ctas = 0, plan_form = 0;  // work split of the last Euler launch
};

RefitJob make_job(const ProblemDev& P, const SolveDev& S);

// The stream a problem queues its work on, and its sizes (for the server, which
// runs a caller's problem on one of its own streams for the length of a request).
cudaStream_t problem_stream(const cs_problem* p);
void set_problem_stream(cs_problem* p, cudaStream_t s);
int64_t problem_N(const cs_problem* p);
int64_t problem_M(const cs_problem* p);

// One outer iteration of a batch of problems in one launch (batch.cu).
struct BatchLaunch {
  const void* insts;   // device array of per-problem descriptors (fill_batch_inst)
  const int* order;    // device array: processing order, largest first
  int n, T;            // problems of this launch and their (common) trial count
  const cs_params* prm;  // precision and tensor_form of the launch (common to its problems)
  int* queue;          // device work counter
  int outer;
  int* err;
  long long timeout_cycles;
  int ctas;            // CTAs to launch at most (one per SM)
  int cc = 1;          // CTAs per cluster (1, 2, 4 or 8)
  int n_large = 0;     // the first n_large problems (in processing order) are each run by a whole cluster
  int tps = 0;         // column tiles per ring slot (1, 2, 4; 0 = the launch's default)
  int slots = 0;       // ring slots (2..8; 0 = as many as fit)
  int step_cap = 0;    // > 0: at most this many Euler steps per run (tuning runs)
  int test_skip = 0;   // test hook (test_phantom_ctas > 0): each CTA's first ring copy is never issued
};
// Ring shape and cluster size of a batched launch (the batch autotuner's choice).
struct BatchShape {
  int cc = 1, tps = 0, slots = 0, span_rt = 0;  // span_rt: problems with at least this many row tiles span a cluster
};
// Persisted autotuner choices (tune_cache.cu): the device part of every key,
// lookup, store (memory and the cache file), and a count of timed tunings
// (timed = true) or choices taken from the file (timed = false).
std::string tune_device_tag(int device);
bool tune_lookup(const std::string& key, std::string* value);
void tune_store(const std::string& key, const std::string& value);
void tune_note(bool timed);
// cs_solve_batch with problem i drawing its initial amplitudes with instance
// number instances[i] (NULL: i), so that a problem's result does not depend on
// its place in the batch (the server's batches).
cs_status solve_batch(cs_problem* const* ps, const cs_params* const* prms, const int32_t* trials, int32_t n,
                      const int32_t* instances);
// Row tiles of a problem of N rows in the batched kernel's tiling.
int batch_row_tiles(int64_t N);
size_t batch_inst_bytes();
void fill_batch_inst(void* dst, const ProblemDev& P, const SolveDev& S, const cs_params& prm, double theta,
                     int inst);
// Tiled G_off of the batched kernel; frag = the batch_tc_kind of its launches.
cudaError_t launch_store_tiled(ProblemDev& P, int precision, int frag);
// Product form of a batch of this precision, trial count and tensor_form:
// 0 FMAs, 1 mma.sync tensor cores, 2 tcgen05 tensor cores (the last two for
// BF16 / FP16 storage and 8 or 16 trials: tensor_form 3 picks mma.sync, 1 the
// FMAs, 0, 2 and 4 tcgen05).
int batch_tc_kind(int precision, int trials, int tensor_form);
cudaError_t ensure_row_scales(ProblemDev& P);
size_t storage_bytes(int precision);
cudaError_t launch_euler_batch(const BatchLaunch& L, cudaStream_t st);

// Launchers (stream-ordered, no synchronisation).
cudaError_t launch_gram(const ProblemDev& P);
cudaError_t launch_store_coupling(ProblemDev& P, int precision);
// plan_only: choose (and cache) the plan, autotuning if asked, and build its
// streamed tiles, without launching; a later launch of the shape is then a pure
// stream operation (capturable into a CUDA graph).
cudaError_t launch_euler(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer,
                         double eta, long long timeout_cycles, bool plan_only = false);
const char* euler_last_call();  // the CUDA call the last failing Euler launch stopped at
cudaError_t launch_init_R(const RefitJob* jobs, int njobs, int T, int num_sms, cudaStream_t st);
// What the host knows of a single problem's refit, for launch_refit to pick
// the grid-wide damped Jacobi (few trials of one problem); NULL: one block per
// (problem, trial).
struct RefitPlan {
  int refit, jacobi_iters, N, num_sms;
  double* R;  // the problem's R (N x T)
};
cudaError_t launch_refit(const RefitJob* jobs, int njobs, int T, double* pool, size_t pool_stride, int pool_blocks,
                         int outer, cudaStream_t st, const RefitPlan* plan = nullptr, int* queue = nullptr);
// Whether launch_refit takes the grid-wide damped Jacobi (1 + jacobi_iters
// launches instead of 2).
bool refit_grid_wide(const RefitPlan* plan, int njobs, int T, int pool_blocks, size_t pool_stride);
// Objective per trial, kept trial, and the kept result's error against FP64
// (stats[11], stats[12]); err4 is 4 doubles of scratch per job.
cudaError_t launch_finish(const RefitJob* jobs, int njobs, int T, int num_sms, cudaStream_t st, double* err4);
// The LASSO initial R (refit.cu): argmin 1/2 x^T G x - h^z.x + lam1 ||x||_1 by
// `iters` FISTA iterations from 0 (step 1 / the largest absolute row sum of G),
// copied to every trial's column of R (N x T).  work: at least 4 N + 1 doubles.
cudaError_t launch_lasso(const double* G, const double* hz, int N, int T, double lam1, int iters, double* work,
                         double* R, int num_sms, cudaStream_t st);
// Best-configuration readout of one CIM run (euler.cu): per trial the first
// step n in 1 .. S whose summed energy (CTA partials in fixed order) is lowest;
// sigma (N x T) takes that step's configuration.
cudaError_t launch_readout(const double* e_hist, const uint8_t* s_hist, uint8_t* sigma, int N, int T, int S,
                           int ctas, cudaStream_t st);

}  // namespace cs
