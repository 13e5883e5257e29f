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

// Device buffers of one problem (all owned by the library).
struct ProblemDev {
  int64_t M = 0, N = 0, Npad = 0;  // Npad: N rounded up to a multiple of 8
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
  int* flag = nullptr;    // device word: nonzero if A or y had a non-finite value
  int64_t launches = 0;   // kernels launched by the last create + solve
};

// Per-solve device state, sized by (N, trials).
struct SolveDev {
  int trials = 0, n_outer = 0, record_steps = 0, precision = -1, cap_trials = 0, cap_outer = 0,
      cap_record = 0, cap_prec = -1;
  double* R = nullptr;          // N x T (FP64), refit signal
  void* X0 = nullptr;           // Npad x round4(T) coupling operand (blocks of 64 trials), two buffers
  void* X1 = nullptr;
  uint8_t* sigma = nullptr;     // N x T support
  double* energy = nullptr;     // T
  int32_t* ssize = nullptr;     // n_outer x T support sizes
  int32_t* sidx = nullptr;      // T x N support index lists
  double* work = nullptr;       // refit workspace, T x N x N doubles (lazily sized)
  size_t work_elems = 0;
  double* rec_c = nullptr;      // record_steps x N x T
  double* rec_e = nullptr;
  double* x_hat = nullptr;      // N, kept trial
  uint8_t* sigma_hat = nullptr; // N
  double* stats = nullptr;      // CS_STATS_LEN
  unsigned* bar = nullptr;      // grid barrier counter
  int* err = nullptr;           // device error word
  int* singular = nullptr;      // set when a refit used the ridge
  bool done = false;
  int plan_cluster = 0, plan_ctas = 0;  // work split of the last Euler launch
};

// Launchers (stream-ordered, no synchronisation).
cudaError_t launch_gram(const ProblemDev& P);
cudaError_t launch_store_coupling(ProblemDev& P, int precision);
cudaError_t launch_euler(const ProblemDev& P, SolveDev& S, const cs_params& prm, int outer,
                         double eta, long long timeout_cycles);
const char* euler_last_call();  // the CUDA call the last failing Euler launch stopped at
cudaError_t launch_init_R(const ProblemDev& P, SolveDev& S);
cudaError_t launch_refit(const ProblemDev& P, SolveDev& S, const cs_params& prm, int outer);
cudaError_t launch_finish(const ProblemDev& P, SolveDev& S);

}  // namespace cs
