// Dispatch of one CIM run (the persistent Euler kernel of euler_kernel.cuh,
// planned and launched by euler_impl.cuh) to
// the translation unit built for the storage precision of G_off.
#include "internal.h"

namespace cs {

thread_local const char* g_where = "";

cudaError_t launch_euler_fp64(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles, bool plan_only);
cudaError_t launch_euler_fp32(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles, bool plan_only);
cudaError_t launch_euler_bf16(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles, bool plan_only);
cudaError_t launch_euler_fp16(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles, bool plan_only);
cudaError_t launch_euler_fp8(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles, bool plan_only);

const char* euler_last_call() { return g_where; }

cudaError_t launch_euler(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                         long long timeout_cycles, bool plan_only) {
  switch (prm.precision) {
    case CS_P_FP64: return launch_euler_fp64(P, S, prm, outer, eta, timeout_cycles, plan_only);
    case CS_P_FP32: return launch_euler_fp32(P, S, prm, outer, eta, timeout_cycles, plan_only);
    case CS_P_BF16: return launch_euler_bf16(P, S, prm, outer, eta, timeout_cycles, plan_only);
    case CS_P_FP16: return launch_euler_fp16(P, S, prm, outer, eta, timeout_cycles, plan_only);
    case CS_P_FP8: return launch_euler_fp8(P, S, prm, outer, eta, timeout_cycles, plan_only);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cs

namespace cs {
namespace {

// One block per trial: E(n) = sum over CTAs (fixed order) of the energy partials
// of step n, n = 1 .. S; the first n of lowest E wins and sigma takes its
// configuration.
__global__ void readout_kernel(const double* __restrict__ e_hist, const uint8_t* __restrict__ s_hist,
                               uint8_t* __restrict__ sigma, int N, int T, int S, int ctas) {
  const int t = blockIdx.x;
  __shared__ double s_e[256];
  __shared__ int s_n[256];
  double best = 0.0;
  int bn = -1;
  for (int n = 1 + threadIdx.x; n <= S; n += blockDim.x) {
    const double* e = e_hist + (size_t)n * ctas * T + t;
    double E = 0.0;
    for (int c = 0; c < ctas; ++c) E += e[(size_t)c * T];
    if (bn < 0 || E < best) {  // a thread's steps rise, so its first minimum is kept
      best = E;
      bn = n;
    }
  }
  s_e[threadIdx.x] = best;
  s_n[threadIdx.x] = bn;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)blockDim.x; ++i) {
      if (s_n[i] < 0) continue;
      if (bn < 0 || s_e[i] < best || (s_e[i] == best && s_n[i] < bn)) {
        best = s_e[i];
        bn = s_n[i];
      }
    }
    s_n[0] = bn;
  }
  __syncthreads();
  const int n = s_n[0];
  if (n < 1) return;
  for (int r = threadIdx.x; r < N; r += blockDim.x)
    sigma[(size_t)r * T + t] = s_hist[((size_t)n * N + r) * T + t];
}

}  // namespace

cudaError_t launch_readout(const double* e_hist, const uint8_t* s_hist, uint8_t* sigma, int N, int T, int S,
                           int ctas, cudaStream_t st) {
  readout_kernel<<<T, 256, 0, st>>>(e_hist, s_hist, sigma, N, T, S, ctas);
  return cudaGetLastError();
}

}  // namespace cs
