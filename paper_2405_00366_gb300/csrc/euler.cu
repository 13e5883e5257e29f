// Dispatch of one CIM run (the persistent Euler kernel of euler_kernel.cuh,
// planned and launched by euler_impl.cuh) to
// the translation unit built for the storage precision of G_off.
#include "internal.h"

namespace cs {

thread_local const char* g_where = "";

cudaError_t launch_euler_fp64(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles);
cudaError_t launch_euler_fp32(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles);
cudaError_t launch_euler_bf16(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles);
cudaError_t launch_euler_fp16(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles);
cudaError_t launch_euler_fp8(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles);

const char* euler_last_call() { return g_where; }

cudaError_t launch_euler(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                         long long timeout_cycles) {
  switch (prm.precision) {
    case CS_P_FP64: return launch_euler_fp64(P, S, prm, outer, eta, timeout_cycles);
    case CS_P_FP32: return launch_euler_fp32(P, S, prm, outer, eta, timeout_cycles);
    case CS_P_BF16: return launch_euler_bf16(P, S, prm, outer, eta, timeout_cycles);
    case CS_P_FP16: return launch_euler_fp16(P, S, prm, outer, eta, timeout_cycles);
    case CS_P_FP8: return launch_euler_fp8(P, S, prm, outer, eta, timeout_cycles);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cs
