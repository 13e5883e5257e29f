// Euler kernels and launcher for fp8 storage of G_off (compute type float).
#include "euler_impl.cuh"

namespace cs {

cudaError_t launch_euler_fp8(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles, bool plan_only) {
  return launch_typed<__nv_fp8_e4m3, float>(P, S, prm, outer, eta, timeout_cycles, plan_only);
}

}  // namespace cs
