// Euler kernels and launcher for fp32 storage of G_off (compute type float).
#include "euler_impl.cuh"

namespace cs {

cudaError_t launch_euler_fp32(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles, bool plan_only) {
  return launch_typed<float, float>(P, S, prm, outer, eta, timeout_cycles, plan_only);
}

}  // namespace cs
