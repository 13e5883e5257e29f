// Euler kernels and launcher for fp64 storage of G_off (compute type double).
#include "euler_impl.cuh"

namespace cs {

cudaError_t launch_euler_fp64(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles, bool plan_only) {
  return launch_typed<double, double>(P, S, prm, outer, eta, timeout_cycles, plan_only);
}

}  // namespace cs
