// cs_objective_static: the per-trial objective of the solver for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc, or any routine that allocates behind
// their back: code that runs while a stream is being captured into a CUDA
// graph, hosts that hand out all device memory from an arena of their own, and
// latency-critical loops where an allocation (or the synchronisation it may
// imply) is not allowed.  This entry point allocates nothing.  The caller
// passes every input and output in device memory; the one piece of scratch the
// kernel needs (the compacted support indices of every trial) lives in a fixed,
// file-scope device array that is part of the library image, so every GPU that
// loads the library holds it (1 MiB) until the process exits.
//
// Host code cannot use the array's name as a device address: on the host it
// names a stand-in.  The device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace cs {
namespace {

constexpr int64_t kStaticIdxEntries = 262144;  // N * trials support indices (1 MiB of int32)

static __device__ __align__(256) int32_t g_static_idx[kStaticIdxEntries];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
int32_t* g_static_ptr[kMaxDevices] = {};

constexpr int kObjThreads = 256;

// E_t = 1/2 ||y - A (sigma o R)||^2 + lambda |sigma| for trial t = blockIdx.x,
// in FP64 from A and y (Eq. doublel0).  The support of trial t is first
// compacted into idx[t*N ..), every entry written before it is read, so the
// scratch needs no clearing between calls.
__global__ void __launch_bounds__(kObjThreads) objective_static_kernel(
    const double* __restrict__ A, const double* __restrict__ y, const uint8_t* __restrict__ sigma,
    const double* __restrict__ R, int32_t* __restrict__ scratch, double* __restrict__ energy, int M, int N, int T,
    double lambda) {
  __shared__ int warp_tot[kObjThreads / 32];
  __shared__ int base_s;
  __shared__ double red_s[kObjThreads / 32];
  const int t = blockIdx.x, tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  int32_t* idx = scratch + (size_t)t * N;
  if (tid == 0) base_s = 0;
  __syncthreads();
  for (int c0 = 0; c0 < N; c0 += kObjThreads) {
    const int r = c0 + tid;
    const bool on = r < N && sigma[(size_t)r * T + t] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, on);
    if (l == 0) warp_tot[w] = __popc(m);
    __syncthreads();
    int off = base_s;
    for (int i = 0; i < w; ++i) off += warp_tot[i];
    if (on) idx[off + __popc(m & ((1u << l) - 1u))] = r;
    __syncthreads();
    if (tid == 0) {
      int s = 0;
      for (int i = 0; i < kObjThreads / 32; ++i) s += warp_tot[i];
      base_s += s;
    }
    __syncthreads();
  }
  const int n = base_s;
  double s = 0.0;
  for (int k = tid; k < M; k += kObjThreads) {
    const double* Ak = A + (size_t)k * N;
    double v = y[k];
    for (int i = 0; i < n; ++i) v = fma(-Ak[idx[i]], R[(size_t)idx[i] * T + t], v);
    s = fma(v, v, s);
  }
  s = block_sum(s, red_s);
  if (tid == 0) energy[t] = 0.5 * s + lambda * n;
}

cs_status static_fail(cs_status st, const std::string& msg) {
  set_last_error(msg);
  return st;
}

// Device address of g_static_idx on the current device (looked up once per device).
cs_status static_scratch(int32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_fail(CS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return static_fail(CS_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_idx);
    if (e != cudaSuccess || !p)
      return static_fail(CS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_static_ptr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_static_ptr[dev];
  return CS_OK;
}

}  // namespace
}  // namespace cs

extern "C" cs_status cs_objective_static(const double* A, const double* y, const uint8_t* sigma, const double* R,
                                         int64_t M, int64_t N, int32_t trials, double lambda, double* energy,
                                         void* stream) {
  using namespace cs;
  if (!A || !y || !sigma || !R || !energy) return static_fail(CS_EINVAL, "a pointer argument is NULL");
  if (M < 1 || N < 1 || trials < 1) return static_fail(CS_EINVAL, "M, N and trials must be >= 1");
  if (M > (1 << 20) || N > (1 << 20)) return static_fail(CS_EINVAL, "M or N too large");
  if (N * (int64_t)trials > kStaticIdxEntries)
    return static_fail(CS_EINVAL, "N * trials exceeds the static scratch of cs_objective_static (262144 entries)");
  if (!(lambda >= 0.0) || !(lambda < 1e300)) return static_fail(CS_EINVAL, "lambda must be finite and >= 0");
  int32_t* scratch = nullptr;
  cs_status st = static_scratch(&scratch);
  if (st != CS_OK) return st;
  objective_static_kernel<<<trials, kObjThreads, 0, (cudaStream_t)stream>>>(A, y, sigma, R, scratch, energy, (int)M,
                                                                            (int)N, trials, lambda);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(CS_ECUDA, std::string("objective launch: ") + cudaGetErrorString(e));
  return CS_OK;
}
