// The classical half of Algorithm 1 (the "CDP"): refit R on the support the
// CIM run produced, then, after the last outer iteration, the objective of
// Eq. doublel0 per trial and the kept trial.  Every kernel works on a table of
// jobs (one per problem), so a single solve and a batch of problems share them.
//
// Exact refit: R_S solves the normal equations G_SS R_S = (A^T y)_S by an FP64
// Cholesky factorisation; off the support R_r is the Jacobi fixed point
// (h^z_r - sum_{r' in S} G_rr' R_r') / G_rr, so R is defined for every r (the
// local field of Eq. localfieldMFZ needs R_r' for every r').  A factorisation
// that meets a pivot not above 1e-12 times its diagonal entry (numerically
// singular G_SS, e.g. |S| > M) is redone on G_SS + eps I with
// eps = 1e-10 * mean(G_rr over S) and the solve is flagged.
//
// The exact refit depends on the support only, so trials of a problem whose
// supports are identical share one factorisation: the first such trial (the
// "leader") is refitted and the others copy its R.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "refit_core.cuh"

namespace cs {

namespace {

// True (in every thread) when columns t and u of sigma (N x T) are equal.
__device__ bool same_support(const uint8_t* __restrict__ sigma, int N, int T, int t, int u) {
  int diff = 0;
  for (int r = threadIdx.x; r < N; r += kRefitThreads)
    diff |= (sigma[(size_t)r * T + t] != 0) != (sigma[(size_t)r * T + u] != 0);
  return __syncthreads_or(diff) == 0;
}

// Refit of trial t of job J with the workspace W (n^2 + 2n doubles, n = |S|).
__device__ void refit_one(const RefitJob& J, int t, const int* idx, int n, double* W) {
  const int N = J.N, T = J.T;
  if (n == 0) {
    for (int r = threadIdx.x; r < N; r += kRefitThreads) J.R[(size_t)r * T + t] = J.hz[r] / J.g[r];
    return;
  }
  double* x = W + (size_t)n * n;
  double* dg = x + n;  // diagonal of the matrix being factorised
  __shared__ double ridge_s;
  __shared__ double red_s[kRefitThreads / 32];
  if (threadIdx.x == 0) ridge_s = 0.0;
  __syncthreads();
  for (int attempt = 0; attempt < 2; ++attempt) {
    const double ridge = ridge_s;
    for (size_t e = threadIdx.x; e < (size_t)n * n; e += kRefitThreads) {
      const int k = (int)(e / n), i = (int)(e % n);
      if (i >= k) W[e] = J.G[(size_t)idx[i] * N + idx[k]] + (i == k ? ridge : 0.0);
    }
    for (int i = threadIdx.x; i < n; i += kRefitThreads) dg[i] = J.G[(size_t)idx[i] * N + idx[i]] + ridge;
    __syncthreads();
    if (cholesky_lower(W, n, dg)) break;
    if (attempt == 1) {
      if (threadIdx.x == 0) set_error(J.err, DEV_NONFINITE);
      return;
    }
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kRefitThreads) s += J.g[idx[i]];
    s = block_sum(s, red_s);
    if (threadIdx.x == 0) {
      ridge_s = 1e-10 * s / n;
      atomicExch(J.singular, 1);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += kRefitThreads) x[i] = J.hz[idx[i]];
  __syncthreads();
  if (threadIdx.x < 32) cholesky_solve_warp(W, n, x);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kRefitThreads) J.R[(size_t)idx[i] * T + t] = x[i];
  // off the support: one warp per row r
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int r = w; r < N; r += kRefitThreads / 32) {
    if (J.sigma[(size_t)r * T + t]) continue;
    const double* Gr = J.G + (size_t)r * N;
    double s = 0.0;
    for (int i = l; i < n; i += 32) s = fma(Gr[idx[i]], x[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) J.R[(size_t)r * T + t] = (J.hz[r] - s) / J.g[r];
  }
  __syncthreads();
}

// Refit of every (job, trial) item whose support is not a copy of an earlier
// trial's; items are spread over the grid, block b owns workspace b of the pool.
__global__ void __launch_bounds__(kRefitThreads) refit_kernel(const RefitJob* __restrict__ jobs, int T, int items,
                                                              double* __restrict__ pool, size_t pool_stride,
                                                              int outer) {
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const RefitJob& J = jobs[it / T];
    const int t = it % T;
    if (ld_volatile(J.err) != 0) continue;
    int* idx = J.sidx + (size_t)t * J.N;
    const int n = support_list(J.sigma, J.N, T, t, idx);
    int lead = t;
    for (int u = 0; u < t; ++u)
      if (same_support(J.sigma, J.N, T, t, u)) { lead = u; break; }
    if (threadIdx.x == 0) {
      J.ssize[(size_t)outer * T + t] = n;
      J.lead[t] = lead;
    }
    if (lead == t) refit_one(J, t, idx, n, pool + (size_t)blockIdx.x * pool_stride);
    __syncthreads();
  }
}

// Trials that share a leader's support take its R.
__global__ void follow_kernel(const RefitJob* __restrict__ jobs, int T, int items) {
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const RefitJob& J = jobs[it / T];
    const int t = it % T;
    const int lead = J.lead[t];
    if (lead == t || ld_volatile(J.err) != 0) continue;
    for (int r = threadIdx.x; r < J.N; r += blockDim.x) J.R[(size_t)r * T + t] = J.R[(size_t)r * T + lead];
  }
}

// E_t = 1/2 ||y - A (sigma o R)||^2 + lambda |sigma| per (job, trial), in FP64 from A and y.
__global__ void __launch_bounds__(kRefitThreads) energy_kernel(const RefitJob* __restrict__ jobs, int T, int items) {
  __shared__ double red_s[kRefitThreads / 32];
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const RefitJob& J = jobs[it / T];
    const int t = it % T;
    int* idx = J.sidx + (size_t)t * J.N;
    const int n = support_list(J.sigma, J.N, T, t, idx);
    double s = 0.0;
    for (int k = threadIdx.x; k < J.M; k += kRefitThreads) {
      const double* Ak = J.A + (size_t)k * J.N;
      double v = J.y[k];
      for (int i = 0; i < n; ++i) v = fma(-Ak[idx[i]], J.R[(size_t)idx[i] * T + t], v);
      s = fma(v, v, s);
    }
    s = block_sum(s, red_s);
    if (threadIdx.x == 0) J.energy[t] = 0.5 * s + J.lambda * n;
    __syncthreads();
  }
}

// Kept trial = argmin energy (ties to the lower index); x_hat, sigma_hat, stats.
__global__ void select_kernel(const RefitJob* __restrict__ jobs, int T) {
  const RefitJob& J = jobs[blockIdx.x];
  __shared__ int best_s;
  __shared__ int count_s;
  if (threadIdx.x == 0) {
    int best = 0;
    for (int t = 1; t < T; ++t)
      if (J.energy[t] < J.energy[best]) best = t;
    best_s = best;
    count_s = 0;
  }
  __syncthreads();
  const int best = best_s;
  int cnt = 0;
  for (int r = threadIdx.x; r < J.N; r += blockDim.x) {
    const uint8_t s = J.sigma[(size_t)r * T + best];
    J.sigma_hat[r] = s;
    J.x_hat[r] = s ? J.R[(size_t)r * T + best] : 0.0;
    cnt += s;
  }
  atomicAdd(&count_s, cnt);
  __syncthreads();
  if (threadIdx.x == 0) {
    J.stats[0] = best;
    J.stats[1] = count_s;
    J.stats[2] = *J.singular ? 1.0 : 0.0;
    J.stats[3] = *J.err;
    J.stats[4] = T;
    J.stats[5] = J.N;
    J.stats[6] = J.M;
    J.stats[7] = J.energy[best];
  }
}

// Initial R of every trial: the Jacobi fixed point of the empty support, h^z / g.
__global__ void init_R_kernel(const RefitJob* __restrict__ jobs, int T, int njobs) {
  for (int j = blockIdx.y; j < njobs; j += gridDim.y) {
    const RefitJob& J = jobs[j];
    const size_t total = (size_t)J.N * T;
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < total; o += (size_t)gridDim.x * blockDim.x) {
      const int r = (int)(o / T);
      J.R[o] = J.hz[r] / J.g[r];
    }
  }
}

}  // namespace

cudaError_t launch_init_R(const RefitJob* jobs, int njobs, int T, int num_sms, cudaStream_t st) {
  const int gy = std::min(njobs, 65535);
  const int gx = std::max(1, num_sms / gy);
  init_R_kernel<<<dim3(gx, gy), 256, 0, st>>>(jobs, T, njobs);
  return cudaGetLastError();
}

cudaError_t launch_refit(const RefitJob* jobs, int njobs, int T, double* pool, size_t pool_stride, int pool_blocks,
                         int outer, cudaStream_t st) {
  const int items = njobs * T;
  refit_kernel<<<std::min(items, pool_blocks), kRefitThreads, 0, st>>>(jobs, T, items, pool, pool_stride, outer);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  follow_kernel<<<std::min(items, 4096), 256, 0, st>>>(jobs, T, items);
  return cudaGetLastError();
}

cudaError_t launch_finish(const RefitJob* jobs, int njobs, int T, int num_sms, cudaStream_t st) {
  const int items = njobs * T;
  energy_kernel<<<std::min(items, 8 * num_sms), kRefitThreads, 0, st>>>(jobs, T, items);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  select_kernel<<<njobs, 256, 0, st>>>(jobs, T);
  return cudaGetLastError();
}

}  // namespace cs
