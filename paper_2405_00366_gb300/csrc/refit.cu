// The classical half of Algorithm 1 (the "CDP"): refit R on the support the
// CIM run produced, then, after the last outer iteration, the objective of
// Eq. doublel0 per trial and the kept trial.
//
// Exact refit: R_S solves the normal equations G_SS R_S = (A^T y)_S by an FP64
// Cholesky factorisation; off the support R_r is the Jacobi fixed point
// (h^z_r - sum_{r' in S} G_rr' R_r') / G_rr, so R is defined for every r (the
// local field of Eq. localfieldMFZ needs R_r' for every r').  A factorisation
// that meets a pivot not above 1e-12 times its diagonal entry (numerically
// singular G_SS, e.g. |S| > M) is redone on G_SS + eps I with
// eps = 1e-10 * mean(G_rr over S) and the solve is flagged.
#include "common.cuh"
#include "internal.h"

namespace cs {

namespace {

constexpr int kRefitThreads = 256;

// Compacted support of trial t: idx[0..n) = {r : sigma[r][t] = 1} in
// increasing r.  Returns n in every thread.
__device__ int support_list(const uint8_t* __restrict__ sigma, int N, int T, int t, int* idx) {
  __shared__ int warp_tot[kRefitThreads / 32];
  __shared__ int base_s;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  if (tid == 0) base_s = 0;
  __syncthreads();
  for (int c0 = 0; c0 < N; c0 += kRefitThreads) {
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
      for (int i = 0; i < kRefitThreads / 32; ++i) s += warp_tot[i];
      base_s += s;
    }
    __syncthreads();
  }
  return base_s;
}

// In-place Cholesky of the n x n matrix W (lower triangle, column-major:
// element (i, k) at W[k * n + i]), right-looking.  Returns false when a pivot
// is not above kPivotTol times the matrix's own diagonal entry (diag[j]) or is
// not finite: the matrix is then numerically singular.
constexpr double kPivotTol = 1e-12;

__device__ bool cholesky_lower(double* W, int n, const double* diag) {
  __shared__ int ok_s;
  const int tid = threadIdx.x;
  for (int j = 0; j < n; ++j) {
    double* colj = W + (size_t)j * n;
    if (tid == 0) {
      const double d = colj[j];
      ok_s = (d > kPivotTol * diag[j] && isfinite(d)) ? 1 : 0;
      if (ok_s) colj[j] = sqrt(d);
    }
    __syncthreads();
    if (!ok_s) return false;
    const double ljj = colj[j];
    for (int i = j + 1 + tid; i < n; i += kRefitThreads) colj[i] /= ljj;
    __syncthreads();
    for (int k = j + 1; k < n; ++k) {
      const double lkj = colj[k];
      double* colk = W + (size_t)k * n;
      for (int i = k + tid; i < n; i += kRefitThreads) colk[i] = fma(-colj[i], lkj, colk[i]);
    }
    __syncthreads();
  }
  return true;
}

// Solve L L^T x = b in place in b (length n) with one warp.
__device__ void cholesky_solve_warp(const double* W, int n, double* b) {
  const int l = threadIdx.x & 31;
  // forward: L z = b, column-oriented
  for (int k = 0; k < n; ++k) {
    const double* colk = W + (size_t)k * n;
    const double zk = b[k] / colk[k];
    __syncwarp();
    if (l == 0) b[k] = zk;
    for (int i = k + 1 + l; i < n; i += 32) b[i] = fma(-colk[i], zk, b[i]);
    __syncwarp();
  }
  // backward: L^T x = z, dot-product form over column k of L
  for (int k = n - 1; k >= 0; --k) {
    const double* colk = W + (size_t)k * n;
    double s = 0.0;
    for (int i = k + 1 + l; i < n; i += 32) s = fma(colk[i], b[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double xk = (b[k] - s) / colk[k];
    __syncwarp();
    if (l == 0) b[k] = xk;
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kRefitThreads) refit_exact_kernel(
    const double* __restrict__ G, const double* __restrict__ hz, const double* __restrict__ g,
    const uint8_t* __restrict__ sigma, double* __restrict__ R, int* __restrict__ sidx,
    double* __restrict__ work, size_t work_stride, int32_t* __restrict__ ssize, int N, int T, int outer,
    int* singular, int* err) {
  const int t = blockIdx.x;
  if (ld_volatile(err) != 0) return;
  int* idx = sidx + (size_t)t * N;
  const int n = support_list(sigma, N, T, t, idx);
  if (threadIdx.x == 0) ssize[(size_t)outer * T + t] = n;
  if (n == 0) {
    for (int r = threadIdx.x; r < N; r += kRefitThreads) R[(size_t)r * T + t] = hz[r] / g[r];
    return;
  }
  double* W = work + (size_t)t * work_stride;
  double* x = W + (size_t)n * n;
  double* dg = x + n;  // diagonal of the matrix being factorised
  __shared__ double ridge_s;
  if (threadIdx.x == 0) ridge_s = 0.0;
  __syncthreads();
  for (int attempt = 0; attempt < 2; ++attempt) {
    const double ridge = ridge_s;
    for (size_t e = threadIdx.x; e < (size_t)n * n; e += kRefitThreads) {
      const int k = (int)(e / n), i = (int)(e % n);
      if (i >= k) W[e] = G[(size_t)idx[i] * N + idx[k]] + (i == k ? ridge : 0.0);
    }
    for (int i = threadIdx.x; i < n; i += kRefitThreads) dg[i] = G[(size_t)idx[i] * N + idx[i]] + ridge;
    __syncthreads();
    if (cholesky_lower(W, n, dg)) break;
    if (attempt == 1) { if (threadIdx.x == 0) set_error(err, DEV_NONFINITE); return; }
    // ridge eps = 1e-10 * mean(g_S)
    __shared__ double red_s[kRefitThreads / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kRefitThreads) s += g[idx[i]];
    s = block_sum(s, red_s);
    if (threadIdx.x == 0) { ridge_s = 1e-10 * s / n; atomicExch(singular, 1); }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += kRefitThreads) x[i] = hz[idx[i]];
  __syncthreads();
  if (threadIdx.x < 32) cholesky_solve_warp(W, n, x);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kRefitThreads) R[(size_t)idx[i] * T + t] = x[i];
  // off the support: one warp per row r
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int r = w; r < N; r += kRefitThreads / 32) {
    if (sigma[(size_t)r * T + t]) continue;
    const double* Gr = G + (size_t)r * N;
    double s = 0.0;
    for (int i = l; i < n; i += 32) s = fma(Gr[idx[i]], x[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) R[(size_t)r * T + t] = (hz[r] - s) / g[r];
  }
}

// E_t = 1/2 ||y - A (sigma o R)||^2 + lambda |sigma| for trial t, in FP64 from A and y.
__global__ void __launch_bounds__(kRefitThreads) energy_kernel(
    const double* __restrict__ A, const double* __restrict__ y, const uint8_t* __restrict__ sigma,
    const double* __restrict__ R, int* __restrict__ sidx, double* __restrict__ energy, int M, int N, int T,
    double lambda) {
  const int t = blockIdx.x;
  int* idx = sidx + (size_t)t * N;
  const int n = support_list(sigma, N, T, t, idx);
  __shared__ double red_s[kRefitThreads / 32];
  double s = 0.0;
  for (int k = threadIdx.x; k < M; k += kRefitThreads) {
    const double* Ak = A + (size_t)k * N;
    double v = y[k];
    for (int i = 0; i < n; ++i) v = fma(-Ak[idx[i]], R[(size_t)idx[i] * T + t], v);
    s = fma(v, v, s);
  }
  s = block_sum(s, red_s);
  if (threadIdx.x == 0) energy[t] = 0.5 * s + lambda * n;
}

// Kept trial = argmin energy (ties to the lower index); x_hat, sigma_hat, stats.
__global__ void select_kernel(const double* __restrict__ energy, const uint8_t* __restrict__ sigma,
                              const double* __restrict__ R, double* __restrict__ x_hat,
                              uint8_t* __restrict__ sigma_hat, double* __restrict__ stats, int N, int M, int T,
                              const int* singular, const int* err) {
  __shared__ int best_s;
  __shared__ int count_s;
  if (threadIdx.x == 0) {
    int best = 0;
    for (int t = 1; t < T; ++t)
      if (energy[t] < energy[best]) best = t;
    best_s = best;
    count_s = 0;
  }
  __syncthreads();
  const int best = best_s;
  int cnt = 0;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const uint8_t s = sigma[(size_t)r * T + best];
    sigma_hat[r] = s;
    x_hat[r] = s ? R[(size_t)r * T + best] : 0.0;
    cnt += s;
  }
  atomicAdd(&count_s, cnt);
  __syncthreads();
  if (threadIdx.x == 0) {
    stats[0] = best;
    stats[1] = count_s;
    stats[2] = *singular ? 1.0 : 0.0;
    stats[3] = *err;
    stats[4] = T;
    stats[5] = N;
    stats[6] = M;
    stats[7] = energy[best];
  }
}

// Initial R of every trial: the Jacobi fixed point of the empty support, h^z / g.
__global__ void init_R_kernel(const double* __restrict__ hz, const double* __restrict__ g, double* __restrict__ R,
                              int N, int T) {
  const size_t total = (size_t)N * T;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < total; o += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(o / T);
    R[o] = hz[r] / g[r];
  }
}

}  // namespace

cudaError_t launch_init_R(const ProblemDev& P, SolveDev& S) {
  init_R_kernel<<<P.num_sms, 256, 0, P.stream>>>(P.hz, P.g, S.R, (int)P.N, S.trials);
  return cudaGetLastError();
}

cudaError_t launch_refit(const ProblemDev& P, SolveDev& S, const cs_params& prm, int outer) {
  (void)prm;
  const int N = (int)P.N, T = S.trials;
  const size_t stride = (size_t)N * N + 2 * (size_t)N;
  refit_exact_kernel<<<T, kRefitThreads, 0, P.stream>>>(P.G, P.hz, P.g, S.sigma, S.R, S.sidx, S.work, stride,
                                                        S.ssize, N, T, outer, S.singular, S.err);
  return cudaGetLastError();
}

cudaError_t launch_finish(const ProblemDev& P, SolveDev& S) {
  const int N = (int)P.N, M = (int)P.M, T = S.trials;
  energy_kernel<<<T, kRefitThreads, 0, P.stream>>>(P.A, P.y, S.sigma, S.R, S.sidx, S.energy, M, N, T, P.lambda);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  select_kernel<<<1, 256, 0, P.stream>>>(S.energy, S.sigma, S.R, S.x_hat, S.sigma_hat, S.stats, N, M, T,
                                         S.singular, S.err);
  return cudaGetLastError();
}

}  // namespace cs
