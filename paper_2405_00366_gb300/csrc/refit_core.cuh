// Block-level building blocks of the refit (the classical half of Algorithm 1):
// support compaction, an FP64 Cholesky factorisation with a relative pivot
// test, and the triangular solves.  Every function is called by all threads of
// a block of kRefitThreads threads.
#pragma once

#include "common.cuh"

namespace cs {

constexpr int kRefitThreads = 256;

// Compacted support of trial t: idx[0..n) = {r : sigma[r][t] = 1} in
// increasing r.  Returns n in every thread.
__device__ __forceinline__ int support_list(const uint8_t* __restrict__ sigma, int N, int T, int t, int* idx) {
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

__device__ __forceinline__ bool cholesky_lower(double* W, int n, const double* diag) {
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
__device__ __forceinline__ void cholesky_solve_warp(const double* W, int n, double* b) {
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

}  // namespace cs
