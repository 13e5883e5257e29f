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
// The damped Jacobi refit of the paper (refit = CS_REFIT_JACOBI) is the other
// option: a fixed number of relaxed sweeps from the trial's current R.
//
// The exact refit depends on the support only, so trials of a problem whose
// supports are identical share one factorisation: the first such trial (the
// "leader") is refitted and the others copy its R.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "kernels_common.cuh"
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

constexpr size_t kBlockedSmem = (32 * 33 + 2 * 64 * 33) * sizeof(float);  // solve_mixed_blocked's tiles

__device__ __forceinline__ size_t packed_off(int k, int n) { return (size_t)k * n - (size_t)k * (k - 1) / 2; }

__device__ __forceinline__ double block_max(double v, double* scratch) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  double m = 0.0;
  for (int i = 0; i < kRefitThreads / 32; ++i) m = fmax(m, scratch[i]);
  return m;
}

// Mixed-precision solve of G_SS x = (A^T y)_S: FP32 Cholesky of G_SS held packed
// (lower triangle, column-major) in shared memory, then FP64 iterative
// refinement: r = h^z_S - G_SS x in FP64 from the FP64 G, d = (L L^T)^-1 r in
// FP32, x += d, until the residual stops shrinking.  Returns false (in every
// thread) when a pivot is not above 1e-5 G_jj, i.e. the matrix is too close to
// singular for an FP32 factor, or when the residual does not fall below
// 1e-12 |h^z_S|; the caller then takes the FP64 factorisation.  x and r are
// global FP64 vectors of length n; Lp and d live in shared memory.
__device__ bool solve_mixed(const RefitJob& J, const int* idx, int n, float* Lp, float* d, double* x, double* r) {
  const int N = J.N, tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  constexpr int nw = kRefitThreads / 32;
  __shared__ int ok_s;
  __shared__ double red_s[kRefitThreads / 32];
  for (int k = w; k < n; k += nw) {
    const double* Gk = J.G + (size_t)idx[k] * N;
    float* ck = Lp + packed_off(k, n);
    for (int i = k + l; i < n; i += 32) ck[i - k] = (float)Gk[idx[i]];
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    float* cj = Lp + packed_off(j, n);
    if (tid == 0) {
      const float dj = cj[0];
      ok_s = (dj > 1e-5f * (float)J.g[idx[j]] && isfinite(dj)) ? 1 : 0;
      if (ok_s) cj[0] = sqrtf(dj);
    }
    __syncthreads();
    if (!ok_s) return false;
    const float ljj = cj[0];
    for (int i = j + 1 + tid; i < n; i += kRefitThreads) cj[i - j] /= ljj;
    __syncthreads();
    for (int k = j + 1 + w; k < n; k += nw) {
      const float lkj = cj[k - j];
      float* ck = Lp + packed_off(k, n);
      for (int i = k + l; i < n; i += 32) ck[i - k] = fmaf(-cj[i - j], lkj, ck[i - k]);
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += kRefitThreads) {
    x[i] = 0.0;
    r[i] = J.hz[idx[i]];
  }
  double rn0 = 0.0;
  for (int i = tid; i < n; i += kRefitThreads) rn0 = fmax(rn0, fabs(J.hz[idx[i]]));
  rn0 = block_max(rn0, red_s);
  if (rn0 == 0.0) return true;
  double prev = rn0;
  for (int it = 0; it < 8; ++it) {
    if (w == 0) {
      for (int i = l; i < n; i += 32) d[i] = (float)r[i];
      __syncwarp();
      for (int k = 0; k < n; ++k) {  // L z = d
        const float* ck = Lp + packed_off(k, n);
        const float zk = d[k] / ck[0];
        __syncwarp();
        if (l == 0) d[k] = zk;
        for (int i = k + 1 + l; i < n; i += 32) d[i] = fmaf(-ck[i - k], zk, d[i]);
        __syncwarp();
      }
      for (int k = n - 1; k >= 0; --k) {  // L^T d = z
        const float* ck = Lp + packed_off(k, n);
        float s = 0.f;
        for (int i = k + 1 + l; i < n; i += 32) s = fmaf(ck[i - k], d[i], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float xk = (d[k] - s) / ck[0];
        __syncwarp();
        if (l == 0) d[k] = xk;
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = tid; i < n; i += kRefitThreads) x[i] += (double)d[i];
    __syncthreads();
    for (int i = w; i < n; i += nw) {
      const double* Gi = J.G + (size_t)idx[i] * N;
      double s = 0.0;
      for (int k = l; k < n; k += 32) s = fma(Gi[idx[k]], x[k], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (l == 0) r[i] = J.hz[idx[i]] - s;
    }
    __syncthreads();
    double rm = 0.0;
    for (int i = tid; i < n; i += kRefitThreads) rm = fmax(rm, fabs(r[i]));
    rm = block_max(rm, red_s);
    if (rm <= 1e-14 * rn0 || (it >= 1 && rm > 0.5 * prev)) return rm <= 1e-12 * rn0;
    prev = rm;
  }
  return prev <= 1e-12 * rn0;
}

// Blocked form of solve_mixed for supports whose packed factor does not fit in
// shared memory: the FP32 copy of G_SS lives in this block's global workspace
// (column-major, lower triangle), factorised right-looking in panels of 32
// columns (the diagonal block by one warp in shared memory, the panel below it
// by one thread per row, the trailing update in 64 x 64 tiles staged through
// shared memory), then FP32 triangular solves by blocks of 32 and the same FP64
// refinement and acceptance as solve_mixed.  W holds x and r (FP64, n each),
// then L (n x n FP32) and d (n FP32); `sm` needs 21 KB.
__device__ bool solve_mixed_blocked(const RefitJob& J, const int* idx, int n, double* W, float* sm) {
  constexpr int NB = 32, TB = 64, LD = NB + 1;
  constexpr int nw = kRefitThreads / 32;
  const int N = J.N, tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  double* x = W;
  double* r = W + n;
  float* L = reinterpret_cast<float*>(W + 2 * (size_t)n);
  float* d = L + (size_t)n * n;
  float* D = sm;                // NB x LD: diagonal block
  float* Ti = sm + NB * LD;     // TB x LD: rows of the panel for one tile row
  float* Tk = Ti + TB * LD;     // TB x LD: rows of the panel for one tile column
  __shared__ int ok_s;
  __shared__ double red_s[kRefitThreads / 32];
  for (int k = w; k < n; k += nw) {
    const double* Gk = J.G + (size_t)idx[k] * N;
    for (int i = k + l; i < n; i += 32) L[i + (size_t)k * n] = (float)Gk[idx[i]];
  }
  __syncthreads();
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int b = min(NB, n - j0);
    for (int e = tid; e < b * b; e += kRefitThreads) {
      const int c = e / b, i = e % b;
      if (i >= c) D[i * LD + c] = L[(j0 + i) + (size_t)(j0 + c) * n];
    }
    __syncthreads();
    if (w == 0) {  // unblocked Cholesky of the diagonal block, lane = row
      int ok = 1;
      for (int c = 0; c < b && ok; ++c) {
        const float dc = D[c * LD + c];
        ok = (dc > 1e-5f * (float)J.g[idx[j0 + c]] && isfinite(dc)) ? 1 : 0;
        if (!ok) break;
        const float sc = sqrtf(dc);
        __syncwarp();
        if (l == c) D[c * LD + c] = sc;
        if (l > c && l < b) D[l * LD + c] /= sc;
        __syncwarp();
        for (int c2 = c + 1; c2 < b; ++c2)
          if (l >= c2 && l < b) D[l * LD + c2] = fmaf(-D[l * LD + c], D[c2 * LD + c], D[l * LD + c2]);
        __syncwarp();
      }
      if (l == 0) ok_s = ok;
    }
    __syncthreads();
    if (!ok_s) return false;
    for (int e = tid; e < b * b; e += kRefitThreads) {
      const int c = e / b, i = e % b;
      if (i >= c) L[(j0 + i) + (size_t)(j0 + c) * n] = D[i * LD + c];
    }
    // panel below the diagonal block: row i solves v L11^T = A[i, j0 : j0 + b]
    for (int i = j0 + b + tid; i < n; i += kRefitThreads) {
      float v[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) v[c] = c < b ? L[i + (size_t)(j0 + c) * n] : 0.f;
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        if (c < b) {
          float s = v[c];
#pragma unroll
          for (int c2 = 0; c2 < c; ++c2) s = fmaf(-v[c2], D[c * LD + c2], s);
          v[c] = s / D[c * LD + c];
        }
      }
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c < b) L[i + (size_t)(j0 + c) * n] = v[c];
    }
    __syncthreads();
    // trailing update A22 -= L21 L21^T (lower tiles), rows and columns from j1
    const int j1 = j0 + b, m = n - j1, nt = (m + TB - 1) / TB;
    const int tr = (tid & 15) * 4, tc = (tid >> 4) * 4;
    for (int ti = 0; ti < nt; ++ti) {
      for (int tk = 0; tk <= ti; ++tk) {
        const int ri0 = j1 + ti * TB, rk0 = j1 + tk * TB;
        for (int e = tid; e < TB * NB; e += kRefitThreads) {
          const int c = e / TB, rr = e % TB;
          Ti[rr * LD + c] = (c < b && ri0 + rr < n) ? L[(ri0 + rr) + (size_t)(j0 + c) * n] : 0.f;
          Tk[rr * LD + c] = (c < b && rk0 + rr < n) ? L[(rk0 + rr) + (size_t)(j0 + c) * n] : 0.f;
        }
        __syncthreads();
        float acc[4][4] = {};
        for (int c = 0; c < b; ++c) {
          float a4[4], b4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            a4[q] = Ti[(tr + q) * LD + c];
            b4[q] = Tk[(tc + q) * LD + c];
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int q2 = 0; q2 < 4; ++q2) acc[q][q2] = fmaf(a4[q], b4[q2], acc[q][q2]);
        }
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
          const int col = rk0 + tc + q2;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int row = ri0 + tr + q;
            if (row < n && col < n && row >= col) L[row + (size_t)col * n] -= acc[q][q2];
          }
        }
        __syncthreads();
      }
    }
  }
  // FP64 refinement with FP32 solves L L^T d = r
  for (int i = tid; i < n; i += kRefitThreads) {
    x[i] = 0.0;
    r[i] = J.hz[idx[i]];
  }
  double rn0 = 0.0;
  for (int i = tid; i < n; i += kRefitThreads) rn0 = fmax(rn0, fabs(J.hz[idx[i]]));
  rn0 = block_max(rn0, red_s);
  if (rn0 == 0.0) return true;
  double prev = rn0;
  for (int it = 0; it < 8; ++it) {
    for (int i = tid; i < n; i += kRefitThreads) d[i] = (float)r[i];
    __syncthreads();
    for (int j0 = 0; j0 < n; j0 += NB) {  // L z = d
      const int b = min(NB, n - j0);
      if (w == 0) {
        float zi = l < b ? d[j0 + l] : 0.f;
        for (int c = 0; c < b; ++c) {
          const float zc = __shfl_sync(0xffffffffu, zi, c) / L[(j0 + c) + (size_t)(j0 + c) * n];
          if (l == c) zi = zc;
          if (l > c && l < b) zi = fmaf(-L[(j0 + l) + (size_t)(j0 + c) * n], zc, zi);
        }
        if (l < b) d[j0 + l] = zi;
      }
      __syncthreads();
      for (int i = j0 + b + tid; i < n; i += kRefitThreads) {
        float s = d[i];
        for (int c = 0; c < b; ++c) s = fmaf(-L[i + (size_t)(j0 + c) * n], d[j0 + c], s);
        d[i] = s;
      }
      __syncthreads();
    }
    for (int j0 = ((n - 1) / NB) * NB; j0 >= 0; j0 -= NB) {  // L^T d = z
      const int b = min(NB, n - j0);
      if (w == 0) {
        float xi = l < b ? d[j0 + l] : 0.f;
        for (int c = b - 1; c >= 0; --c) {
          const float xc = __shfl_sync(0xffffffffu, xi, c) / L[(j0 + c) + (size_t)(j0 + c) * n];
          if (l == c) xi = xc;
          if (l < c) xi = fmaf(-L[(j0 + c) + (size_t)(j0 + l) * n], xc, xi);
        }
        if (l < b) d[j0 + l] = xi;
      }
      __syncthreads();
      for (int i = tid; i < j0; i += kRefitThreads) {
        float s = d[i];
        const float* Li = L + (size_t)i * n + j0;  // row block j0 of column i
        for (int c = 0; c < b; ++c) s = fmaf(-Li[c], d[j0 + c], s);
        d[i] = s;
      }
      __syncthreads();
    }
    for (int i = tid; i < n; i += kRefitThreads) x[i] += (double)d[i];
    __syncthreads();
    for (int i = w; i < n; i += nw) {
      const double* Gi = J.G + (size_t)idx[i] * N;
      double s = 0.0;
      for (int k = l; k < n; k += 32) s = fma(Gi[idx[k]], x[k], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (l == 0) r[i] = J.hz[idx[i]] - s;
    }
    __syncthreads();
    double rm = 0.0;
    for (int i = tid; i < n; i += kRefitThreads) rm = fmax(rm, fabs(r[i]));
    rm = block_max(rm, red_s);
    if (rm <= 1e-14 * rn0 || (it >= 1 && rm > 0.5 * prev)) return rm <= 1e-12 * rn0;
    prev = rm;
  }
  return prev <= 1e-12 * rn0;
}

// Refit of trial t of job J.  W is this block's global workspace (n^2 + 4n
// doubles); `smem` (smem_bytes) holds the FP32 factor of the mixed-precision
// path, taken when it fits and succeeds; otherwise the FP64 factorisation.
__device__ void refit_one(const RefitJob& J, int t, const int* idx, int n, double* W, float* smem,
                          size_t smem_bytes) {
  const int N = J.N, T = J.T;
  if (n == 0) {
    for (int r = threadIdx.x; r < N; r += kRefitThreads) J.R[(size_t)r * T + t] = J.hz[r] / J.g[r];
    return;
  }
  double* x;
  const size_t packed = (size_t)n * (n + 1) / 2;
  bool done = false;
  // a support larger than M makes G_SS singular: straight to the FP64 ridge path
  if (n <= J.M && (packed + (size_t)n) * sizeof(float) <= smem_bytes) {
    x = W;
    done = solve_mixed(J, idx, n, smem, smem + packed, W, W + n);
  } else if (n <= J.M && smem_bytes >= kBlockedSmem) {
    x = W;
    done = solve_mixed_blocked(J, idx, n, W, smem);
  }
  if (!done) {
    x = W + (size_t)n * n;
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
  }
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

// Damped Jacobi CDP of trial t (the paper's iteration for random data), warm
// started from the trial's current R: each sweep forms, for every r,
// R~_r = (h^z_r - sum_{r' in S, r' != r} G_rr' R_r') / G_rr from a snapshot of
// R_S (xs, n doubles) and moves R_r by jacobi_dt (R~_r - R_r).  One warp per row.
__device__ void jacobi_one(const RefitJob& J, int t, const int* idx, int n, double* xs) {
  const int N = J.N, T = J.T, w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int sweep = 0; sweep < J.jacobi_iters; ++sweep) {
    for (int i = threadIdx.x; i < n; i += kRefitThreads) xs[i] = J.R[(size_t)idx[i] * T + t];
    __syncthreads();
    for (int r = w; r < N; r += kRefitThreads / 32) {
      const double* Gr = J.G + (size_t)r * N;
      double s = 0.0;
      for (int i = l; i < n; i += 32) {
        const int c = idx[i];
        if (c != r) s = fma(Gr[c], xs[i], s);
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (l == 0) {
        double* Rr = J.R + (size_t)r * T + t;
        const double Rt = (J.hz[r] - s) / J.g[r];
        *Rr = *Rr + J.jacobi_dt * (Rt - *Rr);
      }
    }
    __syncthreads();
  }
}

// Conjugate-gradient CDP of trial t (the paper's iteration for MRI data) in
// FP64: G_SS is gathered once into W (row-major, n x n); from x = R_S of the
// trial, r = h^z_S - G_SS x, p = r, and for at most cg_iters iterations, until
// ||r|| <= cg_tol ||h^z_S||: q = G_SS p (one warp per row), alpha = r.r / p.q,
// x += alpha p, r -= alpha q, beta = r'.r' / r.r, p = r + beta p.  Dot products
// are fixed-order block sums, so the iteration is deterministic.  Then R_S = x
// and off the support the Jacobi fixed point, as for the exact refit.
__device__ void cg_one(const RefitJob& J, int t, const int* idx, int n, double* W) {
  const int N = J.N, T = J.T, w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __shared__ double red_s[kRefitThreads / 32];
  if (n == 0) {
    for (int r = threadIdx.x; r < N; r += kRefitThreads) J.R[(size_t)r * T + t] = J.hz[r] / J.g[r];
    __syncthreads();
    return;
  }
  double* Gs = W;
  double* x = W + (size_t)n * n;
  double* rv = x + n;
  double* pv = rv + n;
  double* qv = pv + n;
  for (size_t e = threadIdx.x; e < (size_t)n * n; e += kRefitThreads) {
    const int i = (int)(e / n), k = (int)(e % n);
    Gs[e] = J.G[(size_t)idx[i] * N + idx[k]];
  }
  for (int i = threadIdx.x; i < n; i += kRefitThreads) x[i] = J.R[(size_t)idx[i] * T + t];
  __syncthreads();
  // q = G_SS v, one warp per row, lanes over the columns, shuffle sum
  auto matvec = [&](const double* v, double* q) {
    for (int i = w; i < n; i += kRefitThreads / 32) {
      const double* Gi = Gs + (size_t)i * n;
      double s = 0.0;
      for (int k = l; k < n; k += 32) s = fma(Gi[k], v[k], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (l == 0) q[i] = s;
    }
    __syncthreads();
  };
  auto dot = [&](const double* a, const double* b) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kRefitThreads) s = fma(a[i], b[i], s);
    return block_sum(s, red_s);
  };
  matvec(x, qv);
  double bb = 0.0;
  for (int i = threadIdx.x; i < n; i += kRefitThreads) {
    const double b = J.hz[idx[i]];
    rv[i] = b - qv[i];
    pv[i] = rv[i];
    bb = fma(b, b, bb);
  }
  const double bnorm = sqrt(block_sum(bb, red_s));
  double rr = dot(rv, rv);
  for (int it = 0; it < J.cg_iters; ++it) {
    if (!(sqrt(rr) > J.cg_tol * bnorm)) break;
    matvec(pv, qv);
    const double alpha = rr / dot(pv, qv);
    for (int i = threadIdx.x; i < n; i += kRefitThreads) {
      x[i] = fma(alpha, pv[i], x[i]);
      rv[i] = fma(-alpha, qv[i], rv[i]);
    }
    __syncthreads();
    const double rr_new = dot(rv, rv);
    const double beta = rr_new / rr;
    for (int i = threadIdx.x; i < n; i += kRefitThreads) pv[i] = fma(beta, pv[i], rv[i]);
    __syncthreads();
    rr = rr_new;
  }
  for (int i = threadIdx.x; i < n; i += kRefitThreads) J.R[(size_t)idx[i] * T + t] = x[i];
  // off the support: one warp per row r
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
// trial's; block b owns workspace b of the pool.  Items go to the blocks in
// order, each block taking the next one when it is done with its last (a
// device counter, `queue`, zero at launch), so the expensive items of the
// large problems (listed first by the batched solve) do not pile up on a few
// blocks; queue = NULL spreads them round-robin instead.
__global__ void __launch_bounds__(kRefitThreads) refit_kernel(const RefitJob* __restrict__ jobs, int T, int items,
                                                              double* __restrict__ pool, size_t pool_stride,
                                                              int outer, size_t smem_bytes, int* queue) {
  extern __shared__ __align__(16) float refit_smem[];
  __shared__ int s_item;
  for (int it = blockIdx.x;;) {
    if (queue) {
      __syncthreads();
      if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
      __syncthreads();
      it = s_item;
    }
    if (it >= items) break;
    const int it_cur = it;
    if (!queue) it += gridDim.x;
    const RefitJob& J = jobs[it_cur / T];
    const int t = it_cur % T;
    if (ld_volatile(J.err) != 0) continue;
    int* idx = J.sidx + (size_t)t * J.N;
    const int n = support_list(J.sigma, J.N, T, t, idx);
    if (J.refit == CS_REFIT_JACOBI) {  // depends on the trial's own R: no sharing
      if (threadIdx.x == 0) {
        J.ssize[(size_t)outer * T + t] = n;
        J.lead[t] = t;
      }
      double* xs = (size_t)n * sizeof(double) <= smem_bytes ? reinterpret_cast<double*>(refit_smem)
                                                             : pool + (size_t)blockIdx.x * pool_stride;
      jacobi_one(J, t, idx, n, xs);
      __syncthreads();
      continue;
    }
    if (J.refit == CS_REFIT_CG) {  // warm started from the trial's own R: no sharing
      if (threadIdx.x == 0) {
        J.ssize[(size_t)outer * T + t] = n;
        J.lead[t] = t;
      }
      cg_one(J, t, idx, n, pool + (size_t)blockIdx.x * pool_stride);
      continue;
    }
    int lead = t;
    for (int u = 0; u < t; ++u)
      if (same_support(J.sigma, J.N, T, t, u)) { lead = u; break; }
    if (threadIdx.x == 0) {
      J.ssize[(size_t)outer * T + t] = n;
      J.lead[t] = lead;
    }
    if (lead == t) refit_one(J, t, idx, n, pool + (size_t)blockIdx.x * pool_stride, refit_smem, smem_bytes);
    __syncthreads();
  }
}

// Support lists of every trial for the grid-wide damped Jacobi refit (one
// block per trial): sidx, the support size of this outer iteration, no leader.
__global__ void __launch_bounds__(kRefitThreads) support_kernel(const RefitJob* __restrict__ jobs, int T, int outer) {
  const RefitJob& J = jobs[0];
  const int t = blockIdx.x;
  const int n = support_list(J.sigma, J.N, T, t, J.sidx + (size_t)t * J.N);
  if (threadIdx.x == 0) {
    J.ssize[(size_t)outer * T + t] = n;
    J.lead[t] = t;
  }
}

// One damped Jacobi sweep of every trial of one problem over the whole grid:
// Rb_r = Ra_r + jacobi_dt (R~_r - Ra_r), R~_r = (h^z_r - sum_{r' in S, r' != r}
// G_rr' Ra_r') / G_rr, one warp per (row, trial), the same arithmetic and
// summation order as jacobi_one.  Ra and Rb are N x T ([r][t]).
__global__ void jacobi_sweep_kernel(const RefitJob* __restrict__ jobs, int T, int outer, const double* __restrict__ Ra,
                                    double* __restrict__ Rb) {
  const RefitJob& J = jobs[0];
  const int t = blockIdx.y;
  const int n = J.ssize[(size_t)outer * T + t];
  const int* idx = J.sidx + (size_t)t * J.N;
  const int l = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < J.N; r += gridDim.x * wpb) {
    const double* Gr = J.G + (size_t)r * J.N;
    double s = 0.0;
    for (int i = l; i < n; i += 32) {
      const int c = idx[i];
      if (c != r) s = fma(Gr[c], Ra[(size_t)c * T + t], s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) {
      const double Rr = Ra[(size_t)r * T + t];
      const double Rt = (J.hz[r] - s) / J.g[r];
      Rb[(size_t)r * T + t] = Rr + J.jacobi_dt * (Rt - Rr);
    }
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

// G_rk rounded to the storage precision the Euler kernels used for G_off (with
// the row's scale for FP8), widened back to FP64.
__device__ __forceinline__ double stored_value(double v, int precision, const float* gscale, int r) {
  switch (precision) {
    case CS_P_FP32: return (double)to_storage<float>(v);
    case CS_P_BF16: return (double)__bfloat162float(to_storage<__nv_bfloat16>(v));
    case CS_P_FP16: return (double)__half2float(to_storage<__half>(v));
    case CS_P_FP8: {
      const double sc = (double)gscale[r];
      return sc > 0.0 ? (double)float(to_storage<__nv_fp8_e4m3>(v / sc)) * sc : 0.0;
    }
    default: return v;
  }
}

__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

// Error of the kept result against FP64, per problem (after select_kernel):
//  err[0] = max_r |U^s_r - U_r|, err[1] = max_r |U_r|  with U = G_off x_hat in
//           FP64 and U^s the same product with G_off rounded to its storage
//           precision (the coupling the Euler kernels used); U^s - U is summed
//           directly as sum_k (G^s_rk - G_rk) x_k (exactly zero for FP64);
//  err[2] = max over the support of |h^z_r - (G x_hat)_r|, err[3] = max over the
//           support of |h^z_r|: the FP64 residual of the refit's normal equations.
// One warp per row, FP64 throughout; maxima are order independent.
__global__ void error_kernel(const RefitJob* __restrict__ jobs, double* __restrict__ err4) {
  const RefitJob& J = jobs[blockIdx.y];
  double* e = err4 + 4 * (size_t)blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < J.N; r += gridDim.x * wpb) {
    const double* Gr = J.G + (size_t)r * J.N;
    double u = 0.0, du = 0.0, gx = 0.0;
    for (int k = lane; k < J.N; k += 32) {
      const double xk = J.x_hat[k];
      if (xk == 0.0) continue;
      const double v = Gr[k];
      gx += v * xk;
      if (k != r) {
        u += v * xk;
        du += (stored_value(v, J.precision, J.gscale, r) - v) * xk;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      u += __shfl_xor_sync(0xffffffffu, u, o);
      du += __shfl_xor_sync(0xffffffffu, du, o);
      gx += __shfl_xor_sync(0xffffffffu, gx, o);
    }
    if (lane == 0) {
      atomic_max_nonneg(e + 0, fabs(du));
      atomic_max_nonneg(e + 1, fabs(u));
      if (J.sigma_hat[r]) {
        atomic_max_nonneg(e + 2, fabs(J.hz[r] - gx));
        atomic_max_nonneg(e + 3, fabs(J.hz[r]));
      }
    }
  }
}

// stats[11] = err[0] / err[1] (0 when U = 0), stats[12] = err[2] / err[3].
__global__ void error_stats_kernel(const RefitJob* __restrict__ jobs, const double* __restrict__ err4, int njobs) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < njobs; j += gridDim.x * blockDim.x) {
    const double* e = err4 + 4 * (size_t)j;
    jobs[j].stats[11] = e[1] > 0.0 ? e[0] / e[1] : 0.0;
    jobs[j].stats[12] = e[3] > 0.0 ? e[2] / e[3] : 0.0;
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

// Largest absolute row sum of G (N x N, FP64) into *L: one warp per row,
// the maximum by an order-independent atomic (L zeroed beforehand).
__global__ void row_abs_max_kernel(const double* __restrict__ G, int N, double* L) {
  const int l = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < N; r += gridDim.x * wpb) {
    const double* Gr = G + (size_t)r * N;
    double s = 0.0;
    for (int k = l; k < N; k += 32) s += fabs(Gr[k]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) atomic_max_nonneg(L, s);
  }
}

// q = G z - h^z, one warp per row (fixed summation order).
__global__ void fista_grad_kernel(const double* __restrict__ G, const double* __restrict__ hz,
                                  const double* __restrict__ z, double* __restrict__ q, int N) {
  const int l = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < N; r += gridDim.x * wpb) {
    const double* Gr = G + (size_t)r * N;
    double s = 0.0;
    for (int k = l; k < N; k += 32) s = fma(Gr[k], z[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) q[r] = s - hz[r];
  }
}

// xn = soft(z - q / L, lam1 / L); z = xn + c (xn - x)   (c = (t_k - 1) / t_{k+1}).
__global__ void fista_step_kernel(const double* __restrict__ x, double* __restrict__ xn, double* __restrict__ z,
                                  const double* __restrict__ q, const double* __restrict__ L, double lam1, double c,
                                  int N) {
  const double Lv = *L;
  const double thr = lam1 / Lv;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < N; r += gridDim.x * blockDim.x) {
    const double v = z[r] - q[r] / Lv;
    const double a = fabs(v) - thr;
    const double xr = a > 0.0 ? copysign(a, v) : 0.0;
    xn[r] = xr;
    z[r] = xr + c * (xr - x[r]);
  }
}

// R[r][t] = x[r] for every trial.
__global__ void broadcast_R_kernel(const double* __restrict__ x, double* __restrict__ R, int N, int T) {
  const size_t total = (size_t)N * T;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < total; o += (size_t)gridDim.x * blockDim.x)
    R[o] = x[o / T];
}

}  // namespace

cudaError_t launch_lasso(const double* G, const double* hz, int N, int T, double lam1, int iters, double* work,
                         double* R, int num_sms, cudaStream_t st) {
  double* xa = work;
  double* xb = work + N;
  double* z = work + 2 * (size_t)N;
  double* q = work + 3 * (size_t)N;
  double* L = work + 4 * (size_t)N;
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(double) * (4 * (size_t)N + 1), st);
  if (e != cudaSuccess) return e;
  const int rows_grid = std::max(1, std::min((N + 7) / 8, 8 * num_sms));
  row_abs_max_kernel<<<rows_grid, 256, 0, st>>>(G, N, L);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int vec_grid = std::max(1, std::min((N + 255) / 256, 4 * num_sms));
  double t = 1.0;
  for (int k = 0; k < iters; ++k) {
    const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
    fista_grad_kernel<<<rows_grid, 256, 0, st>>>(G, hz, z, q, N);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    fista_step_kernel<<<vec_grid, 256, 0, st>>>(xa, xb, z, q, L, lam1, (t - 1.0) / tn, N);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::swap(xa, xb);
    t = tn;
  }
  broadcast_R_kernel<<<std::max(1, std::min((int)(((size_t)N * T + 255) / 256), 4 * num_sms)), 256, 0, st>>>(xa, R, N,
                                                                                                          T);
  return cudaGetLastError();
}

cudaError_t launch_init_R(const RefitJob* jobs, int njobs, int T, int num_sms, cudaStream_t st) {
  const int gy = std::min(njobs, 65535);
  const int gx = std::max(1, num_sms / gy);
  init_R_kernel<<<dim3(gx, gy), 256, 0, st>>>(jobs, T, njobs);
  return cudaGetLastError();
}

bool refit_grid_wide(const RefitPlan* plan, int njobs, int T, int pool_blocks, size_t pool_stride) {
  return plan && plan->refit == CS_REFIT_JACOBI && njobs == 1 && T * 8 <= plan->num_sms &&
         (size_t)pool_blocks * pool_stride >= (size_t)plan->N * T;
}

cudaError_t launch_refit(const RefitJob* jobs, int njobs, int T, double* pool, size_t pool_stride, int pool_blocks,
                         int outer, cudaStream_t st, const RefitPlan* plan, int* queue) {
  const int items = njobs * T;
  if (refit_grid_wide(plan, njobs, T, pool_blocks, pool_stride)) {
    // a few trials of one problem: the sweeps spread over the whole GPU, R
    // alternating between the problem's R and the workspace
    support_kernel<<<T, kRefitThreads, 0, st>>>(jobs, T, outer);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int wpb = 8;
    const dim3 grid(std::max(1, std::min((plan->N + wpb - 1) / wpb, 4 * plan->num_sms / T)), T);
    double* Ra = plan->R;
    double* Rb = pool;
    for (int sw = 0; sw < plan->jacobi_iters; ++sw) {
      jacobi_sweep_kernel<<<grid, 32 * wpb, 0, st>>>(jobs, T, outer, Ra, Rb);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      std::swap(Ra, Rb);
    }
    if (Ra != plan->R)
      return cudaMemcpyAsync(plan->R, Ra, sizeof(double) * plan->N * T, cudaMemcpyDeviceToDevice, st);
    return cudaSuccess;
  }
  // shared memory for the FP32 factor of the mixed-precision refit (|S| up to about 310)
  static thread_local size_t smem = 0;
  if (smem == 0) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, refit_kernel);
    if (e != cudaSuccess) return e;
    smem = std::min<size_t>(200 * 1024, (size_t)optin - fa.sharedSizeBytes);
    e = cudaFuncSetAttribute(refit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (queue) {
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
  }
  refit_kernel<<<std::min(items, pool_blocks), kRefitThreads, smem, st>>>(jobs, T, items, pool, pool_stride, outer,
                                                                           smem, queue);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  follow_kernel<<<std::min(items, 4096), 256, 0, st>>>(jobs, T, items);
  return cudaGetLastError();
}

cudaError_t launch_finish(const RefitJob* jobs, int njobs, int T, int num_sms, cudaStream_t st, double* err4) {
  const int items = njobs * T;
  energy_kernel<<<std::min(items, 8 * num_sms), kRefitThreads, 0, st>>>(jobs, T, items);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  select_kernel<<<njobs, 256, 0, st>>>(jobs, T);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(err4, 0, sizeof(double) * 4 * (size_t)njobs, st);
  if (e != cudaSuccess) return e;
  const int gx = std::max(1, std::min(4 * num_sms / std::max(1, std::min(njobs, 65535)), 4 * num_sms));
  error_kernel<<<dim3(gx, njobs), 256, 0, st>>>(jobs, err4);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  error_stats_kernel<<<(njobs + 255) / 256, 256, 0, st>>>(jobs, err4, njobs);
  return cudaGetLastError();
}

}  // namespace cs
