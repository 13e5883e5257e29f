// Problem set-up on the GPU: the Gram matrix G = A^T A, the Zeeman vector
// h^z = A^T y, g = diag G (Eq. l0Hamiltonian; the Zeeman term of
// Eq. localfieldMFZ) and the copy of G used by the Euler loop: G with its
// diagonal removed (the sums of Eq. localfieldMFZ and Eq. localfieldMFZBN run
// over r' != r), in the storage precision of the solve.
#include "common.cuh"
#include "internal.h"

namespace cs {

namespace {

constexpr int GT_TILE = 64;   // output tile edge
constexpr int GT_K = 16;      // rows of A per stage

// One 64 x 64 tile (bi <= bj) of G in FP64.  Tile pairs are enumerated over the
// upper triangle; each tile is written to (bi, bj) and mirrored to (bj, bi), so
// G is exactly symmetric.  Entry order of the k-sum is the same for (i, j) and
// (j, i) inside a diagonal tile, so those are bitwise equal too.
__global__ void __launch_bounds__(256) gram_kernel(const double* __restrict__ A, double* __restrict__ G,
                                                   int M, int N, int nb) {
  __shared__ double As[GT_K][GT_TILE];
  __shared__ double Bs[GT_K][GT_TILE];
  // decode the upper-triangle pair index
  int p = blockIdx.x, bi = 0;
  while (p >= nb - bi) { p -= nb - bi; ++bi; }
  const int bj = bi + p;
  const int i0 = bi * GT_TILE, j0 = bj * GT_TILE;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

  const int lc = threadIdx.x & 63, lk = threadIdx.x >> 6;  // loader coordinates
  for (int k0 = 0; k0 < M; k0 += GT_K) {
#pragma unroll
    for (int m = 0; m < GT_K / 4; ++m) {
      const int k = k0 + lk + 4 * m;
      const int ci = i0 + lc, cj = j0 + lc;
      As[lk + 4 * m][lc] = (k < M && ci < N) ? A[(size_t)k * N + ci] : 0.0;
      Bs[lk + 4 * m][lc] = (k < M && cj < N) ? A[(size_t)k * N + cj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GT_K; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i >= N || j >= N) continue;
      if (bi == bj && i > j) continue;
      G[(size_t)i * N + j] = acc[a][b];
      G[(size_t)j * N + i] = acc[a][b];
    }
}

// h^z_j = sum_k A_kj y_k (one thread per column, coalesced over j); also g_j
// and the finite check of A and y.
__global__ void zeeman_kernel(const double* __restrict__ A, const double* __restrict__ y,
                              const double* __restrict__ G, double* __restrict__ hz,
                              double* __restrict__ g, int M, int N, int* flag) {
  const int jcol = blockIdx.x * blockDim.x + threadIdx.x;
  if (jcol >= N) return;
  double s = 0.0;
  bool finite = true;
  for (int k = 0; k < M; ++k) {
    const double a = A[(size_t)k * N + jcol], yk = y[k];
    finite &= isfinite(a) && isfinite(yk);
    s = fma(a, yk, s);
  }
  hz[jcol] = s;
  g[jcol] = G[(size_t)jcol * N + jcol];
  if (!finite) atomicExch(flag, 1);
}

template <typename GT> __device__ __forceinline__ GT narrow(double v);
template <> __device__ __forceinline__ double narrow<double>(double v) { return v; }
template <> __device__ __forceinline__ float narrow<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 narrow<__nv_bfloat16>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ __half narrow<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __nv_fp8_e4m3 narrow<__nv_fp8_e4m3>(double v) {
  return __nv_fp8_e4m3((float)v);
}

// Gs = G with a zero diagonal, rounded to GT (divided by its row's scale when GT
// is row-scaled), zero-padded to Npad x Npad.
template <typename GT>
__global__ void store_coupling_kernel(const double* __restrict__ G, GT* __restrict__ Gs, int N, int Npad,
                                      const float* __restrict__ gscale) {
  const size_t total = (size_t)Npad * Npad;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / Npad), j = (int)(idx % Npad);
    double v = (i < N && j < N && i != j) ? G[(size_t)i * N + j] : 0.0;
    if constexpr (row_scaled<GT>::value) v = i < N ? v / gscale[i] : 0.0;
    Gs[idx] = narrow<GT>(v);
  }
}

// Row scales for FP8 storage: s_r = max_{k != r} |G_rk| / 448 (E4M3's largest
// finite value), 1 for an all-zero row.  One block per row.
__global__ void row_scale_kernel(const double* __restrict__ G, float* __restrict__ gscale, int N) {
  __shared__ double red[8];
  const int r = blockIdx.x;
  double m = 0.0;
  for (int k = threadIdx.x; k < N; k += blockDim.x)
    if (k != r) m = fmax(m, fabs(G[(size_t)r * N + k]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mm = fmax(mm, red[i]);
    gscale[r] = mm > 0.0 ? (float)(mm / 448.0) : 1.0f;
  }
}

}  // namespace

cudaError_t launch_gram(const ProblemDev& P) {
  const int N = (int)P.N, M = (int)P.M;
  const int nb = (N + GT_TILE - 1) / GT_TILE;
  const int pairs = nb * (nb + 1) / 2;
  gram_kernel<<<pairs, 256, 0, P.stream>>>(P.A, P.G, M, N, nb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  zeeman_kernel<<<(N + 127) / 128, 128, 0, P.stream>>>(P.A, P.y, P.G, P.hz, P.g, M, N, P.flag);
  return cudaGetLastError();
}

size_t storage_bytes(int precision) {
  switch (precision) {
    case CS_P_FP64: return 8;
    case CS_P_FP32: return 4;
    case CS_P_FP8: return 1;
    default: return 2;
  }
}

cudaError_t ensure_row_scales(ProblemDev& P) {
  if (P.gscale) return cudaSuccess;
  cudaError_t e = dev_alloc((void**)&P.gscale, (size_t)P.N * sizeof(float), P.stream);
  if (e != cudaSuccess) return e;
  row_scale_kernel<<<(int)P.N, 256, 0, P.stream>>>(P.G, P.gscale, (int)P.N);
  return cudaGetLastError();
}

cudaError_t launch_store_coupling(ProblemDev& P, int precision) {
  if (P.gs_prec == precision && P.Gs) return cudaSuccess;
  if (P.Gs) { dev_free(P.Gs, P.stream); P.Gs = nullptr; P.gs_prec = -1; }
  const size_t bytes = (size_t)P.Npad * P.Npad * storage_bytes(precision);
  cudaError_t e = dev_alloc(&P.Gs, bytes, P.stream);
  if (e != cudaSuccess) return e;
  const int N = (int)P.N, Npad = (int)P.Npad;
  const int blocks = P.num_sms * 4;
  float* sc = P.gscale;
  switch (precision) {
    case CS_P_FP64: store_coupling_kernel<double><<<blocks, 256, 0, P.stream>>>(P.G, (double*)P.Gs, N, Npad, sc); break;
    case CS_P_FP32: store_coupling_kernel<float><<<blocks, 256, 0, P.stream>>>(P.G, (float*)P.Gs, N, Npad, sc); break;
    case CS_P_BF16:
      store_coupling_kernel<__nv_bfloat16><<<blocks, 256, 0, P.stream>>>(P.G, (__nv_bfloat16*)P.Gs, N, Npad, sc);
      break;
    case CS_P_FP16: store_coupling_kernel<__half><<<blocks, 256, 0, P.stream>>>(P.G, (__half*)P.Gs, N, Npad, sc); break;
    case CS_P_FP8:
      if ((e = ensure_row_scales(P)) != cudaSuccess) return e;
      store_coupling_kernel<__nv_fp8_e4m3><<<blocks, 256, 0, P.stream>>>(P.G, (__nv_fp8_e4m3*)P.Gs, N, Npad,
                                                                         P.gscale);
      break;
    default: return cudaErrorInvalidValue;
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) P.gs_prec = precision;
  return e;
}

}  // namespace cs
