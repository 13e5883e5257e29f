// One CIM run of Algorithm 1 as a single persistent, cooperative kernel:
// initial amplitudes, the constant part of the injection, every explicit Euler
// step of Eq. mfeq1 / Eq. GMFZEC5 and the sign readout sigma = H(c).
//
// Per step the cost is the coupling product U = G_off X with X = R o c
// (continuous field, Eq. localfieldMFZ) or X = R o H(c) (binarised field,
// Eq. localfieldMFZBN), for all T trials at once (an N x N x T product).  The
// rest of the local field is constant within a run because R is fixed there,
// so it is folded into one vector per trial computed before the first step:
//   cn: R_r h_r - theta = -1/4 R_r U_r + b_r,
//       b_r = R_r (-(sqrt tau / 4) (G_off R)_r + (sqrt tau / 2) (A^T y)_r) - theta
//   bn: R_r h_r - theta = -(sqrt tau / 2) R_r U_r + q_r,
//       q_r = (sqrt tau / 2) R_r (A^T y)_r - theta
// with theta = sqrt(tau) eta^2 / 4 (Eq. MFZlocalfieldmain).
//
// Work split: CTA b owns rows [b*RB, (b+1)*RB) of G_off, which it keeps in
// shared memory for the whole run (loaded once), together with its rows of the
// state c, e, b.  Each step every CTA reads all of X (N x T) from L2, forms its
// rows of U with FP32 (or FP64) FMAs, updates its rows of c and e, writes its
// rows of the next X, and meets the other CTAs at a bounded grid barrier.  X is
// double-buffered, so one barrier per step suffices.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace cs {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTChunk = 64;  // trials per pass of the product

template <typename CT>
struct EulerArgs {
  int N, Npad, T, rows_per_cta;
  const void* Gs;  // Npad x Npad storage-precision G_off
  const double* R;
  const double* hz;
  CT* c;
  CT* e;
  CT* b;
  CT* X0;
  CT* X1;
  uint8_t* sigma;
  double* rec_c;
  double* rec_e;
  int record_steps;
  int n_steps;
  double dt;
  int pump_kind;
  double p0, p1, p_thr, d, t0, width;
  double beta, tau, Kj, theta;
  int field;
  int init_kind;
  double init_scale;
  uint64_t seed;
  int instance, outer;
  unsigned* bar;
  int* err;
  long long timeout_cycles;
  unsigned phantom;
};

__device__ __forceinline__ double pump_at(int n, int S, int kind, double p0, double p1, double p_thr,
                                          double d, double dt, double t0, double width) {
  if (kind == CS_PUMP_LINEAR) return p0 + (p1 - p0) * (double)n / (double)S;
  const double t = (double)n * dt;
  return (p_thr - d) + 2.0 * d / (1.0 + exp(-(t - t0) / width));
}

// Four consecutive storage values widened to CT.
template <typename CT, typename GT>
__device__ __forceinline__ void load4(const GT* p, CT out[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) out[j] = widen<CT, GT>(p[j]);
}
template <>
__device__ __forceinline__ void load4<float, float>(const float* p, float out[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <>
__device__ __forceinline__ void load4<double, double>(const double* p, double out[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}
template <>
__device__ __forceinline__ void load4<float, __nv_bfloat16>(const __nv_bfloat16* p, float out[4]) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&v.x);
  const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&v.y);
  const float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
  out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}
template <>
__device__ __forceinline__ void load4<float, __half>(const __half* p, float out[4]) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const __half2 lo = *reinterpret_cast<const __half2*>(&v.x);
  const __half2 hi = *reinterpret_cast<const __half2*>(&v.y);
  const float2 a = __half22float2(lo), b = __half22float2(hi);
  out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}

// U[r][tt] = sum_k Gsm[r][k] X[k][t0 + tt] for r < nr, tt < tc, written to the
// reduction buffer `red` as the per-warp partials [w][r][tt]; the caller sums
// over w.  Threads split k (in quads of 4) and t; lanes along t read X
// coalesced, lanes along k read consecutive G quads.
template <typename GT, typename CT, int RB>
__device__ __forceinline__ void product_partials(const GT* __restrict__ Gsm, int ldg, const CT* __restrict__ X,
                                                 int T, int t0, int tc, int nr, int Npad, CT* red) {
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  int TL = 1;
  while (TL < tc && TL < 32) TL <<= 1;
  const int KL = 32 / TL;
  const int tl = l % TL, kl = l / TL;
  const int KS = kWarps * KL;
  const int nq = Npad >> 2;
  const int tA = t0 + tl, tB = t0 + tl + TL;
  const bool okA = tl < tc, okB = (tl + TL) < tc;
  CT acc[RB][2];
#pragma unroll
  for (int r = 0; r < RB; ++r) { acc[r][0] = CT(0); acc[r][1] = CT(0); }
  for (int q = w * KL + kl; q < nq; q += KS) {
    CT xa[4], xb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const size_t row = (size_t)(4 * q + j) * T;
      xa[j] = okA ? __ldcg(X + row + tA) : CT(0);
      xb[j] = okB ? __ldcg(X + row + tB) : CT(0);
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (r < nr) {
        CT gv[4];
        load4<CT, GT>(Gsm + (size_t)r * ldg + 4 * q, gv);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[r][0] = fma(gv[j], xa[j], acc[r][0]);
          acc[r][1] = fma(gv[j], xb[j], acc[r][1]);
        }
      }
    }
  }
  // reduce over the k-lanes of the warp
  for (int o = TL; o < 32; o <<= 1) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      acc[r][0] += __shfl_xor_sync(0xffffffffu, acc[r][0], o);
      acc[r][1] += __shfl_xor_sync(0xffffffffu, acc[r][1], o);
    }
  }
  if (kl == 0) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (r < nr) {
        if (okA) red[(w * RB + r) * kTChunk + tl] = acc[r][0];
        if (okB) red[(w * RB + r) * kTChunk + tl + TL] = acc[r][1];
      }
    }
  }
}

template <typename GT, typename CT, int RB>
__global__ void __launch_bounds__(kThreads, 1) euler_kernel(EulerArgs<CT> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N, T = a.T, Npad = a.Npad;
  const int r0 = blockIdx.x * a.rows_per_cta;
  const int nr = max(0, min(a.rows_per_cta, N - r0));
  GT* Gsm = reinterpret_cast<GT*>(smem_raw);
  CT* red = reinterpret_cast<CT*>(smem_raw + (((size_t)RB * Npad * sizeof(GT) + 15) & ~(size_t)15));

  // Stage this CTA's rows of G_off (zero rows past the end).
  {
    const GT* src = reinterpret_cast<const GT*>(a.Gs);
    const int per = (int)(16 / sizeof(GT));
    const int vec_per_row = Npad / per;
    const int total = RB * vec_per_row;
    for (int v = threadIdx.x; v < total; v += kThreads) {
      const int r = v / vec_per_row, cv = v % vec_per_row;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (r < nr) val = *reinterpret_cast<const uint4*>(src + (size_t)(r0 + r) * Npad + cv * per);
      *reinterpret_cast<uint4*>(Gsm + (size_t)r * Npad + cv * per) = val;
    }
  }
  const double st = sqrt(a.tau);
  const CT wcoef = (a.field == CS_FIELD_CN) ? CT(-0.25) : CT(-0.5 * st);
  unsigned bar_k = 0;

  // ---- prologue: b (or q), initial c and e, first X.
  if (a.field == CS_FIELD_CN) {
    for (int idx = threadIdx.x; idx < nr * T; idx += kThreads) {
      const int r = idx / T, t = idx % T;
      a.X0[(size_t)(r0 + r) * T + t] = CT(a.R[(size_t)(r0 + r) * T + t]);
    }
    if (!grid_barrier(a.bar, ++bar_k, a.err, a.timeout_cycles, a.phantom)) return;
    for (int t0 = 0; t0 < T; t0 += kTChunk) {
      const int tc = min(kTChunk, T - t0);
      product_partials<GT, CT, RB>(Gsm, Npad, a.X0, T, t0, tc, nr, Npad, red);
      __syncthreads();
      for (int idx = threadIdx.x; idx < nr * tc; idx += kThreads) {
        const int r = idx / tc, tt = idx % tc;
        CT v = CT(0);
        for (int w = 0; w < kWarps; ++w) v += red[(w * RB + r) * kTChunk + tt];
        const size_t o = (size_t)(r0 + r) * T + t0 + tt;
        const double Rr = a.R[o];
        const double bb = Rr * (-(st / 4.0) * (double)v + (st / 2.0) * a.hz[r0 + r]) - a.theta;
        a.b[o] = CT(bb);
      }
      __syncthreads();
    }
  } else {
    for (int idx = threadIdx.x; idx < nr * T; idx += kThreads) {
      const int r = idx / T, t = idx % T;
      const size_t o = (size_t)(r0 + r) * T + t;
      a.b[o] = CT((st / 2.0) * a.R[o] * a.hz[r0 + r] - a.theta);
    }
  }
  for (int idx = threadIdx.x; idx < nr * T; idx += kThreads) {
    const int r = idx / T, t = idx % T;
    const size_t o = (size_t)(r0 + r) * T + t;
    const uint64_t key = run_key(a.seed, (uint64_t)a.instance, (uint64_t)t, (uint64_t)a.outer);
    const CT c0 = CT(initial_amplitude(key, (uint64_t)(r0 + r), a.init_kind, a.init_scale));
    a.c[o] = c0;
    a.e[o] = CT(1);
    const CT Rr = CT(a.R[o]);
    a.X1[o] = (a.field == CS_FIELD_CN) ? Rr * c0 : (c0 > CT(0) ? Rr : CT(0));
  }
  if (!grid_barrier(a.bar, ++bar_k, a.err, a.timeout_cycles, a.phantom)) return;

  // ---- Euler steps
  const CT dt = CT(a.dt), beta = CT(a.beta), tau = CT(a.tau), Kj = CT(a.Kj);
  CT* Xc = a.X1;
  CT* Xn = a.X0;
  for (int n = 0; n < a.n_steps; ++n) {
    const CT p = CT(pump_at(n, a.n_steps, a.pump_kind, a.p0, a.p1, a.p_thr, a.d, a.dt, a.t0, a.width));
    const bool last = (n + 1 == a.n_steps);
    const bool rec = n < a.record_steps;
    for (int t0 = 0; t0 < T; t0 += kTChunk) {
      const int tc = min(kTChunk, T - t0);
      product_partials<GT, CT, RB>(Gsm, Npad, Xc, T, t0, tc, nr, Npad, red);
      __syncthreads();
      for (int idx = threadIdx.x; idx < nr * tc; idx += kThreads) {
        const int r = idx / tc, tt = idx % tc;
        CT U = CT(0);
        for (int w = 0; w < kWarps; ++w) U += red[(w * RB + r) * kTChunk + tt];
        const size_t o = (size_t)(r0 + r) * T + t0 + tt;
        const CT Rr = CT(a.R[o]);
        const CT f = wcoef * Rr * U + a.b[o];
        const CT cc = a.c[o], ee = a.e[o];
        const CT c2 = cc * cc;
        const CT cn = cc + dt * ((CT(-1) + p - c2) * cc + Kj * ee * f);
        const CT en = ee + dt * (-beta * (c2 - tau) * ee);
        a.c[o] = cn;
        a.e[o] = en;
        Xn[o] = (a.field == CS_FIELD_CN) ? Rr * cn : (cn > CT(0) ? Rr : CT(0));
        if (rec) {
          const size_t ro = (size_t)n * N * T + o;
          a.rec_c[ro] = (double)cn;
          a.rec_e[ro] = (double)en;
        }
        if (last) a.sigma[o] = cn > CT(0) ? 1 : 0;
      }
      __syncthreads();
    }
    if (last) break;
    if (!grid_barrier(a.bar, ++bar_k, a.err, a.timeout_cycles, a.phantom)) return;
    CT* tmp = Xc; Xc = Xn; Xn = tmp;
  }
}

template <typename GT, typename CT, int RB>
cudaError_t launch_typed(const ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                         long long timeout_cycles, int rows_per_cta, int grid) {
  EulerArgs<CT> a;
  a.N = (int)P.N; a.Npad = (int)P.Npad; a.T = S.trials; a.rows_per_cta = rows_per_cta;
  a.Gs = P.Gs; a.R = S.R; a.hz = P.hz;
  a.c = (CT*)S.c; a.e = (CT*)S.e; a.b = (CT*)S.b; a.X0 = (CT*)S.X0; a.X1 = (CT*)S.X1;
  a.sigma = S.sigma;
  a.record_steps = (outer == 0) ? std::min(S.record_steps, prm.n_steps) : 0;
  a.rec_c = S.rec_c; a.rec_e = S.rec_e;
  a.n_steps = prm.n_steps; a.dt = prm.dt;
  a.pump_kind = prm.pump_kind; a.p0 = prm.p0; a.p1 = prm.p1; a.p_thr = prm.p_thr; a.d = prm.d;
  a.t0 = prm.t0; a.width = prm.width;
  a.beta = prm.beta; a.tau = prm.tau; a.Kj = prm.K * prm.j;
  a.theta = sqrt(prm.tau) * eta * eta / 4.0;
  a.field = prm.field; a.init_kind = prm.init_kind; a.init_scale = prm.init_scale;
  a.seed = prm.seed; a.instance = prm.instance; a.outer = outer;
  a.bar = S.bar; a.err = S.err; a.timeout_cycles = timeout_cycles;
  a.phantom = (unsigned)prm.test_phantom_ctas;

  const size_t smem = (((size_t)RB * P.Npad * sizeof(GT) + 15) & ~(size_t)15) +
                      (size_t)kWarps * RB * kTChunk * sizeof(CT);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;  // rows of G_off do not fit on chip
  auto fn = euler_kernel<GT, CT, RB>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(S.bar, 0, sizeof(unsigned), P.stream);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(kThreads), args, smem, P.stream);
}

template <typename GT, typename CT>
cudaError_t launch_rb(const ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                      long long timeout_cycles) {
  const int N = (int)P.N;
  const int ctas = std::min(P.num_sms, N);
  const int rows = (N + ctas - 1) / ctas;
  const int grid = (N + rows - 1) / rows;
  if (rows <= 2) return launch_typed<GT, CT, 2>(P, S, prm, outer, eta, timeout_cycles, rows, grid);
  if (rows <= 4) return launch_typed<GT, CT, 4>(P, S, prm, outer, eta, timeout_cycles, rows, grid);
  if (rows <= 8) return launch_typed<GT, CT, 8>(P, S, prm, outer, eta, timeout_cycles, rows, grid);
  if (rows <= 16) return launch_typed<GT, CT, 16>(P, S, prm, outer, eta, timeout_cycles, rows, grid);
  return cudaErrorInvalidConfiguration;  // N above 16 x SMs: not supported by this kernel
}

}  // namespace

cudaError_t launch_euler(const ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                         long long timeout_cycles) {
  switch (prm.precision) {
    case CS_P_FP64: return launch_rb<double, double>(P, S, prm, outer, eta, timeout_cycles);
    case CS_P_FP32: return launch_rb<float, float>(P, S, prm, outer, eta, timeout_cycles);
    case CS_P_BF16: return launch_rb<__nv_bfloat16, float>(P, S, prm, outer, eta, timeout_cycles);
    case CS_P_FP16: return launch_rb<__half, float>(P, S, prm, outer, eta, timeout_cycles);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cs
