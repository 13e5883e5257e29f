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
// Work split: CTA b owns a block of rows of G_off, which it keeps in shared
// memory for the whole run (loaded once), and the same rows of the state c, e,
// b.  Each step every CTA streams all of X (N x T) from L2 into shared memory
// with bulk copies (each warp double-buffers its own run of k-rows), forms its
// rows of U with FP32 (or FP64) FMAs, updates its rows of c and e, writes its
// rows of the next X, and meets the other CTAs at a bounded grid barrier.  X is
// double-buffered in global memory, so one barrier per step suffices.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tma.cuh"

namespace cs {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTChunk = 64;  // trials per pass of the product
constexpr int kChunkQuads = 4;  // k-quads (16 rows of X) per bulk copy

__host__ __device__ __forceinline__ size_t align128(size_t b) { return (b + 127) & ~(size_t)127; }

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

// Offset of element (r, t) of a coupling operand X.  X is stored in blocks of
// kTChunk trials: block tc holds trials [64 tc, 64 tc + tw) as an Npad x tw
// row-major matrix, so any run of k-rows of one block is contiguous in memory
// and can be moved by one bulk copy.
__device__ __forceinline__ size_t xoff(int r, int t, int T, int Npad) {
  const int tc = t / kTChunk, tt = t % kTChunk;
  const int tw = min(kTChunk, T - tc * kTChunk);
  return (size_t)tc * Npad * kTChunk + (size_t)r * tw + tt;
}

// Per-warp partial products of one block of trials:
//   U[r][tt] = sum_k Gsm[r][k] X[k][tt],  r < nr, tt < tw,
// with the k range split into one contiguous run of k-quads per warp.  Each
// warp streams its run of X through two private shared-memory slots: lane 0
// issues a bulk copy of the next chunk (kChunkQuads quads of k-rows) while the
// warp computes on the current one, completion signalled by the slot's
// mbarrier.  Lanes split (t, k); lanes along t read X conflict-free, lanes
// along k read consecutive quads of the G row.  On return the per-warp
// partials are in `red` as [w][r][tt] (red aliases the slot ring, so the
// whole CTA synchronises first).  Returns false if a copy wait timed out.
template <typename GT, typename CT, int RB>
__device__ __forceinline__ bool product_partials(const GT* __restrict__ Gsm, int Npad, const CT* __restrict__ Xblk,
                                                 int tw, int nr, CT* ring, uint64_t* bars, unsigned& phases,
                                                 long long timeout_cycles, int* err, CT* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  int TL = 1;
  while (TL < tw && TL < 32) TL <<= 1;
  const int KL = 32 / TL;
  const int tl = l % TL, kl = l / TL;
  const bool okA = tl < tw, okB = (tl + TL) < tw;
  const int nq = Npad >> 2;
  const int qb = (int)((long long)nq * w / kWarps), qe = (int)((long long)nq * (w + 1) / kWarps);
  const int nch = (qe - qb + kChunkQuads - 1) / kChunkQuads;
  const size_t slot_elems = (size_t)kChunkQuads * 4 * tw;
  CT* wslots = ring + (size_t)w * 2 * slot_elems;
  uint64_t* wb = bars + 2 * w;
  int issued = 0;
  auto issue = [&](int ci) {
    const int q0 = qb + ci * kChunkQuads;
    const int cq = min(kChunkQuads, qe - q0);
    const unsigned bytes = (unsigned)((size_t)cq * 4 * tw * sizeof(CT));
    const int s = ci & 1;
    mbar_arrive_expect_tx(wb + s, bytes);
    bulk_copy_g2s(wslots + s * slot_elems, Xblk + (size_t)q0 * 4 * tw, bytes, wb + s);
  };
  if (l == 0) {
    fence_proxy_async_global();
    fence_proxy_async_shared();
    if (nch > 0) issue(0);
    if (nch > 1) issue(1);
  }
  issued = min(nch, 2);
  CT acc[RB][2];
#pragma unroll
  for (int r = 0; r < RB; ++r) { acc[r][0] = CT(0); acc[r][1] = CT(0); }
  bool ok = true;
  for (int ci = 0; ci < issued; ++ci) {
    const int s = ci & 1;
    const bool got = mbar_wait(wb + s, (phases >> s) & 1u, timeout_cycles);
    phases ^= 1u << s;
    if (!got) {
      ok = false;
      if (l == 0) set_error(err, DEV_TIMEOUT);
    }
    if (ok) {
      const CT* xs = wslots + s * slot_elems;
      const int q0 = qb + ci * kChunkQuads;
      const int cq = min(kChunkQuads, qe - q0);
      for (int j = kl; j < cq; j += KL) {
        CT xa[4], xb[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          xa[jj] = okA ? xs[(4 * j + jj) * tw + tl] : CT(0);
          xb[jj] = okB ? xs[(4 * j + jj) * tw + tl + TL] : CT(0);
        }
        const GT* gq = Gsm + 4 * (q0 + j);
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          if (r < nr) {
            CT gv[4];
            load4<CT, GT>(gq + (size_t)r * Npad, gv);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              acc[r][0] = fma(gv[jj], xa[jj], acc[r][0]);
              acc[r][1] = fma(gv[jj], xb[jj], acc[r][1]);
            }
          }
        }
      }
    }
    __syncwarp();
    if (ok && ci + 2 < nch) {
      if (l == 0) issue(ci + 2);
      issued = ci + 3;
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
  __syncthreads();  // every warp is done with its slots: red may overwrite the ring
  if (kl == 0) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (r < nr) {
        if (okA) red[(w * RB + r) * tw + tl] = acc[r][0];
        if (okB) red[(w * RB + r) * tw + tl + TL] = acc[r][1];
      }
    }
  }
  __syncthreads();
  return ok;
}

template <typename GT, typename CT, int RB>
__global__ void __launch_bounds__(kThreads, 1) euler_kernel(EulerArgs<CT> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int N = a.N, T = a.T, Npad = a.Npad;
  const int r0 = blockIdx.x * a.rows_per_cta;
  const int nr = max(0, min(a.rows_per_cta, N - r0));
  const int twmax = min(T, kTChunk);
  GT* Gsm = reinterpret_cast<GT*>(smem_raw);
  const size_t g_bytes = align128((size_t)a.rows_per_cta * Npad * sizeof(GT));
  CT* ring = reinterpret_cast<CT*>(smem_raw + g_bytes);
  const size_t ring_bytes = align128((size_t)kWarps * 2 * kChunkQuads * 4 * twmax * sizeof(CT));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + g_bytes + ring_bytes);
  CT* red = ring;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2 * kWarps; ++i) mbar_init(bars + i, 1);
    fence_mbar_init();
  }
  // Stage this CTA's rows of G_off.
  {
    const GT* src = reinterpret_cast<const GT*>(a.Gs);
    const int per = (int)(16 / sizeof(GT));
    const int vec_per_row = Npad / per;
    const int total = nr * vec_per_row;
    for (int v = threadIdx.x; v < total; v += kThreads) {
      const int r = v / vec_per_row, cv = v % vec_per_row;
      *reinterpret_cast<uint4*>(Gsm + (size_t)r * Npad + cv * per) =
          *reinterpret_cast<const uint4*>(src + (size_t)(r0 + r) * Npad + cv * per);
    }
  }
  __syncthreads();
  unsigned phases = 0;
  const double st = sqrt(a.tau);
  const CT wcoef = (a.field == CS_FIELD_CN) ? CT(-0.25) : CT(-0.5 * st);
  unsigned bar_k = 0;

  // ---- prologue: b (or q), initial c and e, first X.
  if (a.field == CS_FIELD_CN) {
    for (int idx = threadIdx.x; idx < nr * T; idx += kThreads) {
      const int r = idx / T, t = idx % T;
      a.X0[xoff(r0 + r, t, T, Npad)] = CT(a.R[(size_t)(r0 + r) * T + t]);
    }
    fence_proxy_async_global();
    if (!grid_barrier(a.bar, ++bar_k, a.err, a.timeout_cycles, a.phantom)) return;
    for (int t0 = 0; t0 < T; t0 += kTChunk) {
      const int tw = min(kTChunk, T - t0);
      product_partials<GT, CT, RB>(Gsm, Npad, a.X0 + (size_t)t0 * Npad, tw, nr, ring, bars, phases,
                                   a.timeout_cycles, a.err, red);
      for (int idx = threadIdx.x; idx < nr * tw; idx += kThreads) {
        const int r = idx / tw, tt = idx % tw;
        CT v = CT(0);
        for (int w = 0; w < kWarps; ++w) v += red[(w * RB + r) * tw + tt];
        const size_t o = (size_t)(r0 + r) * T + t0 + tt;
        const double Rr = a.R[o];
        const double bb = Rr * (-(st / 4.0) * (double)v + (st / 2.0) * a.hz[r0 + r]) - a.theta;
        a.b[o] = CT(bb);
      }
      fence_proxy_async_shared();
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
    a.X1[xoff(r0 + r, t, T, Npad)] = (a.field == CS_FIELD_CN) ? Rr * c0 : (c0 > CT(0) ? Rr : CT(0));
  }
  fence_proxy_async_global();
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
      const int tw = min(kTChunk, T - t0);
      product_partials<GT, CT, RB>(Gsm, Npad, Xc + (size_t)t0 * Npad, tw, nr, ring, bars, phases,
                                   a.timeout_cycles, a.err, red);
      CT* Xnb = Xn + (size_t)t0 * Npad;
      for (int idx = threadIdx.x; idx < nr * tw; idx += kThreads) {
        const int r = idx / tw, tt = idx % tw;
        CT U = CT(0);
        for (int w = 0; w < kWarps; ++w) U += red[(w * RB + r) * tw + tt];
        const size_t o = (size_t)(r0 + r) * T + t0 + tt;
        const CT Rr = CT(a.R[o]);
        const CT f = wcoef * Rr * U + a.b[o];
        const CT cc = a.c[o], ee = a.e[o];
        const CT c2 = cc * cc;
        const CT cn = cc + dt * ((CT(-1) + p - c2) * cc + Kj * ee * f);
        const CT en = ee + dt * (-beta * (c2 - tau) * ee);
        a.c[o] = cn;
        a.e[o] = en;
        Xnb[(size_t)(r0 + r) * tw + tt] = (a.field == CS_FIELD_CN) ? Rr * cn : (cn > CT(0) ? Rr : CT(0));
        if (rec) {
          const size_t ro = (size_t)n * N * T + o;
          a.rec_c[ro] = (double)cn;
          a.rec_e[ro] = (double)en;
        }
        if (last) a.sigma[o] = cn > CT(0) ? 1 : 0;
      }
      // the next X is read by bulk copies (async proxy) after the grid barrier, and
      // the ring that held `red` is refilled by bulk copies
      fence_proxy_async_global();
      fence_proxy_async_shared();
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

  const int twmax = std::min(S.trials, kTChunk);
  const size_t smem = align128((size_t)rows_per_cta * P.Npad * sizeof(GT)) +
                      align128((size_t)kWarps * 2 * kChunkQuads * 4 * twmax * sizeof(CT)) +
                      2 * kWarps * sizeof(uint64_t);
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
