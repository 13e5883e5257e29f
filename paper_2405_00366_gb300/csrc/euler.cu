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
// Work split (2-D, over thread-block clusters of C CTAs):
//  * cluster c owns rows [c*RPC, (c+1)*RPC) of G_off; CTA rank j of the cluster
//    owns the j-th 1/C of the k range, so its block of G_off (RPC x N/C) stays
//    in shared memory for the whole run;
//  * each step, a producer warp streams this CTA's k rows of X (N/C x T) from
//    L2 into a shared-memory ring with bulk copies (mbarrier full/empty
//    handshake), while eight consumer warps form RPC x T partial products;
//  * the C partials of a row are summed through distributed shared memory:
//    CTA j reduces and updates rows [j*RPC/C, (j+1)*RPC/C) of its cluster,
//    whose c, e, b stay in its shared memory, and writes their next X;
//  * all CTAs then meet at a bounded grid barrier; X is double-buffered in
//    global memory, so one barrier per step suffices.
// Versus every CTA reading all of X, the cluster cuts the L2 -> SM traffic of
// X by C.  C = 1 is the plain row-block split.
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "kernels_common.cuh"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace cs {

namespace {

constexpr int kConsumerWarps = 8;
constexpr int kThreads = (kConsumerWarps + 1) * 32;  // + one producer warp
constexpr int kTChunk = 64;                          // trials per block of X
constexpr int kMaxRowsPerLane = 8;                   // accumulator rows per lane

// Consumer warps per column block of trials (one: every warp takes all trials of
// a block; measured faster on GB300 than splitting the trials between warps).
__host__ __device__ __forceinline__ int col_warps(int) { return 1; }

template <typename CT>
struct EulerArgs {
  int N, Npad, T;
  int C;        // CTAs per cluster
  int RPC;      // rows of G_off per cluster
  int ORW;      // rows reduced and updated per CTA (RPC / C rounded up)
  int kq;       // k-quads per CTA (the last rank may have fewer)
  int kch;      // k rows per bulk copy (multiple of 4)
  int slots;    // ring slots
  int RW;       // rows per consumer warp (RG * MR; RPC_pad = 8 RW rows are staged)
  size_t slot_bytes;  // bytes of one ring slot
  size_t xoff;        // offset of the X chunk inside a slot (after the G tile when streaming)
  const void* Gt2;    // streamed G_off tiles [cluster][k tile][RPC_pad][32] (streaming plans)
  int nkct;           // k tiles of 32 columns (Npad / 32)
  int RG;       // row groups of a warp
  int RPC_pad;  // staged rows per CTA (multiple of 8 RW >= RPC; padding rows are zero)
  const void* Gs;  // Npad x Npad storage-precision G_off
  const float* gscale;  // row scales of G_off (FP8 storage only)
  const double* R;
  const double* hz;
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

// X is stored in blocks of kTChunk trials: block t0 (t0 a multiple of 64) holds
// trials [t0, t0 + tw) as an Npad x twp row-major matrix (twp = tw rounded up to
// 4, padding columns zero), so any run of k rows of a block is contiguous and
// moves with one bulk copy.
__host__ __device__ __forceinline__ size_t xblock(int t0, int Npad) { return (size_t)t0 * Npad; }
__host__ __device__ __forceinline__ int xwidth(int t0, int T) {
  return round4(T - t0 < kTChunk ? T - t0 : kTChunk);
}

// Shared-memory layout of one CTA (byte offsets): resident G block (absent when
// streaming), ring, partials, owned state, mbarriers.
struct Smem {
  size_t g, ring, part, st, bars, total;
};
__host__ __device__ __forceinline__ Smem smem_layout(size_t gbytes_block, size_t slot_bytes, int slots, int RPC_pad,
                                                     int twmax, int ORW, int T, size_t cbytes) {
  Smem s;
  s.g = 0;
  s.ring = align128(gbytes_block);
  s.part = s.ring + align128((size_t)slots * slot_bytes);
  s.st = s.part + align128((size_t)RPC_pad * twmax * cbytes);
  s.bars = s.st + align128((size_t)4 * ORW * T * cbytes);
  s.total = s.bars + 2 * (size_t)slots * sizeof(uint64_t);
  return s;
}

// Streamed G_off tiles of a cluster plan: tile (cluster c, k tile kc) holds rows
// [c RPC, c RPC + RPC_pad) (zero past the cluster's rows and past N) and
// columns [32 kc, 32 kc + 32), contiguous, with the quad q of row r at
// q ^ (r & 7) so that the row groups of a warp read distinct banks.
constexpr int kStreamK = 32;

template <typename GT>
__global__ void store_cluster_tiles_kernel(const double* __restrict__ G, GT* __restrict__ Gt, int N, int RPC,
                                           int RPC_pad, int NC, int nkct, const float* __restrict__ gscale) {
  const size_t total = (size_t)NC * nkct * RPC_pad * kStreamK;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t tile = idx / ((size_t)RPC_pad * kStreamK);
    const int within = (int)(idx % ((size_t)RPC_pad * kStreamK));
    const int r = within / kStreamK, kp = within % kStreamK;
    const int c = (int)(tile / nkct), kc = (int)(tile % nkct);
    const int k = 4 * ((kp >> 2) ^ (r & 7)) + (kp & 3);
    const int row = c * RPC + r, col = kc * kStreamK + k;
    double v = (r < RPC && row < N && col < N && row != col) ? G[(size_t)row * N + col] : 0.0;
    if constexpr (row_scaled<GT>::value) v = (r < RPC && row < N) ? v / gscale[row] : 0.0;
    Gt[idx] = to_storage<GT>(v);
  }
}

// Partial products of this CTA's block for one block of trials:
//   P[r][tt] = sum_{k in this CTA's range} G_off[row0 + r][k] X[k][tt].
// Warp 8 (lane 0) streams the k rows of X through the ring; warps 0-7 compute.
// `gctr` counts ring uses across calls so the mbarrier phases stay consistent.
// Consumer lanes: CG = twp/4 (rounded up to a power of two) column groups of
// four trials, RG row groups and KG = 32/(CG RG) k groups; a lane accumulates
// MR rows x 4 trials (its warp's RW = RG * MR rows are interleaved over the row
// groups) over every KG-th k-quad of each chunk, and the k groups are summed
// with shuffles at the end.  The inner loop loads four k-rows of X and MR x 4
// entries of G, then issues 16 MR independent FMAs.
template <typename GT, typename CT, int MR, bool STREAM>
__device__ __forceinline__ void cluster_partials(const EulerArgs<CT>& a, const GT* __restrict__ Gsm,
                                                 const CT* __restrict__ Xblk, int twp, int k0, int klen, int nrows,
                                                 int cl, unsigned char* ring, CT* P, uint64_t* full,
                                                 uint64_t* empty, unsigned& gctr) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nch = (klen + a.kch - 1) / a.kch;
  const int ldg = a.kq * 4;
  if (w == kConsumerWarps) {
    if (l == 0) {
      fence_proxy_async_global();
      for (int ci = 0; ci < nch; ++ci) {
        const unsigned g = gctr + ci;
        const int s = (int)(g % a.slots);
        const unsigned u = g / a.slots;
        if (u >= 1 && !mbar_wait(empty + s, (u - 1) & 1u, a.timeout_cycles)) {
          set_error(a.err, DEV_TIMEOUT);
          break;
        }
        const int kr = min(a.kch, klen - ci * a.kch);
        const unsigned bytes = (unsigned)((size_t)kr * twp * sizeof(CT));
        unsigned char* slot = ring + (size_t)s * a.slot_bytes;
        if constexpr (STREAM) {
          const unsigned gtb = (unsigned)((size_t)a.RPC_pad * kStreamK * sizeof(GT));
          const size_t kc = (size_t)(k0 + ci * a.kch) / kStreamK;
          const GT* src = reinterpret_cast<const GT*>(a.Gt2) + ((size_t)cl * a.nkct + kc) * a.RPC_pad * kStreamK;
          mbar_arrive_expect_tx(full + s, gtb + bytes);
          bulk_copy_g2s(slot, src, gtb, full + s);
        } else {
          mbar_arrive_expect_tx(full + s, bytes);
        }
        bulk_copy_g2s(slot + a.xoff, Xblk + (size_t)(k0 + ci * a.kch) * twp, bytes, full + s);
      }
    }
    gctr += nch;
    return;
  }
  // warp grid: WR row-warps x WC column-warps; a column-warp owns tcw trials
  const int WC = col_warps(twp), WR = kConsumerWarps / WC;
  const int wr = w % WR, wc = w / WR;
  const int tcw = twp / WC;
  int CG = 1;
  while (CG * 4 < tcw) CG <<= 1;
  const int RG = a.RG;             // row groups (power of two, CG * RG <= 32)
  const int KG = 32 / (CG * RG);   // k groups: lanes that split the k rows of a chunk
  const int cgi = l % CG, rg = (l / CG) % RG, kg = l / (CG * RG);
  const bool colok = cgi * 4 < tcw;
  const int col = wc * tcw + cgi * 4;  // first of this lane's four trials
  const int rbase = wr * a.RW + rg;    // this lane's rows: rbase + RG * i, i < MR
  CT acc[MR][4];
#pragma unroll
  for (int i = 0; i < MR; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = CT(0);
  bool ok = true;
  for (int ci = 0; ci < nch; ++ci) {
    const unsigned g = gctr + ci;
    const int s = (int)(g % a.slots);
    const unsigned u = g / a.slots;
    if (ok && !mbar_wait(full + s, u & 1u, a.timeout_cycles)) {
      ok = false;
      if (l == 0) set_error(a.err, DEV_TIMEOUT);
    }
    if (ok && colok) {
      const CT* xs = reinterpret_cast<const CT*>(ring + (size_t)s * a.slot_bytes + a.xoff) + col;
      const int kr = min(a.kch, klen - ci * a.kch);
      const GT* gk = STREAM ? reinterpret_cast<const GT*>(ring + (size_t)s * a.slot_bytes) + (size_t)rbase * kStreamK
                            : Gsm + (size_t)rbase * ldg + ci * a.kch;
#pragma unroll 2
      for (int kk = 4 * kg; kk < kr; kk += 4 * KG) {
        CT xv[4][4], gv[MR][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) load4<CT, CT>(xs + (size_t)(kk + j) * twp, xv[j]);
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          if constexpr (STREAM) {
            const int r = rbase + RG * i;
            load4<CT, GT>(gk + (size_t)(RG * i) * kStreamK + 4 * ((kk >> 2) ^ (r & 7)), gv[i]);
          } else {
            load4<CT, GT>(gk + (size_t)(RG * i) * ldg + kk, gv[i]);
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][q] = fma(gv[i][j], xv[j][q], acc[i][q]);
      }
    }
    __syncwarp();
    if (l == 0) mbar_arrive(empty + s);
  }
  gctr += nch;
  // sum over the k groups of the warp
  for (int o = CG * RG; o < 32; o <<= 1) {
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][q] += __shfl_xor_sync(0xffffffffu, acc[i][q], o);
  }
  if (colok && kg == 0) {
#pragma unroll
    for (int i = 0; i < MR; ++i) {
      const int r = rbase + RG * i;
      if (r < nrows) {
#pragma unroll
        for (int q = 0; q < 4; ++q) P[(size_t)r * twp + col + q] = acc[i][q];
      }
    }
  }
}

// Sum of the C cluster partials at offset `off` (all loads issued before the
// adds; fixed order rank 0, 1, ...).
template <typename CT>
__device__ __forceinline__ CT sum_partials(cg::cluster_group& cluster, CT* P, size_t off, int C) {
  CT v[8];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) v[jj] = jj < C ? cluster.map_shared_rank(P, jj)[off] : CT(0);
  CT s = v[0];
#pragma unroll
  for (int jj = 1; jj < 8; ++jj) s += v[jj];
  return s;
}

template <typename GT, typename CT, int MR, bool STREAM>
__global__ void __launch_bounds__(kThreads, 1) euler_kernel(EulerArgs<CT> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = a.C;
  const int j = (int)cluster.block_rank();
  const int cl = blockIdx.x / C;
  const int N = a.N, T = a.T, Npad = a.Npad;
  const int row0 = cl * a.RPC;                     // first row of this cluster
  const int nrows = max(0, min(a.RPC, N - row0));  // rows of this cluster
  const int nq = Npad >> 2;
  const int q0 = j * a.kq;
  const int nqj = max(0, min(a.kq, nq - q0));      // k-quads of this CTA
  const int k0 = q0 * 4, klen = nqj * 4;
  const int own0 = j * a.ORW;                      // first owned row (cluster-local)
  const int nown = max(0, min(a.ORW, nrows - own0));
  const int twmax = round4(min(T, kTChunk));
  const Smem L = smem_layout(STREAM ? 0 : (size_t)a.RPC_pad * a.kq * 4 * sizeof(GT), a.slot_bytes, a.slots,
                             a.RPC_pad, twmax, a.ORW, T, sizeof(CT));
  GT* Gsm = reinterpret_cast<GT*>(smem_raw + L.g);
  unsigned char* ring = smem_raw + L.ring;
  CT* P = reinterpret_cast<CT*>(smem_raw + L.part);
  CT* c_s = reinterpret_cast<CT*>(smem_raw + L.st);
  CT* e_s = c_s + (size_t)a.ORW * T;
  CT* b_s = e_s + (size_t)a.ORW * T;
  CT* R_s = b_s + (size_t)a.ORW * T;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + L.bars);
  uint64_t* empty = full + a.slots;

  if (threadIdx.x == 0) {
    for (int i = 0; i < a.slots; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, kConsumerWarps);
    }
    fence_mbar_init();
  }
  // Stage this CTA's block of G_off: rows [row0, row0 + nrows), k in [k0, k0 + klen).
  if (!STREAM) {
    const GT* src = reinterpret_cast<const GT*>(a.Gs);
    const int ldg = a.kq * 4;
    const int total = a.RPC_pad * nqj;
    for (int v = threadIdx.x; v < total; v += kThreads) {
      const int r = v / nqj, q = v % nqj;
      GT* d4 = Gsm + (size_t)r * ldg + 4 * q;
      if (r < nrows) {
        const GT* s4 = src + (size_t)(row0 + r) * Npad + k0 + 4 * q;
#pragma unroll
        for (int e = 0; e < 4; ++e) d4[e] = s4[e];
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) d4[e] = GT(0.0f);
      }
    }
  }
  // owned R
  for (int idx = threadIdx.x; idx < nown * T; idx += kThreads) {
    const int r = idx / T, t = idx % T;
    R_s[idx] = CT(a.R[(size_t)(row0 + own0 + r) * T + t]);
  }
  __syncthreads();
  unsigned gctr = 0;
  const double st = sqrt(a.tau);
  const CT wcoef = (a.field == CS_FIELD_CN) ? CT(-0.25) : CT(-0.5 * st);
  unsigned bar_k = 0;

  // ---- prologue: b (or q), initial c and e, first X.
  if (a.field == CS_FIELD_CN) {
    for (int idx = threadIdx.x; idx < nown * T; idx += kThreads) {
      const int r = idx / T, t = idx % T;
      const int t0 = t - t % kTChunk, twp = xwidth(t0, T);
      a.X0[xblock(t0, Npad) + (size_t)(row0 + own0 + r) * twp + (t - t0)] =
          CT(a.R[(size_t)(row0 + own0 + r) * T + t]);
    }
    fence_proxy_async_global();
    if (!grid_barrier(a.bar, ++bar_k, a.err, a.timeout_cycles, a.phantom)) { cluster.sync(); return; }
    for (int t0 = 0; t0 < T; t0 += kTChunk) {
      const int tw = min(kTChunk, T - t0), twp = round4(tw);
      cluster_partials<GT, CT, MR, STREAM>(a, Gsm, a.X0 + xblock(t0, Npad), twp, k0, klen, nrows, cl, ring, P, full,
                                            empty, gctr);
      cluster.sync();
      for (int idx = threadIdx.x; idx < nown * tw; idx += kThreads) {
        const int r = idx / tw, tt = idx % tw;
        const int gr = row0 + own0 + r;
        const CT v = sum_partials(cluster, P, (size_t)(own0 + r) * twp + tt, C) * row_scale<GT, CT>(a.gscale, gr);
        const double Rr = a.R[(size_t)gr * T + t0 + tt];
        b_s[(size_t)r * T + t0 + tt] = CT(Rr * (-(st / 4.0) * (double)v + (st / 2.0) * a.hz[gr]) - a.theta);
      }
      cluster.sync();
    }
  } else {
    for (int idx = threadIdx.x; idx < nown * T; idx += kThreads) {
      const int r = idx / T, t = idx % T;
      const int gr = row0 + own0 + r;
      b_s[idx] = CT((st / 2.0) * a.R[(size_t)gr * T + t] * a.hz[gr] - a.theta);
    }
  }
  for (int idx = threadIdx.x; idx < nown * T; idx += kThreads) {
    const int r = idx / T, t = idx % T;
    const int gr = row0 + own0 + r;
    const uint64_t key = run_key(a.seed, (uint64_t)a.instance, (uint64_t)t, (uint64_t)a.outer);
    const CT c0 = CT(initial_amplitude(key, (uint64_t)gr, a.init_kind, a.init_scale));
    c_s[idx] = c0;
    e_s[idx] = CT(1);
    const CT Rr = R_s[idx];
    const int t0 = t - t % kTChunk, twp = xwidth(t0, T);
    a.X1[xblock(t0, Npad) + (size_t)gr * twp + (t - t0)] =
        (a.field == CS_FIELD_CN) ? Rr * c0 : (c0 > CT(0) ? Rr : CT(0));
  }
  fence_proxy_async_global();
  if (!grid_barrier(a.bar, ++bar_k, a.err, a.timeout_cycles, a.phantom)) { cluster.sync(); return; }

  // ---- Euler steps
  const CT dt = CT(a.dt), beta = CT(a.beta), tau = CT(a.tau), Kj = CT(a.Kj);
  CT* Xc = a.X1;
  CT* Xn = a.X0;
  for (int n = 0; n < a.n_steps; ++n) {
    const CT p = pump_at<CT>(n, a.n_steps, a.pump_kind, a.p0, a.p1, a.p_thr, a.d, a.dt, a.t0, a.width);
    const bool last = (n + 1 == a.n_steps);
    const bool rec = n < a.record_steps;
    for (int t0 = 0; t0 < T; t0 += kTChunk) {
      const int tw = min(kTChunk, T - t0), twp = round4(tw);
      cluster_partials<GT, CT, MR, STREAM>(a, Gsm, Xc + xblock(t0, Npad), twp, k0, klen, nrows, cl, ring, P, full,
                                            empty, gctr);
      cluster.sync();
      CT* Xnb = Xn + xblock(t0, Npad);
      for (int idx = threadIdx.x; idx < nown * tw; idx += kThreads) {
        const int r = idx / tw, tt = idx % tw;
        const CT U =
            sum_partials(cluster, P, (size_t)(own0 + r) * twp + tt, C) * row_scale<GT, CT>(a.gscale, row0 + own0 + r);
        const size_t so = (size_t)r * T + t0 + tt;
        const CT Rr = R_s[so];
        const CT f = wcoef * Rr * U + b_s[so];
        const CT cc = c_s[so], ee = e_s[so];
        const CT c2 = cc * cc;
        const CT cn = cc + dt * ((CT(-1) + p - c2) * cc + Kj * ee * f);
        const CT en = ee + dt * (-beta * (c2 - tau) * ee);
        c_s[so] = cn;
        e_s[so] = en;
        const int gr = row0 + own0 + r;
        Xnb[(size_t)gr * twp + tt] = (a.field == CS_FIELD_CN) ? Rr * cn : (cn > CT(0) ? Rr : CT(0));
        const size_t o = (size_t)gr * T + t0 + tt;
        if (rec) {
          const size_t ro = (size_t)n * N * T + o;
          a.rec_c[ro] = (double)cn;
          a.rec_e[ro] = (double)en;
        }
        if (last) a.sigma[o] = cn > CT(0) ? 1 : 0;
      }
      // every CTA of the cluster has read this CTA's partials before they are rewritten
      if (t0 + kTChunk < T) cluster.sync();
    }
    if (last) break;
    // the next X is read by bulk copies (async proxy) of every CTA after the barrier
    fence_proxy_async_global();
    if (!grid_barrier(a.bar, ++bar_k, a.err, a.timeout_cycles, a.phantom)) break;
    CT* tmp = Xc; Xc = Xn; Xn = tmp;
  }
  cluster.sync();  // peers may still read this CTA's partials
}

thread_local const char* g_where = "";  // last CUDA call attempted by the launcher

struct Plan {
  int C, NC, RPC, RPC_pad, ORW, kq, kch, slots, RW, RG, MR;
  bool stream;
  size_t smem, slot_bytes, xoff;
};

template <typename CT>
using EulerFn = void (*)(EulerArgs<CT>);

template <typename GT, typename CT, bool STREAM>
EulerFn<CT> kernel_for_s(int MR) {
  switch (MR) {
    case 1: return euler_kernel<GT, CT, 1, STREAM>;
    case 2: return euler_kernel<GT, CT, 2, STREAM>;
    case 3: return euler_kernel<GT, CT, 3, STREAM>;
    case 4: return euler_kernel<GT, CT, 4, STREAM>;
    case 5: return euler_kernel<GT, CT, 5, STREAM>;
    case 6: return euler_kernel<GT, CT, 6, STREAM>;
    case 7: return euler_kernel<GT, CT, 7, STREAM>;
    default: return euler_kernel<GT, CT, 8, STREAM>;
  }
}

// Streaming (G_off tiles from memory every step) is built for the reduced
// storage types only; FP64 problems must fit on chip.
template <typename GT> struct streamable { static constexpr bool value = !std::is_same<GT, double>::value; };

template <typename GT, typename CT>
EulerFn<CT> kernel_for(int MR, bool stream) {
  if constexpr (streamable<GT>::value) {
    if (stream) return kernel_for_s<GT, CT, true>(MR);
  }
  return kernel_for_s<GT, CT, false>(MR);
}

// Work split for N and T on this GPU.  For each cluster size C in {1, 2, 4, 8}
// (or only the caller's hint) take the largest number of clusters that is
// resident at once with the footprint it implies (rows per lane MR, ring slots),
// first with G_off resident in shared memory and, if that cannot fit, with
// G_off tiles streamed from memory every step.  Keep the plan with the lowest
// estimate of one step per CTA: FMAs at 128 per clock, X bytes at 32 per clock,
// streamed G bytes at 22 per clock (one SM's share of HBM), and a fixed cost per
// cluster rank for the reduction through distributed shared memory.
template <typename GT, typename CT>
cudaError_t make_plan(const ProblemDev& P, int T, int hint, int max_ctas, bool force_stream, Plan* out) {
  const int N = (int)P.N, nq = (int)(P.Npad / 4);
  const int sms = max_ctas > 0 ? std::min(max_ctas, P.num_sms) : P.num_sms;
  const int twmax = round4(std::min(T, kTChunk));
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P.device);
  if (e != cudaSuccess) { g_where = "cudaDeviceGetAttribute(optin)"; return e; }
  const int WC = col_warps(twmax), WR = kConsumerWarps / WC;
  int CG = 1;
  while (CG * 4 < twmax / WC) CG <<= 1;
  double best_cost = 0.0;
  bool found = false;
  Plan bp{};
  const int cands[] = {1, 2, 4, 8};
  for (int pass = force_stream ? 1 : 0; pass < 2 && !found; ++pass) {
    const bool stream = pass == 1;
    if (stream && !streamable<GT>::value) break;
    for (int C : cands) {
      if (hint > 0 && C != hint) continue;
      if (C > nq || sms < C) continue;
      Plan pl{};
      pl.C = C;
      pl.stream = stream;
      if (stream) {
        pl.kq = ((nq + C - 1) / C + 7) / 8 * 8;  // whole 32-column tiles per rank
        pl.kch = kStreamK;
      } else {
        pl.kq = (nq + C - 1) / C;
        // 16 KB of X per bulk copy (measured: fewer, larger chunks cut the ring overhead)
        pl.kch = std::max(4, std::min(pl.kq * 4, (int)((16384 / (twmax * sizeof(CT))) & ~(size_t)3)));
      }
      for (int NC = std::min(sms / C, N); NC >= 1; --NC) {
        pl.RPC = (N + NC - 1) / NC;
        pl.NC = (N + pl.RPC - 1) / pl.RPC;  // no cluster without rows
        if (pl.NC != NC && NC != std::min(sms / C, N)) continue;
        // rows per row-warp, then row groups (a power of two that fits beside the
        // column groups, aiming at about four rows per lane) and rows per lane;
        // leftover lanes split k
        const int rw_need = (pl.RPC + WR - 1) / WR;
        int RG = 1;
        while (RG * 4 < rw_need && CG * RG * 2 <= 32) RG <<= 1;
        pl.RG = RG;
        pl.MR = (rw_need + RG - 1) / RG;
        if (pl.MR > kMaxRowsPerLane) break;  // fewer clusters only need more rows
        pl.RW = RG * pl.MR;
        pl.RPC_pad = WR * pl.RW;
        pl.ORW = (pl.RPC + C - 1) / C;
        EulerFn<CT> fn = kernel_for<GT, CT>(pl.MR, stream);
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, fn);
        if (e != cudaSuccess) { g_where = "cudaFuncGetAttributes"; return e; }
        const size_t cap = (size_t)optin - fa.sharedSizeBytes;
        const size_t gblock = stream ? 0 : (size_t)pl.RPC_pad * pl.kq * 4 * sizeof(GT);
        const size_t gtile = stream ? (size_t)pl.RPC_pad * kStreamK * sizeof(GT) : 0;
        pl.xoff = align128(gtile);
        pl.slot_bytes = align128(pl.xoff + (size_t)pl.kch * twmax * sizeof(CT));
        pl.slots = 0;
        for (int slots = 8; slots >= (stream ? 2 : 3); --slots) {
          pl.smem = smem_layout(gblock, pl.slot_bytes, slots, pl.RPC_pad, twmax, pl.ORW, T, sizeof(CT)).total;
          if (pl.smem <= cap) { pl.slots = slots; break; }
        }
        if (pl.slots == 0) break;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
        if (e != cudaSuccess) { g_where = "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)"; return e; }
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) { g_where = "cudaFuncSetAttribute(NonPortableClusterSizeAllowed)"; return e; }
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(C * pl.NC);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = pl.smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int maxc = 0;
        if (cudaOccupancyMaxActiveClusters(&maxc, (void*)fn, &cfg) != cudaSuccess) {
          cudaGetLastError();
          maxc = 0;
        }
        if (pl.NC > maxc) continue;
        const double fma = (double)pl.RPC_pad * pl.kq * 4 * T;
        const double xbytes = (double)pl.kq * 4 * twmax * sizeof(CT) * ((T + kTChunk - 1) / kTChunk);
        const double gbytes = stream ? (double)pl.RPC_pad * pl.kq * 4 * sizeof(GT) : 0.0;
        const double cost = fma / 128.0 + xbytes / 32.0 + gbytes / 22.0 + 300.0 * C;
        if (!found || cost < best_cost) {
          best_cost = cost;
          bp = pl;
          found = true;
        }
        break;
      }
    }
  }
  if (!found) { g_where = "make_plan: no work split fits"; return cudaErrorInvalidConfiguration; }
  *out = bp;
  return cudaSuccess;
}

// Streamed G_off tiles for a plan, rebuilt when the precision or split changes.
template <typename GT>
cudaError_t ensure_cluster_tiles(ProblemDev& P, int precision, const Plan& pl) {
  if (P.Gt2 && P.gt2_prec == precision && P.gt2_rpc == pl.RPC && P.gt2_rpcpad == pl.RPC_pad && P.gt2_nc == pl.NC)
    return cudaSuccess;
  if (P.Gt2) { dev_free(P.Gt2, P.stream); P.Gt2 = nullptr; P.gt2_prec = -1; }
  if (row_scaled<GT>::value) {
    cudaError_t e = ensure_row_scales(P);
    if (e != cudaSuccess) return e;
  }
  const int nkct = (int)(P.Npad / kStreamK);
  const size_t elems = (size_t)pl.NC * nkct * pl.RPC_pad * kStreamK;
  cudaError_t e = dev_alloc(&P.Gt2, elems * sizeof(GT), P.stream);
  if (e != cudaSuccess) return e;
  store_cluster_tiles_kernel<GT><<<P.num_sms * 4, 256, 0, P.stream>>>(P.G, (GT*)P.Gt2, (int)P.N, pl.RPC, pl.RPC_pad,
                                                                        pl.NC, nkct, P.gscale);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  P.gt2_prec = precision;
  P.gt2_rpc = pl.RPC;
  P.gt2_rpcpad = pl.RPC_pad;
  P.gt2_nc = pl.NC;
  return cudaSuccess;
}

template <typename GT, typename CT>
cudaError_t launch_typed(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                         long long timeout_cycles) {
  // plans depend only on (N, T, hint) for a given device and precision
  static thread_local struct { int64_t N; int T, hint, cap, strm, dev; Plan pl; bool valid; } cache = {
      0, 0, 0, 0, 0, -1, {}, false};
  Plan pl;
  if (cache.valid && cache.N == P.N && cache.T == S.trials && cache.hint == prm.cluster_size &&
      cache.cap == prm.max_ctas && cache.strm == prm.stream_g && cache.dev == P.device) {
    pl = cache.pl;
  } else {
    cudaError_t e = make_plan<GT, CT>(P, S.trials, prm.cluster_size, prm.max_ctas, prm.stream_g == 1, &pl);
    if (e != cudaSuccess) return e;
    cache.N = P.N; cache.T = S.trials; cache.hint = prm.cluster_size; cache.cap = prm.max_ctas;
    cache.strm = prm.stream_g; cache.dev = P.device; cache.pl = pl; cache.valid = true;
  }
  EulerArgs<CT> a;
  a.N = (int)P.N; a.Npad = (int)P.Npad; a.T = S.trials;
  a.C = pl.C; a.RPC = pl.RPC; a.ORW = pl.ORW; a.kq = pl.kq; a.kch = pl.kch; a.slots = pl.slots; a.RW = pl.RW;
  a.RPC_pad = pl.RPC_pad;
  a.slot_bytes = pl.slot_bytes;
  a.xoff = pl.xoff;
  a.nkct = (int)(P.Npad / kStreamK);
  a.Gt2 = nullptr;
  if (pl.stream) {
    cudaError_t e = ensure_cluster_tiles<GT>(P, prm.precision, pl);
    if (e != cudaSuccess) { g_where = "streamed G_off tiles"; return e; }
    a.Gt2 = P.Gt2;
  }
  a.RG = pl.RG;
  a.Gs = P.Gs; a.gscale = P.gscale; a.R = S.R; a.hz = P.hz;
  a.X0 = (CT*)S.X0; a.X1 = (CT*)S.X1;
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
  S.plan_cluster = pl.C;
  S.plan_ctas = pl.C * pl.NC;

  EulerFn<CT> fn = kernel_for<GT, CT>(pl.MR, pl.stream);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) { g_where = "cudaFuncSetAttribute(launch)"; return e; }
  e = cudaMemsetAsync(S.bar, 0, sizeof(unsigned), P.stream);
  if (e != cudaSuccess) { g_where = "cudaMemsetAsync(barrier)"; return e; }
  g_where = pl.C == 1 ? "cudaLaunchKernelEx(cooperative)" : "cudaLaunchKernelEx(cluster)";
  // A cooperative launch guarantees that every CTA is resident, which the grid
  // barrier needs; the runtime does not combine it with clusters, so a cluster
  // launch relies on the planner keeping the grid within the resident cluster
  // count (a shortfall would surface as CS_ETIMEOUT from the bounded barrier).
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  if (pl.C == 1) {
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
  } else {
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = pl.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
  }
  cfg.gridDim = dim3(pl.C * pl.NC);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = P.stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, a);
}

}  // namespace

const char* euler_last_call() { return g_where; }

cudaError_t launch_euler(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                         long long timeout_cycles) {
  switch (prm.precision) {
    case CS_P_FP64: return launch_typed<double, double>(P, S, prm, outer, eta, timeout_cycles);
    case CS_P_FP32: return launch_typed<float, float>(P, S, prm, outer, eta, timeout_cycles);
    case CS_P_BF16: return launch_typed<__nv_bfloat16, float>(P, S, prm, outer, eta, timeout_cycles);
    case CS_P_FP16: return launch_typed<__half, float>(P, S, prm, outer, eta, timeout_cycles);
    case CS_P_FP8: return launch_typed<__nv_fp8_e4m3, float>(P, S, prm, outer, eta, timeout_cycles);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cs
