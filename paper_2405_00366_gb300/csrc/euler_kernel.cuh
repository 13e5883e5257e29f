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
#pragma once

#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "kernels_common.cuh"
#include "mma.cuh"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace cs {

// The last CUDA call attempted by an Euler launcher on this thread.
extern thread_local const char* g_where;

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
  int WK;       // wide split: k-warps per row-warp (1 for the narrow split)
  int ldg;      // row stride of the resident G block, in elements
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
// trials [t0, t0 + tw) as an Npad x twp matrix (twp = tw rounded up to 4,
// padding columns zero), row-major or, for the wide split, k-pair interleaved
// (see xoff), so any run of k rows of a block is contiguous and moves with one
// bulk copy.
__host__ __device__ __forceinline__ size_t xblock(int t0, int Npad) { return (size_t)t0 * Npad; }
__host__ __device__ __forceinline__ int xwidth(int t0, int T) {
  return round4(T - t0 < kTChunk ? T - t0 : kTChunk);
}

// Shared-memory layout of one CTA (byte offsets): resident G block (absent when
// streaming), ring, partials (prows rows), owned state, mbarriers.
struct Smem {
  size_t g, ring, part, st, bars, total;
};
__host__ __device__ __forceinline__ Smem smem_layout(size_t gbytes_block, size_t slot_bytes, int slots, int prows,
                                                     int twmax, int ORW, int T, size_t cbytes) {
  Smem s;
  s.g = 0;
  s.ring = align128(gbytes_block);
  s.part = s.ring + align128((size_t)slots * slot_bytes);
  s.st = s.part + align128((size_t)prows * twmax * cbytes);
  s.bars = s.st + align128((size_t)4 * ORW * T * cbytes);
  s.total = s.bars + 2 * (size_t)slots * sizeof(uint64_t);
  return s;
}

// Streamed G_off tiles of a cluster plan: tile (cluster c, k tile kc) holds rows
// [c RPC, c RPC + RPC_pad) (zero past the cluster's rows and past N) and
// columns [32 kc, 32 kc + 32), contiguous.  A ring slot carries kch / 32
// consecutive tiles of one cluster (one bulk copy).  Inside a tile:
//  * FMA forms: row-major with the quad q of row r at q ^ (r & 7), so that the
//    row groups of a warp read distinct banks;
//  * tensor-core form (frag = 1): [row tile rt][k half h][lane][8], each
//    16 x 16 sub-tile (rows 16 rt .., columns 16 h ..) stored as the A operands
//    of one m16n8k16 MMA, lane by lane (see tc_partials).
constexpr int kStreamK = 32;

template <typename GT>
__global__ void store_cluster_tiles_kernel(const double* __restrict__ G, GT* __restrict__ Gt, int N, int RPC,
                                           int RPC_pad, int NC, int nkct, const float* __restrict__ gscale,
                                           int frag) {
  const size_t total = (size_t)NC * nkct * RPC_pad * kStreamK;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t tile = idx / ((size_t)RPC_pad * kStreamK);
    const int within = (int)(idx % ((size_t)RPC_pad * kStreamK));
    const int c = (int)(tile / nkct), kc = (int)(tile % nkct);
    int r, k;
    if (frag) {
      // sub-tile (row tile, k half) = within / 256, lane L, element e (mma.cuh)
      const int sub = within >> 8, L = (within >> 3) & 31, e = within & 7;
      int rr, kk;
      tc_arow_col(L, e, rr, kk);
      r = (sub >> 1) * 16 + rr;
      k = 16 * (sub & 1) + kk;
    } else {
      r = within / kStreamK;
      const int kp = within % kStreamK;
      k = 4 * ((kp >> 2) ^ (r & 7)) + (kp & 3);
    }
    const int row = c * RPC + r, col = kc * kStreamK + k;
    double v = (r < RPC && row < N && col < N && row != col) ? G[(size_t)row * N + col] : 0.0;
    if constexpr (row_scaled<GT>::value) v = (r < RPC && row < N) ? v / gscale[row] : 0.0;
    Gt[idx] = to_storage<GT>(v);
  }
}

// Producer side of one block of trials (lane 0 of warp 8): stream this CTA's
// k rows of X (and, when streaming, the G_off tiles) through the ring.  `gctr`
// counts ring uses across calls so the mbarrier phases stay consistent.
template <typename GT, typename CT, bool STREAM>
__device__ __forceinline__ void produce_chunks(const EulerArgs<CT>& a, const CT* __restrict__ Xblk, int twp, int k0,
                                               int klen, int cl, unsigned char* ring, uint64_t* full,
                                               uint64_t* empty, unsigned gctr) {
  const int nch = (klen + a.kch - 1) / a.kch;
  if ((threadIdx.x & 31) == 0) {
    // earlier generic accesses of X and of the ring come before the copies
    fence_proxy_async_global();
    fence_proxy_async_shared();
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
        // kr / 32 consecutive tiles of this cluster's G_off (contiguous in memory)
        const unsigned gtb = (unsigned)((size_t)(kr / kStreamK) * a.RPC_pad * kStreamK * sizeof(GT));
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
  const int ldg = a.ldg;
  if (w == kConsumerWarps) {
    produce_chunks<GT, CT, STREAM>(a, Xblk, twp, k0, klen, cl, ring, full, empty, gctr);
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
            const int r = rbase + RG * i, q = kk >> 2;  // tile q / 8 of the chunk, quad q % 8 of the tile
            load4<CT, GT>(gk + (size_t)(q >> 3) * a.RPC_pad * kStreamK + (size_t)(RG * i) * kStreamK +
                              4 * ((q & 7) ^ (r & 7)),
                          gv[i]);
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

// Partial products of the wide split (FP32 compute; a block of twp trials,
// twp in {8, 16, 32, 64}; X k-pair interleaved).  Lane (cg, rg) accumulates MR
// rows (rbase + RG i) x 4 trials (4 cg .. 4 cg + 3) with CG = twp / 4 and
// RG = 32 / CG; a quarter-warp covers 8 / cq rows x cq column groups
// (cq = min(CG, 4)), so that each shared-memory load of a half-warp is one
// wavefront.  The sums over even and odd k are kept apart in the two halves of
// each 64-bit accumulator (packed FMAs with a G pair and an X pair, no operand
// shuffling) and added at the end.  The consumer warps form WR row-warps x WK
// k-warps; k-warp kw takes every WK-th k-quad of each chunk.  The k-warps'
// partials are left in the ring (idle once every chunk of the block has been
// consumed) as [kw][RPC_pad][twp], for sum_k_warps.
template <typename GT, int MR, bool STREAM>
__device__ __forceinline__ void wide_partials(const EulerArgs<float>& a, const GT* __restrict__ Gsm,
                                              const float* __restrict__ Xblk, int twp, int k0, int klen, int nrows,
                                              int cl, unsigned char* ring, float* P, uint64_t* full,
                                              uint64_t* empty, unsigned& gctr) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nch = (klen + a.kch - 1) / a.kch;
  if (w == kConsumerWarps) {
    produce_chunks<GT, float, STREAM>(a, Xblk, twp, k0, klen, cl, ring, full, empty, gctr);
    gctr += nch;
    return;
  }
  const int WK = a.WK, WR = kConsumerWarps / WK;
  const int wr = w % WR, kw = w / WR;
  const int CG = twp >> 2, RG = 32 / CG;
  const int cq = CG < 4 ? CG : 4, qd = l >> 3, li = l & 7;
  const int cg = (qd % (CG / cq)) * cq + li % cq, rg = (qd / (CG / cq)) * (8 / cq) + li / cq;
  const int rbase = wr * a.RW + rg;
  const int c = 4 * cg;
  uint64_t acc[MR][4];
#pragma unroll
  for (int i = 0; i < MR; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0ull;
  bool ok = true;
  for (int ci = 0; ci < nch; ++ci) {
    const unsigned g = gctr + ci;
    const int s = (int)(g % a.slots);
    const unsigned u = g / a.slots;
    if (ok && !mbar_wait(full + s, u & 1u, a.timeout_cycles)) {
      ok = false;
      if (l == 0) set_error(a.err, DEV_TIMEOUT);
    }
    if (ok) {
      const unsigned char* slot = ring + (size_t)s * a.slot_bytes;
      const float* xs = reinterpret_cast<const float*>(slot + a.xoff) + 2 * c;
      const int nqc = min(a.kch, klen - ci * a.kch) >> 2;
      const GT* gk = STREAM ? reinterpret_cast<const GT*>(slot) + (size_t)rbase * kStreamK
                            : Gsm + (size_t)rbase * a.ldg + ci * a.kch;
#pragma unroll 1
      for (int q = kw; q < nqc; q += WK) {
        ulonglong2 gp[MR];
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          if constexpr (STREAM) {  // tile q / 8 of the chunk, quad q % 8 of the tile
            gp[i] = load_gpairs<GT>(gk + (size_t)(q >> 3) * a.RPC_pad * kStreamK + (size_t)(RG * i) * kStreamK +
                                    4 * ((q & 7) ^ ((rbase + RG * i) & 7)));
          } else {
            gp[i] = load_gpairs<GT>(gk + (size_t)(RG * i) * a.ldg + 4 * q);
          }
        }
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
          // k-pair 2q + pp: (X[k][t], X[k+1][t]) for the lane's four trials
          const float* xp = xs + (size_t)(2 * q + pp) * twp * 2;
          const ulonglong2 x01 = *reinterpret_cast<const ulonglong2*>(xp);
          const ulonglong2 x23 = *reinterpret_cast<const ulonglong2*>(xp + 4);
#pragma unroll
          for (int i = 0; i < MR; ++i) {
            const uint64_t gg = pp ? gp[i].y : gp[i].x;
            fma2(acc[i][0], gg, x01.x);
            fma2(acc[i][1], gg, x01.y);
            fma2(acc[i][2], gg, x23.x);
            fma2(acc[i][3], gg, x23.y);
          }
        }
      }
    }
    __syncwarp();
    if (l == 0) mbar_arrive(empty + s);
  }
  gctr += nch;
  // every consumer warp is done with the ring before it holds partials
  asm volatile("bar.sync 1, %0;" ::"r"(kConsumerWarps * 32) : "memory");
  float* dst = reinterpret_cast<float*>(ring) + (size_t)kw * a.RPC_pad * twp;
#pragma unroll
  for (int i = 0; i < MR; ++i) {
    const int r = rbase + RG * i;
    {
      float v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 h = unpack2(acc[i][q]);
        v[q] = h.x + h.y;
      }
      *reinterpret_cast<float4*>(dst + (size_t)r * twp + c) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

// P = the sum of the WK k-warp partials left in the ring (fixed order), for the
// first nrows rows; then the ring may be refilled by bulk copies.  (Measured on
// GB300: cheaper than letting the cluster read all C x WK planes remotely.)
__device__ __forceinline__ void sum_k_warps(const EulerArgs<float>& a, const unsigned char* ring, float* P,
                                            int twp, int nrows) {
  __syncthreads();
  const float* Pw = reinterpret_cast<const float*>(ring);
  const size_t plane = (size_t)a.RPC_pad * twp;
  for (int idx = threadIdx.x; idx < nrows * twp; idx += kThreads) {
    float v = Pw[idx];
    for (int kw = 1; kw < a.WK; ++kw) v += Pw[kw * plane + idx];
    P[idx] = v;
  }
  fence_proxy_async_shared();
}

// Tensor-core form (streamed FP16 or BF16 G_off, one block of eight trials):
// the product G_off X of each chunk as m16n8k16 MMAs (mma.sync, FP32
// accumulation; 16 rows x 8 trials x 16 k per instruction).  The 16-bit A
// operand is the stored G_off itself, as in the FMA forms.  X, whose B operand
// must have the same 16-bit type, is carried in two parts,
//   hi = rn(X),  lo = rn((X - hi) 2^s)   (s = kLoShift<GT>),
// whose products are accumulated apart and added as hi + 2^-s lo, so the
// product sees X to about 2 (s + 1) significant bits (22 for FP16, 16 for BF16)
// rather than the 11 or 8 of one part.  Before the first step X is scaled by a
// power of two that maps the largest |R| below 1 (so |X| <= |c|: FP16 X stays
// in range on every run that is not diverging, see xput) and U is scaled back
// exactly.
//
// Accumulation: each MMA starts from zero and its result is added to the FP32
// sums with round-to-nearest additions; chaining the MMAs of a whole k range in
// one accumulator would let the tensor cores' truncating accumulation build a
// bias (measured on GB300: about 1e-5 relative over a few hundred MMAs).
// Contraction order: the MMA sums k = 2i, 2i + 1 (operand register 0) and
// 2i + 8, 2i + 9 (register 2) in lane group i; both operands here put the
// consecutive k 4i .. 4i + 3 there instead, which only renames the summation
// index, so a lane loads its four k of G_off (per row) and of X (per trial)
// with one access each.
// Layouts: G_off tiles as in store_cluster_tiles_kernel (frag = 1); X of the
// block as [k / 16][part][trial][k % 16] (xput), 512 bytes per 16 k; lane
// L = 4 g + i of a warp reads, for 16 k, 8 bytes of X (trial g, k 4i .. 4i + 3)
// per part and 16 bytes of G_off per row tile, and holds the MMA results for
// rows g, g + 8 and trials 2i, 2i + 1.  The consumer warps form WR row-warps
// (MR row tiles of 16 each) x WK k-warps (every WK-th 16-k block of a chunk);
// the k-warps' partials go through the ring as in the wide split.

template <typename GT, int MR>
__device__ __forceinline__ void tc_partials(const EulerArgs<float>& a, const float* __restrict__ Xblk, int twp,
                                            int k0, int klen, int cl, unsigned char* ring, float* P,
                                            uint64_t* full, uint64_t* empty, unsigned& gctr) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nch = (klen + a.kch - 1) / a.kch;
  if (w == kConsumerWarps) {
    produce_chunks<GT, float, true>(a, Xblk, twp, k0, klen, cl, ring, full, empty, gctr);
    gctr += nch;
    return;
  }
  const int WK = a.WK, WR = kConsumerWarps / WK;
  const int wr = w % WR, kw = w / WR;
  const int rt0 = wr * MR;  // first row tile of this warp
  const size_t tile_u4 = (size_t)a.RPC_pad * kStreamK * sizeof(GT) / 16;  // 16-byte words per 32-column tile
  float acc[MR][2][4];
#pragma unroll
  for (int i = 0; i < MR; ++i)
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][p][q] = 0.f;
  bool ok = true;
  for (int ci = 0; ci < nch; ++ci) {
    const unsigned g = gctr + ci;
    const int s = (int)(g % a.slots);
    const unsigned u = g / a.slots;
    if (ok && !mbar_wait(full + s, u & 1u, a.timeout_cycles)) {
      ok = false;
      if (l == 0) set_error(a.err, DEV_TIMEOUT);
    }
    if (ok) {
      const unsigned char* slot = ring + (size_t)s * a.slot_bytes;
      const uint4* gt = reinterpret_cast<const uint4*>(slot) + (size_t)rt0 * 64 + l;
      const uint2* xt = reinterpret_cast<const uint2*>(slot + a.xoff) + l;
      const int nkb = min(a.kch, klen - ci * a.kch) >> 4;
#pragma unroll 1
      for (int kb = kw; kb < nkb; kb += WK) {
        const uint2 xh = xt[(size_t)kb * 64];
        const uint2 xl = xt[(size_t)kb * 64 + 32];
        // tile kb / 2 of the slot, k half kb % 2, row tiles rt0 ..
        const uint4* gb = gt + (size_t)(kb >> 1) * tile_u4 + (kb & 1) * 32;
        uint4 av[MR];
#pragma unroll
        for (int i = 0; i < MR; ++i) av[i] = gb[(size_t)i * 64];
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          float dh[4] = {0.f, 0.f, 0.f, 0.f}, dl[4] = {0.f, 0.f, 0.f, 0.f};
          mma16816<GT>(dh, av[i], xh);
          mma16816<GT>(dl, av[i], xl);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            acc[i][0][q] += dh[q];
            acc[i][1][q] += dl[q];
          }
        }
      }
    }
    __syncwarp();
    if (l == 0) mbar_arrive(empty + s);
  }
  gctr += nch;
  // one k-warp: the partials go straight to P; else every consumer warp is done
  // with the ring before it holds the k-warps' partials
  float* dst = P;
  if (WK > 1) {
    asm volatile("bar.sync 1, %0;" ::"r"(kConsumerWarps * 32) : "memory");
    dst = reinterpret_cast<float*>(ring) + (size_t)kw * a.RPC_pad * twp;
  }
  const float wlo = 1.0f / (float)(1 << tc_type<GT>::kLoShift);
  const int gq = l >> 2, c = 2 * (l & 3);
#pragma unroll
  for (int i = 0; i < MR; ++i) {
    const int r = (rt0 + i) * 16 + gq;
    *reinterpret_cast<float2*>(dst + (size_t)r * twp + c) =
        make_float2(fmaf(wlo, acc[i][1][0], acc[i][0][0]), fmaf(wlo, acc[i][1][1], acc[i][0][1]));
    *reinterpret_cast<float2*>(dst + (size_t)(r + 8) * twp + c) =
        make_float2(fmaf(wlo, acc[i][1][2], acc[i][0][2]), fmaf(wlo, acc[i][1][3], acc[i][0][3]));
  }
}

// FP32 tensor-core form (G_off resident in shared memory, FP32 problems, trial
// blocks of 16, 32 or 64): G_off X as m16n8k16 FP16 MMAs on three-way splits.
// Each CTA scales its block of G_off by a power of two (max |G| < 1) and keeps
// it as two FP16 parts, G = hi + 2^-11 lo (hi = rn(G), lo = rn((G - hi) 2^11)),
// stored once per launch in the MMA's A-operand order (the 16-bit form's tile
// layout, [row tile][16-k block][part][lane][8]); X comes in the same two FP16
// parts as in the 16-bit form (xput, power-of-two scale from max |R|).  Per
// 16 x 8 x 16 tile three MMAs, hi_G hi_X into one zeroed accumulator and
// hi_G lo_X + lo_G hi_X into another, dropping only the 2^-22 lo_G lo_X term:
// each product keeps about 22 significant bits, without bias, below the FP32
// accumulation error of a sum over the k range, so the form stands in for FP32
// FMAs.  (FP16 MMAs issue at twice the TF32 rate per k on GB300, and the
// split costs no ALU work per use.)  Warps: WC = twp / 16 column-warps of two
// n-tiles (16 trials) x WR row-warps (MR row tiles of 16) x WK k-warps (every
// WK-th 16-k block of a chunk); partials through the ring as in the wide split,
// scaled back by the block's power of two.
template <int MR>
__device__ __forceinline__ void h3_partials(const EulerArgs<float>& a, const float* __restrict__ Gsm,
                                            const float* __restrict__ Xblk, int twp, int k0, int klen, int cl,
                                            unsigned char* ring, float* P, uint64_t* full, uint64_t* empty,
                                            unsigned& gctr, float gsi) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nch = (klen + a.kch - 1) / a.kch;
  if (w == kConsumerWarps) {
    produce_chunks<float, float, false>(a, Xblk, twp, k0, klen, cl, ring, full, empty, gctr);
    gctr += nch;
    return;
  }
  const int WC = twp >> 4, WK = a.WK, WR = kConsumerWarps / (WC * WK);
  const int wc = w % WC, wr = (w / WC) % WR, kw = w / (WC * WR);
  const int rt0 = wr * MR, n0 = wc * 16;
  const int nkb16 = klen >> 4;  // 16-k blocks of this CTA's G_off block
  const uint4* ga = reinterpret_cast<const uint4*>(Gsm) + (size_t)rt0 * nkb16 * 64 + l;
  float acc[MR][2][2][4];
#pragma unroll
  for (int i = 0; i < MR; ++i)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][nt][p][q] = 0.f;
  bool ok = true;
  for (int ci = 0; ci < nch; ++ci) {
    const unsigned g = gctr + ci;
    const int s = (int)(g % a.slots);
    const unsigned u = g / a.slots;
    if (ok && !mbar_wait(full + s, u & 1u, a.timeout_cycles)) {
      ok = false;
      if (l == 0) set_error(a.err, DEV_TIMEOUT);
    }
    if (ok) {
      const uint2* xs = reinterpret_cast<const uint2*>(ring + (size_t)s * a.slot_bytes) + (size_t)n0 * 4 + l;
      const int nkb = min(a.kch, klen - ci * a.kch) >> 4;
      const uint4* gc = ga + (size_t)((ci * a.kch) >> 4) * 64;
#pragma unroll 1
      for (int kb = kw; kb < nkb; kb += WK) {
        uint2 xh[2], xl[2];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          xh[nt] = xs[((size_t)(2 * kb) * twp + nt * 8) * 4];
          xl[nt] = xs[((size_t)(2 * kb + 1) * twp + nt * 8) * 4];
        }
        const uint4* gp = gc + (size_t)kb * 64;
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          const uint4 ah = gp[(size_t)i * nkb16 * 64];
          const uint4 al = gp[(size_t)i * nkb16 * 64 + 32];
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            float dh[4] = {0.f, 0.f, 0.f, 0.f}, dl[4] = {0.f, 0.f, 0.f, 0.f};
            mma16816<__half>(dh, ah, xh[nt]);
            mma16816<__half>(dl, ah, xl[nt]);
            mma16816<__half>(dl, al, xh[nt]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              acc[i][nt][0][q] += dh[q];
              acc[i][nt][1][q] += dl[q];
            }
          }
        }
      }
    }
    __syncwarp();
    if (l == 0) mbar_arrive(empty + s);
  }
  gctr += nch;
  // one k-warp: the partials go straight to P; else every consumer warp is done
  // with the ring before it holds the k-warps' partials
  float* dst = P;
  if (WK > 1) {
    asm volatile("bar.sync 1, %0;" ::"r"(kConsumerWarps * 32) : "memory");
    dst = reinterpret_cast<float*>(ring) + (size_t)kw * a.RPC_pad * twp;
  }
  const float wlo = 1.0f / 2048.0f;
  const int gq = l >> 2, i4 = l & 3;
#pragma unroll
  for (int i = 0; i < MR; ++i) {
    const int r = (rt0 + i) * 16 + gq;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int c = n0 + nt * 8 + 2 * i4;
      const float* h = acc[i][nt][0];
      const float* o = acc[i][nt][1];
      *reinterpret_cast<float2*>(dst + (size_t)r * twp + c) =
          make_float2(fmaf(wlo, o[0], h[0]) * gsi, fmaf(wlo, o[1], h[1]) * gsi);
      *reinterpret_cast<float2*>(dst + (size_t)(r + 8) * twp + c) =
          make_float2(fmaf(wlo, o[2], h[2]) * gsi, fmaf(wlo, o[3], h[3]) * gsi);
    }
  }
}

// Stage this CTA's block of FP32 G_off for the FP32 tensor-core form: rows
// [row0, row0 + nrows) (zero up to RPC_pad), k in [k0, k0 + klen) (klen a
// multiple of 16), scaled by 2^-e with max |G| < 2^e and split into two FP16
// parts in A-operand order (h3_partials).  Returns 2^e.  Uses P as scratch.
__device__ __forceinline__ float stage_h3(const float* __restrict__ src, int Npad, int row0, int nrows, int k0,
                                          int klen, int RPC_pad, float* Gsm, float* P) {
  float m = 0.f;
  for (int v = threadIdx.x; v < nrows * klen; v += kThreads) {
    const int r = v / klen, k = v % klen;
    m = fmaxf(m, fabsf(src[(size_t)(row0 + r) * Npad + k0 + k]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) P[threadIdx.x >> 5] = m;
  __syncthreads();
  for (int i = 0; i < kThreads / 32; ++i) m = fmaxf(m, P[i]);
  __syncthreads();
  int ex = 0;
  if (m > 0.f && m <= 1e30f) frexpf(m, &ex);
  ex = max(-100, min(100, ex));
  const float gsc = ldexpf(1.f, -ex);
  __half* gh = reinterpret_cast<__half*>(Gsm);
  const int nkb16 = klen >> 4;
  const int total = (RPC_pad >> 4) * nkb16 * 512;
  for (int idx = threadIdx.x; idx < total; idx += kThreads) {
    const int unit = idx >> 9, within = idx & 511;
    const int rt = unit / nkb16, kb = unit % nkb16;
    const int part = within >> 8, L = (within >> 3) & 31, e = within & 7;
    int rr, kk;
    tc_arow_col(L, e, rr, kk);
    const int r = rt * 16 + rr, k = kb * 16 + kk;
    const float v = r < nrows ? src[(size_t)(row0 + r) * Npad + k0 + k] * gsc : 0.f;
    const __half hi = __float2half_rn(v);
    gh[idx] = part ? __float2half_rn((v - __half2float(hi)) * 2048.f) : hi;
  }
  return ldexpf(1.f, ex);
}

// Store X[k][t] = v of a block of twp trials in the layout the kernel form reads:
// xoff for the FMA forms; for the tensor-core forms the hi and lo parts at
// [k / 16][part][t][k % 16].  (With X scaled so that |X| <= |c|, FP16 overflows
// only past |c| = 6.5e4; the explicit Euler step is unstable from about
// |c| = (2 / (3 dt))^(1/2), 8 at dt = 0.01, so only a run that is already
// diverging gets there, and then every form yields non-finite amplitudes.)
template <typename GT, typename CT, bool WIDE, bool TC>
__device__ __forceinline__ void xput(CT* Xb, int k, int t, int twp, CT v) {
  if constexpr (TC) {
    using HT = typename tc_x<GT>::type;
    HT* h = reinterpret_cast<HT*>(Xb);
    const HT hi = HT(v);
    const float hf = float(hi);
    h[tc_xidx(k, t, twp, 0)] = hi;
    h[tc_xidx(k, t, twp, 1)] = HT((v - hf) * (float)(1 << tc_x<GT>::kLoShift));
  } else {
    Xb[xoff<WIDE>(k, t, twp)] = v;
  }
}

// One block of trials: this CTA's partial products in P (rows < nrows).
template <typename GT, typename CT, int MR, bool STREAM, bool WIDE, bool TC>
__device__ __forceinline__ void block_partials(const EulerArgs<CT>& a, const GT* __restrict__ Gsm,
                                               const CT* __restrict__ Xblk, int twp, int k0, int klen, int nrows,
                                               int cl, unsigned char* ring, CT* P, uint64_t* full, uint64_t* empty,
                                               unsigned& gctr, float gsi) {
  if constexpr (TC) {
    if constexpr (tc_type<GT>::value) {
      tc_partials<GT, MR>(a, Xblk, twp, k0, klen, cl, ring, P, full, empty, gctr);
    } else {
      h3_partials<MR>(a, Gsm, Xblk, twp, k0, klen, cl, ring, P, full, empty, gctr, gsi);
    }
    // (with one k-warp the partials are already in P; the cluster barrier that
    // follows orders them before any reader)
    if (a.WK > 1) sum_k_warps(a, ring, P, twp, nrows);
  } else if constexpr (WIDE) {
    wide_partials<GT, MR, STREAM>(a, Gsm, Xblk, twp, k0, klen, nrows, cl, ring, P, full, empty, gctr);
    sum_k_warps(a, ring, P, twp, nrows);
  } else {
    cluster_partials<GT, CT, MR, STREAM>(a, Gsm, Xblk, twp, k0, klen, nrows, cl, ring, P, full, empty, gctr);
  }
}

// Sum of the C cluster partials at offset `off`, in the fixed order rank 0, 1,
// ...  (A plain loop over the C ranks: measured on GB300 about 2 us per Euler
// step faster than predicated loads from all eight possible ranks.)
template <typename CT>
__device__ __forceinline__ CT sum_partials(cg::cluster_group& cluster, CT* P, size_t off, int C) {
  CT s = CT(0);
  for (int jj = 0; jj < C; ++jj) s += cluster.map_shared_rank(P, jj)[off];
  return s;
}

template <typename GT, typename CT, int MR, bool STREAM, bool WIDE, bool TC>
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
  const Smem L = smem_layout(STREAM ? 0 : (size_t)a.RPC_pad * a.ldg * sizeof(GT), a.slot_bytes, a.slots,
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
  float gsi = 1.f;  // scale of the staged block (FP32 tensor-core form)
  if constexpr (TC && !STREAM) {
    gsi = stage_h3(reinterpret_cast<const float*>(a.Gs), Npad, row0, nrows, k0, klen, a.RPC_pad,
                   reinterpret_cast<float*>(Gsm), reinterpret_cast<float*>(P));
  } else if (!STREAM) {
    const GT* src = reinterpret_cast<const GT*>(a.Gs);
    const int ldg = a.ldg;
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
  // scale of X (tensor-core form): 2^-e with max |R| < 2^e; every CTA forms it
  // from all of R, so all agree without communication
  CT xsc = CT(1), xsi = CT(1);
  if constexpr (TC) {
    double m = 0.0;
    for (size_t idx = threadIdx.x; idx < (size_t)N * T; idx += kThreads) m = fmax(m, fabs(a.R[idx]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    double* red = reinterpret_cast<double*>(P);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    for (int i = 0; i < kThreads / 32; ++i) m = fmax(m, red[i]);
    int ex = 0;
    if (m > 0.0 && m <= 1e30) frexp(m, &ex);
    ex = max(-100, min(100, ex));
    xsc = CT(ldexp(1.0, -ex));
    xsi = CT(ldexp(1.0, ex));
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
      xput<GT, CT, WIDE, TC>(a.X0 + xblock(t0, Npad), row0 + own0 + r, t - t0, twp,
                             CT(a.R[(size_t)(row0 + own0 + r) * T + t]) * xsc);
    }
    fence_proxy_async_global();
    if (!grid_barrier(a.bar, ++bar_k, a.err, a.timeout_cycles, a.phantom)) { cluster.sync(); return; }
    for (int t0 = 0; t0 < T; t0 += kTChunk) {
      const int tw = min(kTChunk, T - t0), twp = round4(tw);
      block_partials<GT, CT, MR, STREAM, WIDE, TC>(a, Gsm, a.X0 + xblock(t0, Npad), twp, k0, klen, nrows, cl, ring,
                                                    P, full, empty, gctr, gsi);
      cluster.sync();
      for (int idx = threadIdx.x; idx < nown * tw; idx += kThreads) {
        const int r = idx / tw, tt = idx % tw;
        const int gr = row0 + own0 + r;
        const CT v = sum_partials(cluster, P, (size_t)(own0 + r) * twp + tt, C) * row_scale<GT, CT>(a.gscale, gr) * xsi;
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
    xput<GT, CT, WIDE, TC>(a.X1 + xblock(t0, Npad), gr, t - t0, twp,
                           ((a.field == CS_FIELD_CN) ? Rr * c0 : (c0 > CT(0) ? Rr : CT(0))) * xsc);
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
      block_partials<GT, CT, MR, STREAM, WIDE, TC>(a, Gsm, Xc + xblock(t0, Npad), twp, k0, klen, nrows, cl, ring, P,
                                                    full, empty, gctr, gsi);
      cluster.sync();
      CT* Xnb = Xn + xblock(t0, Npad);
      for (int idx = threadIdx.x; idx < nown * tw; idx += kThreads) {
        const int r = idx / tw, tt = idx % tw;
        const int gr = row0 + own0 + r;
        const CT U = sum_partials(cluster, P, (size_t)(own0 + r) * twp + tt, C) * row_scale<GT, CT>(a.gscale, gr) * xsi;
        const size_t so = (size_t)r * T + t0 + tt;
        const CT Rr = R_s[so];
        const CT f = wcoef * Rr * U + b_s[so];
        const CT cc = c_s[so], ee = e_s[so];
        const CT c2 = cc * cc;
        const CT cn = cc + dt * ((CT(-1) + p - c2) * cc + Kj * ee * f);
        const CT en = ee + dt * (-beta * (c2 - tau) * ee);
        c_s[so] = cn;
        e_s[so] = en;
        xput<GT, CT, WIDE, TC>(Xnb, gr, tt, twp, ((a.field == CS_FIELD_CN) ? Rr * cn : (cn > CT(0) ? Rr : CT(0))) * xsc);
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

}  // namespace
}  // namespace cs
