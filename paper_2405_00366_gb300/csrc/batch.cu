// Batched solves of many independent problems of uneven size (Algorithm 1 for
// each): one outer iteration of every problem in one persistent launch.
//
// The launch is a grid of thread-block clusters of cc CTAs that take problems
// from a device work queue, largest first, so the tail is short.  The queue's
// first n_large problems (the large ones) are each run by a whole cluster: CTA
// rank j of the cluster takes row tiles j, j + cc, ... of every product and
// update, and the cluster barrier ends each Euler step (X of the next step is
// complete once every CTA has written its rows).  Every other problem is run
// by one CTA alone, with no inter-CTA synchronisation.  A run is one complete
// CIM run of Algorithm 1's inner loop: the prologue (b or q, initial c and e),
// every Euler step of Eq. mfeq1 / Eq. GMFZEC5 with the field of
// Eq. localfieldMFZ or Eq. localfieldMFZBN, and the readout sigma = H(c).
//
// G_off of a problem is stored for streaming: tiles of kRT rows x kKC columns,
// tile (rt, kc) contiguous, rows zero-padded to a multiple of kRT and columns
// to Npad.  Inside a tile, the quad (4 columns) q of row r sits at position
// q ^ (r & 7), so the lanes of a warp that read the same quad of eight
// consecutive rows hit eight different banks.  Each step, for each row tile, a
// producer warp streams the tile's G_off blocks and the matching k rows of X
// into a shared-memory ring with bulk copies (mbarrier full/empty handshake);
// eight consumer warps accumulate the tile's rows of U = G_off X, then update
// those rows of c and e (kept in global memory, L2-resident) and write their
// next X.  With BF16 / FP16 storage and 8 or 16 trials the product runs on the
// tensor cores instead (tile_product_tc): the tiles then hold G_off in the
// MMA's A-operand order and X is stored in two 16-bit parts.
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "kernels_common.cuh"
#include "mma.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace cs {

namespace cg = cooperative_groups;

namespace {

constexpr int kBWarps = 8;                     // consumer warps
constexpr int kBThreads = (kBWarps + 1) * 32;  // + one producer warp
constexpr int kRT = 128;                       // rows per tile (16 per consumer warp)
constexpr int kKC = 32;                        // columns (k) per tile

// Tiled, swizzled copy of G_off (see the file comment), divided by its row
// scales when the storage type is row-scaled.  frag = 1: inside each tile the
// A-operand order of the mma.sync form, [row tile of 16][k half][lane][8];
// frag = 2: the canonical operand layout of the tcgen05 form.
template <typename GT>
__global__ void store_tiled_kernel(const double* __restrict__ G, GT* __restrict__ Gt, int N, int nrt, int nkc,
                                   const float* __restrict__ gscale, int frag) {
  const size_t total = (size_t)nrt * nkc * kRT * kKC;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t tile = idx / (kRT * kKC);
    const int within = (int)(idx % (kRT * kKC));
    const int rt = (int)(tile / nkc), kc = (int)(tile % nkc);
    int r, k;
    if (frag == 2) {
      // tcgen05 operand order: two 16-k blocks of 128 rows, each in the
      // canonical no-swizzle K-major layout (tcgen05.cuh), 4 KB apart
      const int b = 2 * within, blk = b >> 12, rem = b & 4095;
      r = (rem >> 8) * 8 + ((rem & 127) >> 4);
      k = blk * 16 + ((rem >> 7) & 1) * 8 + ((rem & 15) >> 1);
    } else if (frag) {
      const int sub = within >> 8, L = (within >> 3) & 31, e = within & 7;
      int rr, kk;
      tc_arow_col(L, e, rr, kk);
      r = (sub >> 1) * 16 + rr;
      k = 16 * (sub & 1) + kk;
    } else {
      r = within / kKC;
      const int kp = within % kKC;
      k = 4 * ((kp >> 2) ^ (r & 7)) + (kp & 3);
    }
    const int row = rt * kRT + r, col = kc * kKC + k;
    double v = (row < N && col < N && row != col) ? G[(size_t)row * N + col] : 0.0;
    if constexpr (row_scaled<GT>::value) v = row < N ? v / gscale[row] : 0.0;
    Gt[idx] = to_storage<GT>(v);
  }
}

template <typename CT>
struct BInst {
  int N, nrt, nkc;         // rows, row tiles, column tiles (nkc * kKC = Npad)
  const void* Gt;          // tiled G_off
  const float* gscale;     // row scales (FP8 storage)
  const double* R;         // N x T
  const double* hz;        // N
  const double* g;         // N, diag G (the corrected mode's self-term)
  CT* X0;                  // Npad x twp, rows >= N zero
  CT* X1;
  CT* state;               // c, e, b: 3 x N x T
  uint8_t* sigma;          // N x T
  double theta;            // sqrt(tau) eta^2 / 4 of this problem
  int inst;                // instance number of the initial-amplitude key
  // this problem's run parameters (cs_params)
  int n_steps, pump_kind, field, init_kind, self_term;
  double dt, p0, p1, p_thr, d, t0, width, beta, tau, Kj, init_scale;
  uint64_t seed;
};

template <typename CT>
struct BArgs {
  const BInst<CT>* insts;
  const int* order;  // processing order (largest first)
  int n;
  int T, twp, slots;
  int tps;          // column tiles per ring slot (1, 2 or 4)
  int* queue;
  int outer;
  int* err;
  long long timeout_cycles;
  int cc;           // CTAs per cluster
  int n_large;      // queue items [0, n_large) are run by a whole cluster
  int step_cap;     // > 0: at most this many Euler steps per run (tuning runs)
  int test_skip;    // test hook: the CTA's first ring copy is never issued
};

// One ring slot: tps consecutive column tiles of G_off, then their tps x kKC
// rows of X.
__host__ __device__ __forceinline__ size_t b_slot_bytes(int twp, size_t gbytes, size_t cbytes, int tps) {
  return align128((size_t)tps * kRT * kKC * gbytes + (size_t)tps * kKC * twp * cbytes);
}

// Partials of one row tile: kRT x twp, or for the wide form WK = 64 / twp
// planes of it (64 kRT values either way).
__host__ __device__ __forceinline__ size_t b_part_bytes(int twp, size_t cbytes, bool pair) {
  return align128((size_t)kRT * (pair ? 64 : twp) * cbytes);
}

// Producer of one row tile (lane 0 of the producer warp): chunks [ci0, ci1) of
// its column tiles of G_off, tps per ring slot, each slot followed by the
// matching k rows of X; chunk ci is ring use gctr + ci.
template <typename GT, typename CT>
__device__ __forceinline__ bool produce_row_tile(const BArgs<CT>& a, const BInst<CT>& I, const CT* __restrict__ X,
                                                 int rt, unsigned char* ring, size_t slot, uint64_t* full,
                                                 uint64_t* empty, unsigned gctr, unsigned* issued, int ci0,
                                                 int ci1) {
  const int twp = a.twp, nkc = I.nkc;
  const size_t gtile = (size_t)kRT * kKC * sizeof(GT);
  const unsigned xbytes = (unsigned)(kKC * twp * sizeof(CT));
  fence_proxy_async_global();
  const GT* gsrc = reinterpret_cast<const GT*>(I.Gt) + (size_t)rt * nkc * kRT * kKC;
  for (int ci = ci0; ci < ci1; ++ci) {
    const unsigned g = gctr + ci;
    const int s = (int)(g % a.slots);
    const unsigned u = g / a.slots;
    if (u >= 1 && !mbar_wait(empty + s, (u - 1) & 1u, a.timeout_cycles)) {
      set_error(a.err, DEV_TIMEOUT);
      return false;
    }
    if (a.test_skip && g == 0) continue;  // test hook: the waits on this slot run out
    const int kc0 = ci * a.tps, nt = min(a.tps, nkc - kc0);
    unsigned char* dst = ring + (size_t)s * slot;
    issued[s] = g + 1;
    mbar_arrive_expect_tx(full + s, (unsigned)(nt * (gtile + xbytes)));
    bulk_copy_g2s(dst, gsrc + (size_t)kc0 * kRT * kKC, (unsigned)(nt * gtile), full + s);
    bulk_copy_g2s(dst + a.tps * gtile, X + (size_t)kc0 * kKC * twp, (unsigned)(nt * xbytes), full + s);
  }
  return true;
}

// Partial-free product of one row tile: U[r][tt] = sum_k G_off[rt*kRT + r][k] X[k][tt]
// for r < kRT, written to P (kRT x twp).  Lane layout: CG column groups of four
// trials, RG row groups, KG k groups (CG RG KG = 32), MR = 16 / RG rows per lane.
template <typename GT, typename CT, int MR>
__device__ __forceinline__ bool tile_product(const BArgs<CT>& a, const BInst<CT>& I, const CT* __restrict__ X,
                                             int rt, unsigned char* ring, size_t slot, CT* P, uint64_t* full,
                                             uint64_t* empty, unsigned& gctr, unsigned* issued) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int twp = a.twp, nkc = I.nkc;
  const size_t gtile = (size_t)kRT * kKC * sizeof(GT);
  const int nch = (nkc + a.tps - 1) / a.tps;
  bool ok = true;
  if (w == kBWarps) {
    if (l == 0) produce_row_tile<GT, CT>(a, I, X, rt, ring, slot, full, empty, gctr, issued, 0, nch);
    gctr += nch;
    return true;
  }
  int CG = 1;
  while (CG * 4 < twp) CG <<= 1;
  const int RG = 16 / MR;
  const int KG = 32 / (CG * RG);
  const int cgi = l % CG, rg = (l / CG) % RG, kg = l / (CG * RG);
  const bool colok = cgi * 4 < twp;
  const int col = cgi * 4;
  const int rbase = w * 16 + rg;  // rows rbase + RG * i, i < MR
  CT acc[MR][4];
#pragma unroll
  for (int i = 0; i < MR; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = CT(0);
  for (int ci = 0; ci < nch; ++ci) {
    const unsigned g = gctr + ci;
    const int s = (int)(g % a.slots);
    const unsigned u = g / a.slots;
    if (ok && !mbar_wait(full + s, u & 1u, a.timeout_cycles)) {
      ok = false;
      if (l == 0) set_error(a.err, DEV_TIMEOUT);
    }
    if (ok && colok) {
      const GT* gt = reinterpret_cast<const GT*>(ring + (size_t)s * slot);
      const CT* xs = reinterpret_cast<const CT*>(ring + (size_t)s * slot + a.tps * gtile) + col;
      const int nq = min(a.tps, nkc - ci * a.tps) * (kKC / 4);
#pragma unroll 2
      for (int q = kg; q < nq; q += KG) {
        CT xv[4][4], gv[MR][4];
        const GT* gq = gt + (size_t)(q >> 3) * kRT * kKC;  // tile of quad q
#pragma unroll
        for (int j = 0; j < 4; ++j) load4<CT, CT>(xs + (size_t)(4 * q + j) * twp, xv[j]);
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          const int r = rbase + RG * i;
          load4<CT, GT>(gq + (size_t)r * kKC + 4 * ((q & 7) ^ (r & 7)), gv[i]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) acc[i][qq] = fma(gv[i][j], xv[j][qq], acc[i][qq]);
      }
    }
    __syncwarp();
    if (l == 0) mbar_arrive(empty + s);
  }
  gctr += nch;
  for (int o = CG * RG; o < 32; o <<= 1) {
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) acc[i][qq] += __shfl_xor_sync(0xffffffffu, acc[i][qq], o);
  }
  if (colok && kg == 0) {
#pragma unroll
    for (int i = 0; i < MR; ++i) {
      const int r = rbase + RG * i;
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) P[(size_t)r * twp + col + qq] = acc[i][qq];
    }
  }
  return ok;
}

// Wide form of tile_product for FP32 compute and twp in {8, 16, 32, 64}, with X
// k-pair interleaved (see xoff): lane (cg, rg) holds 8 rows (rbase + RG i) x 4
// trials (4 cg ..) as 64-bit accumulators of the even-k and odd-k sums, fed by
// packed FMAs of a G_off pair and an X pair; CG = twp / 4, RG = 32 / CG, a
// quarter-warp covers 8 / cq rows x cq column groups (cq = min(CG, 4)).  The
// consumer warps form WR = 16 / RG row-warps (RG x 8 rows each, 128 in all) x
// WK = RG / 2 k-warps; k-warp kw takes every WK-th quad of each 32-column tile
// and writes its partials to plane kw of P ([WK][kRT][twp]); the caller sums
// the planes.
template <typename GT>
__device__ __forceinline__ bool tile_product_pair(const BArgs<float>& a, const BInst<float>& I,
                                                  const float* __restrict__ X, int rt, unsigned char* ring,
                                                  size_t slot, float* P, uint64_t* full, uint64_t* empty,
                                                  unsigned& gctr, unsigned* issued) {
  constexpr int MR = 8;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int twp = a.twp, nkc = I.nkc;
  const size_t gtile = (size_t)kRT * kKC * sizeof(GT);
  const int nch = (nkc + a.tps - 1) / a.tps;
  bool ok = true;
  if (w == kBWarps) {
    if (l == 0) produce_row_tile<GT, float>(a, I, X, rt, ring, slot, full, empty, gctr, issued, 0, nch);
    gctr += nch;
    return true;
  }
  const int CG = twp >> 2, RG = 32 / CG;
  const int WR = 16 / RG, WK = kBWarps / WR;
  const int wr = w % WR, kw = w / WR;
  const int cq = CG < 4 ? CG : 4, qd = l >> 3, li = l & 7;
  const int cg = (qd % (CG / cq)) * cq + li % cq, rg = (qd / (CG / cq)) * (8 / cq) + li / cq;
  const int rbase = wr * RG * MR + rg;
  const int c = 4 * cg;
  uint64_t acc[MR][4];
#pragma unroll
  for (int i = 0; i < MR; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0ull;
  for (int ci = 0; ci < nch; ++ci) {
    const unsigned g = gctr + ci;
    const int s = (int)(g % a.slots);
    const unsigned u = g / a.slots;
    if (ok && !mbar_wait(full + s, u & 1u, a.timeout_cycles)) {
      ok = false;
      if (l == 0) set_error(a.err, DEV_TIMEOUT);
    }
    if (ok) {
      const GT* gt = reinterpret_cast<const GT*>(ring + (size_t)s * slot);
      const float* xs = reinterpret_cast<const float*>(ring + (size_t)s * slot + a.tps * gtile) + 2 * c;
      const int nq = min(a.tps, nkc - ci * a.tps) * (kKC / 4);
#pragma unroll 1
      for (int q = kw; q < nq; q += WK) {
        ulonglong2 gp[MR];
        const GT* gq = gt + (size_t)(q >> 3) * kRT * kKC;  // tile of quad q
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          const int r = rbase + RG * i;
          gp[i] = load_gpairs<GT>(gq + (size_t)r * kKC + 4 * ((q & 7) ^ (r & 7)));
        }
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
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
  float* dst = P + (size_t)kw * kRT * twp;
#pragma unroll
  for (int i = 0; i < MR; ++i) {
    const int r = rbase + RG * i;
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 h = unpack2(acc[i][q]);
      v[q] = h.x + h.y;
    }
    *reinterpret_cast<float4*>(dst + (size_t)r * twp + c) = make_float4(v[0], v[1], v[2], v[3]);
  }
  return ok;
}

// Tensor-core form of one row tile (BF16 / FP16 G_off, FP32 compute, twp = 8 NT
// trials): the ring slots hold G_off in A-operand order and X in two 16-bit
// parts ([k / 16][part][t][k % 16], scaled by xsc); warp w takes rows 16 w ..
// 16 w + 15 of the row tile for every trial and every k, two MMAs per
// 16 x 8 x 16 tile (hi and lo of X).  The MMAs of one ring slot chain in
// accumulators that start from zero and are then added to the FP32 sums
// (round to nearest).  P (kRT x twp) receives U, scaled back by xsi.  The
// producer issues the CTA's next row tile's (rt + rstep) first chunks before
// the CTA-wide sync that ends this product (pre counts them; every row tile of
// a pass reads the same X, so only the CTA's last row tile of a pass issues
// none).
template <typename GT, int NT>
__device__ __forceinline__ bool tile_product_tc(const BArgs<float>& a, const BInst<float>& I,
                                                const float* __restrict__ X, int rt, int rstep, unsigned char* ring,
                                                size_t slot, float* P, uint64_t* full, uint64_t* empty,
                                                unsigned& gctr, unsigned* issued, float xsi, int& pre) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int twp = a.twp, nkc = I.nkc;
  const size_t gtile = (size_t)kRT * kKC * sizeof(GT);
  const int nch = (nkc + a.tps - 1) / a.tps;
  bool ok = true;
  if (w == kBWarps) {
    if (l == 0) {
      // the chunks not issued ahead, then the first ring-full of the next row
      // tile of this pass (same X), whose copies then land during the update
      produce_row_tile<GT, float>(a, I, X, rt, ring, slot, full, empty, gctr, issued, pre, nch);
      pre = 0;
      if (rt + rstep < I.nrt) {
        pre = min(a.slots, nch);
        produce_row_tile<GT, float>(a, I, X, rt + rstep, ring, slot, full, empty, gctr + nch, issued, 0, pre);
      }
    }
    gctr += nch;
    return true;
  }
  constexpr int kTileU4 = kRT * kKC * 2 / 16;  // 16-byte words per column tile
  float acc[NT][2][4];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[nt][p][q] = 0.f;
  for (int ci = 0; ci < nch; ++ci) {
    const unsigned g = gctr + ci;
    const int s = (int)(g % a.slots);
    const unsigned u = g / a.slots;
    if (ok && !mbar_wait(full + s, u & 1u, a.timeout_cycles)) {
      ok = false;
      if (l == 0) set_error(a.err, DEV_TIMEOUT);
    }
    if (ok) {
      const uint4* gt = reinterpret_cast<const uint4*>(ring + (size_t)s * slot) + w * 64 + l;
      const uint2* xs = reinterpret_cast<const uint2*>(ring + (size_t)s * slot + a.tps * gtile) + l;
      const int nkb = min(a.tps, nkc - ci * a.tps) * (kKC / 16);
      float d[NT][2][4];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) d[nt][p][q] = 0.f;
#pragma unroll 1
      for (int kb = 0; kb < nkb; ++kb) {
        // column tile kb / 2 of the slot, k half kb % 2, row tile w
        const uint4 av = gt[(size_t)(kb >> 1) * kTileU4 + (kb & 1) * 32];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          mma16816<GT>(d[nt][0], av, xs[((size_t)(2 * kb) * twp + nt * 8) * 4]);
          mma16816<GT>(d[nt][1], av, xs[((size_t)(2 * kb + 1) * twp + nt * 8) * 4]);
        }
      }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[nt][p][q] += d[nt][p][q];
    }
    __syncwarp();
    if (l == 0) mbar_arrive(empty + s);
  }
  gctr += nch;
  const float wlo = 1.0f / (float)(1 << tc_type<GT>::kLoShift);
  const int r = w * 16 + (l >> 2), c = 2 * (l & 3);
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const float* h = acc[nt][0];
    const float* o = acc[nt][1];
    *reinterpret_cast<float2*>(P + (size_t)r * twp + nt * 8 + c) =
        make_float2(fmaf(wlo, o[0], h[0]) * xsi, fmaf(wlo, o[1], h[1]) * xsi);
    *reinterpret_cast<float2*>(P + (size_t)(r + 8) * twp + nt * 8 + c) =
        make_float2(fmaf(wlo, o[2], h[2]) * xsi, fmaf(wlo, o[3], h[3]) * xsi);
  }
  return ok;
}

// Store X[k][t] = v in the layout of the launch's product form; the
// tensor-core form stores two 16-bit parts (X scaled so that |X| <= |c|).
// X of the tcgen05 form: 16-k blocks of NN = 2 twp operand rows (trial t's
// high part is row t, its low part row twp + t), each block in the canonical
// layout (tcgen05.cuh); element index of (k, row n).
__host__ __device__ __forceinline__ size_t tc5_xidx(int k, int n, int NN) {
  return (size_t)(k >> 4) * (size_t)(NN * 16) + tc5::canon_off(n, k & 15) / 2;
}

template <typename GT, typename CT, bool PAIR, bool TC, bool TC5 = false>
__device__ __forceinline__ void bxput(CT* X, int k, int t, int twp, CT v) {
  if constexpr (TC5) {
    GT* h = reinterpret_cast<GT*>(X);
    const GT hi = GT(v);
    const float hf = float(hi);
    h[tc5_xidx(k, t, 2 * twp)] = hi;
    h[tc5_xidx(k, twp + t, 2 * twp)] = GT((v - hf) * (float)(1 << tc_type<GT>::kLoShift));
  } else if constexpr (TC) {
    GT* h = reinterpret_cast<GT*>(X);
    const GT hi = GT(v);
    const float hf = float(hi);
    h[tc_xidx(k, t, twp, 0)] = hi;
    h[tc_xidx(k, t, twp, 1)] = GT((v - hf) * (float)(1 << tc_type<GT>::kLoShift));
  } else {
    X[xoff<PAIR>(k, t, twp)] = v;
  }
}

// U of row rl (tile-local) and trial t: the partials of the row tile, summed
// over the k-warp planes of the wide form (one plane otherwise).
template <typename CT, bool PAIR>
__device__ __forceinline__ CT tile_sum(const CT* P, int rl, int t, int twp) {
  if constexpr (PAIR) {
    const int WK = (32 / (twp >> 2)) / 2;
    CT v = P[(size_t)rl * twp + t];
    for (int kw = 1; kw < WK; ++kw) v += P[(size_t)kw * kRT * twp + (size_t)rl * twp + t];
    return v;
  } else {
    return P[(size_t)rl * twp + t];
  }
}

// Product of one row tile in the form the launch was built for.
template <typename GT, typename CT, int MR, bool PAIR, bool TC>
__device__ __forceinline__ bool row_tile_product(const BArgs<CT>& a, const BInst<CT>& I, const CT* __restrict__ X,
                                                 int rt, int rstep, unsigned char* ring, size_t slot, CT* P,
                                                 uint64_t* full, uint64_t* empty, unsigned& gctr, unsigned* issued,
                                                 float xsi, int& pre) {
  if constexpr (TC) {
    return tile_product_tc<GT, MR>(a, I, X, rt, rstep, ring, slot, P, full, empty, gctr, issued, xsi, pre);
  } else if constexpr (PAIR) {
    return tile_product_pair<GT>(a, I, X, rt, ring, slot, P, full, empty, gctr, issued);
  } else {
    return tile_product<GT, CT, MR>(a, I, X, rt, ring, slot, P, full, empty, gctr, issued);
  }
}

__device__ __forceinline__ size_t zmin(size_t x, size_t y) { return x < y ? x : y; }

// 8 consecutive floats (32-byte aligned) into registers.
__device__ __forceinline__ void load8(const float* p, float (&v)[8]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// tcgen05 form of the batched product (BF16 / FP16 G_off, 8 or 16 trials): the
// product of a row tile is one M = 128, N = NN = 2 twp MMA per 16-k block (A =
// the row tile's G_off block, B = the two 16-bit parts of the block's X rows),
// issued by one thread, lane 0 of the producer warp, which also issues the
// ring's bulk copies.  The 16-k blocks of a row tile rotate over four FP32
// accumulators (limiting how many truncating accumulations any one sum
// takes), summed with round-to-nearest additions in the epilogue.  Two sets of
// accumulators (buf = row-tile count & 1) let the consumer warps read and
// apply one row tile's U while the MMAs of the next run.  Barriers: accfull[b]
// (one arrival: the tcgen05 commit after a row tile's last MMA), accfree[b]
// (the 8 consumer warps, after reading buffer b), fin (the final commit).
struct Tc5 {
  uint64_t* accfull;
  uint64_t* accfree;
  uint64_t* fin;
  uint32_t tmem;    // TMEM base address
  uint32_t idesc;   // instruction descriptor (M = 128, N = NN)
  int NN;           // 2 twp
  unsigned jt = 0;  // producer: row tiles issued
  unsigned jc = 0;  // consumers: row tiles read
};

// Producer lane 0: the copies and MMAs of row tile rt (X = this pass's X), then
// the first ring-full of copies of the CTA's next row tile of the pass.
// Returns false after a timed-out wait.
template <typename GT>
__device__ __forceinline__ bool tc5_row_tile(const BArgs<float>& a, const BInst<float>& I, const float* __restrict__ X, int rt,
                             int rstep, unsigned char* ring, size_t slot, uint64_t* full, uint64_t* empty,
                             unsigned& gctr, unsigned* issued, int& pre, Tc5& t5) {
  const int nkc = I.nkc, nch = (nkc + a.tps - 1) / a.tps;
  const uint32_t gtile = (uint32_t)(kRT * kKC * sizeof(GT));
  const uint32_t xblk = (uint32_t)t5.NN * 32;  // bytes of one 16-k block of X
  const int b = (int)(t5.jt & 1u);
  const unsigned u = t5.jt >> 1;
  ++t5.jt;
  if (u >= 1 && !mbar_wait(t5.accfree + b, (u - 1) & 1u, a.timeout_cycles)) {
    set_error(a.err, DEV_TIMEOUT);
    return false;
  }
  tc5::fence_after_sync();
  const uint32_t acc0 = t5.tmem + (uint32_t)(b * 4 * t5.NN);
  const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
  int next = pre;  // chunks of this row tile whose copies are issued
  if (!produce_row_tile<GT, float>(a, I, X, rt, ring, slot, full, empty, gctr, issued, next, min(nch, a.slots)))
    return false;
  next = max(next, min(nch, a.slots));
  int kb = 0;
  for (int ci = 0; ci < nch; ++ci) {
    const unsigned g = gctr + ci;
    const int s = (int)(g % a.slots);
    if (!mbar_wait(full + s, (g / a.slots) & 1u, a.timeout_cycles)) {
      set_error(a.err, DEV_TIMEOUT);
      return false;
    }
    tc5::fence_after_sync();
    const int nt = min(a.tps, nkc - ci * a.tps);
    const uint32_t sb = ring_s + (uint32_t)(s * slot);
    for (int j = 0; j < nt; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h, ++kb) {
        const uint64_t ad = tc5::smem_desc(sb + j * gtile + h * 4096u, tc5::kLBO, tc5::kSBO);
        const uint64_t bd = tc5::smem_desc(sb + a.tps * gtile + (2 * j + h) * xblk, tc5::kLBO, tc5::kSBO);
        tc5::mma_f16(acc0 + (uint32_t)((kb & 3) * t5.NN), ad, bd, t5.idesc, kb >= 4 ? 1u : 0u);
      }
    tc5::commit(empty + s);  // the slot is free once these MMAs have read it
    // copies ahead: up to chunk ci + slots - 1 (its slot was read by chunk ci - 1)
    const int upto = min(nch, ci + a.slots);
    if (next < upto) {
      if (!produce_row_tile<GT, float>(a, I, X, rt, ring, slot, full, empty, gctr, issued, next, upto)) return false;
      next = upto;
    }
  }
  tc5::commit(t5.accfull + b);
  gctr += nch;
  pre = 0;
  if (rt + rstep < I.nrt) {
    const int nn = min(a.slots, nch);
    if (!produce_row_tile<GT, float>(a, I, X, rt + rstep, ring, slot, full, empty, gctr, issued, 0, nn)) return false;
    pre = nn;
  }
  return true;
}

// Consumer warps: U of this thread's row (32 (warp % 4) + lane of row tile rt)
// and trials 8 (warp / 4) .. + 7 from the row tile's accumulators (the warps
// with no trials there read nothing), then release the accumulators.  Returns
// false after a timed-out wait.
template <typename GT>
__device__ __forceinline__ bool tc5_read(const BArgs<float>& a, const BInst<float>& I, Tc5& t5, float xsi, float (&U)[8]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = (int)(t5.jc & 1u);
  const unsigned u = t5.jc >> 1;
  ++t5.jc;
  // (warp-uniform decision: the TMEM loads below are warp-collective)
  if (!__all_sync(0xffffffffu, mbar_wait(t5.accfull + b, u & 1u, a.timeout_cycles))) {
    if (lane == 0) set_error(a.err, DEV_TIMEOUT);
    return false;
  }
  tc5::fence_after_sync();
  const int hh = w >> 2;
  if (hh * 8 < a.twp) {
    const uint32_t base = tc5::taddr(t5.tmem, 32 * (w & 3), b * 4 * t5.NN + hh * 8);
    float hi[8], lo[8];
    const int nacc = min(4, 2 * I.nkc);
    if (nacc == 4) {
      tc5::ld8x4_sum(base, (uint32_t)t5.NN, hi);
      tc5::ld8x4_sum(base + (uint32_t)a.twp, (uint32_t)t5.NN, lo);
    } else {
      tc5::ld8(base, hi);
      tc5::ld8(base + (uint32_t)a.twp, lo);
      for (int k = 1; k < nacc; ++k) {
        float h2[8], l2[8];
        tc5::ld8(base + (uint32_t)(k * t5.NN), h2);
        tc5::ld8(base + (uint32_t)(k * t5.NN + a.twp), l2);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          hi[i] += h2[i];
          lo[i] += l2[i];
        }
      }
    }
    const float wlo = 1.0f / (float)(1 << tc_type<GT>::kLoShift);
#pragma unroll
    for (int i = 0; i < 8; ++i) U[i] = fmaf(wlo, lo[i], hi[i]) * xsi;
  }
  tc5::fence_before_sync();
  __syncwarp();
  if (lane == 0) mbar_arrive(t5.accfree + b);
  return true;
}

// End of a phase of a run: X (and the state) written by every CTA of the run
// become visible to the next phase's bulk copies.  A run of `span` CTAs (a
// whole cluster) meets at the cluster barrier, where each CTA also posts its
// `ok` (CTA-uniform) in vote[vpar] and then reads every CTA's: every CTA of the
// cluster returns the same decision, so all of them take the same number of
// cluster barriers.  (vote has two entries, used in turn: an entry is rewritten
// only two barriers later, after every CTA has read it.)  `ok` may differ
// between the threads of a CTA; the CTA's is their AND.
__device__ __forceinline__ bool run_sync(int span, bool ok, int* vote, unsigned& vpar) {
  fence_proxy_async_global();
  ok = __syncthreads_and(ok);
  if (span == 1) return ok;
  cg::cluster_group cl = cg::this_cluster();
  if (threadIdx.x == 0) vote[vpar] = ok ? 1 : 0;
  cl.sync();
  int all = 1;
  for (int r = 0; r < span; ++r) all &= *cl.map_shared_rank(vote + vpar, r);
  vpar ^= 1u;
  return all != 0;
}

// One CIM run of problem I by `span` CTAs (rank `rank` of them takes row tiles
// rank, rank + span, ...).  Returns false (in every thread of every CTA of the
// run) if a wait timed out.
template <typename GT, typename CT, int MR, bool PAIR, bool TC, bool TC5>
__device__ bool run_instance(const BArgs<CT>& a, const BInst<CT>& I, int rank, int span, unsigned char* ring,
                             size_t slot, CT* P, uint64_t* full, uint64_t* empty, unsigned& gctr, unsigned* issued,
                             int* vote, unsigned& vpar, Tc5& t5) {
  const int T = a.T, twp = a.twp, N = I.N;
  const size_t NT = (size_t)N * T;
  const size_t tileT = (size_t)kRT * T;  // elements of one row tile
  const int steps = a.step_cap > 0 ? min(I.n_steps, a.step_cap) : I.n_steps;
  int pre = 0;  // producer: chunks of the next row tile already issued
  // tensor-core form: X scaled by 2^-e with max |R| < 2^e (exact; U scaled back)
  CT xsc = CT(1);
  float xsi = 1.f;
  if constexpr (TC || TC5) {
    double m = 0.0;
    for (size_t o = threadIdx.x; o < NT; o += kBThreads) m = fmax(m, fabs(I.R[o]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    double* red = reinterpret_cast<double*>(P);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    for (int i = 0; i < kBThreads / 32; ++i) m = fmax(m, red[i]);
    __syncthreads();
    int ex = 0;
    if (m > 0.0 && m <= 1e30) frexp(m, &ex);
    ex = max(-100, min(100, ex));
    xsc = CT(ldexp(1.0, -ex));
    xsi = (float)ldexp(1.0, ex);
  }
  CT* c = I.state;
  CT* e = I.state + NT;
  CT* b = I.state + 2 * NT;
  const double st = sqrt(I.tau);
  const CT wcoef = (I.field == CS_FIELD_CN) ? CT(-0.25) : CT(-0.5 * st);
  bool ok = true;
  // ---- prologue
  // (the elements of this CTA's rows: row tiles rank, rank + span, ...)
  if (I.field == CS_FIELD_CN) {
    for (int rt = rank; rt < I.nrt; rt += span)
      for (size_t idx = rt * tileT + threadIdx.x; idx < zmin(NT, (rt + 1) * tileT); idx += kBThreads) {
        const int r = (int)(idx / T), t = (int)(idx % T);
        bxput<GT, CT, PAIR, TC, TC5>(I.X0, r, t, twp, CT(I.R[idx]) * xsc);
      }
    ok = run_sync(span, ok, vote, vpar);
    if constexpr (TC5) {
      // b of this CTA's rows from U = G_off X0 (producer lane 0: copies and MMAs;
      // consumer warps: U from TMEM, then b)
      const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
      bool okt = ok;
      if (w == kBWarps) {
        if (lane == 0)
          for (int rt = rank; rt < I.nrt && okt; rt += span)
            okt = tc5_row_tile<GT>(a, I, I.X0, rt, span, ring, slot, full, empty, gctr, issued, pre, t5);
      } else {
        for (int rt = rank; rt < I.nrt && okt; rt += span) {
          float U[8];
          okt = tc5_read<GT>(a, I, t5, xsi, U);
          const int hh = w >> 2, r = rt * kRT + 32 * (w & 3) + lane;
          if (okt && hh * 8 < T && r < N)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const size_t o = (size_t)r * T + hh * 8 + i;
              const double v = (double)U[i];
              const double corr = I.self_term ? (st / 4.0) * I.g[r] * I.R[o] * I.R[o] : 0.0;
              b[o] = CT(I.R[o] * (-(st / 4.0) * v + (st / 2.0) * I.hz[r]) - I.theta - corr);
            }
        }
      }
      ok = __syncthreads_and(okt);
    }
    for (int rt = rank; rt < I.nrt && ok && !TC5; rt += span) {
      ok = __syncthreads_and(row_tile_product<GT, CT, MR, PAIR, TC>(a, I, I.X0, rt, span, ring, slot, P, full, empty,
                                                                    gctr, issued, xsi, pre));
      for (int idx = threadIdx.x; idx < kRT * T; idx += kBThreads) {
        const int r = rt * kRT + idx / T, t = idx % T;
        if (r >= N) continue;
        const double v = (double)(tile_sum<CT, PAIR>(P, idx / T, t, twp) * row_scale<GT, CT>(I.gscale, r));
        const size_t o = (size_t)r * T + t;
        const double corr = I.self_term ? (st / 4.0) * I.g[r] * I.R[o] * I.R[o] : 0.0;
        b[o] = CT(I.R[o] * (-(st / 4.0) * v + (st / 2.0) * I.hz[r]) - I.theta - corr);
      }
      __syncthreads();
    }
  } else {
    for (int rt = rank; rt < I.nrt; rt += span)
      for (size_t o = rt * tileT + threadIdx.x; o < zmin(NT, (rt + 1) * tileT); o += kBThreads) {
        const int r = (int)(o / T);
        const double corr = I.self_term ? (st / 4.0) * I.g[r] * I.R[o] * I.R[o] : 0.0;
        b[o] = CT((st / 2.0) * I.R[o] * I.hz[r] - I.theta - corr);
      }
  }
  for (int rt = rank; rt < I.nrt; rt += span)
    for (size_t o = rt * tileT + threadIdx.x; o < zmin(NT, (rt + 1) * tileT); o += kBThreads) {
      const int r = (int)(o / T), t = (int)(o % T);
      const uint64_t key = run_key(I.seed, (uint64_t)I.inst, (uint64_t)t, (uint64_t)a.outer);
      const CT c0 = CT(initial_amplitude(key, (uint64_t)r, I.init_kind, I.init_scale));
      c[o] = c0;
      e[o] = CT(1);
      const CT Rr = CT(I.R[o]);
      bxput<GT, CT, PAIR, TC, TC5>(I.X1, r, t, twp,
                              ((I.field == CS_FIELD_CN) ? Rr * c0 : (c0 > CT(0) ? Rr : CT(0))) * xsc);
    }
  ok = run_sync(span, ok, vote, vpar);
  // ---- Euler steps
  const CT dt = CT(I.dt), beta = CT(I.beta), tau = CT(I.tau), Kj = CT(I.Kj);
  CT* Xc = I.X1;
  CT* Xn = I.X0;
  for (int n = 0; n < steps && ok; ++n) {
    const CT p = pump_at<CT>(n, I.n_steps, I.pump_kind, I.p0, I.p1, I.p_thr, I.d, I.dt, I.t0, I.width);
    const bool last = (n + 1 == steps);
    if constexpr (TC5) {
      // producer lane 0 streams and multiplies every row tile of the CTA; the
      // consumer warps apply each row tile's U as soon as its accumulators are
      // complete (no CTA-wide barrier until the end of the step)
      const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
      bool okt = true;
      if (w == kBWarps) {
        if (lane == 0)
          for (int rt = rank; rt < I.nrt && okt; rt += span)
            okt = tc5_row_tile<GT>(a, I, Xc, rt, span, ring, slot, full, empty, gctr, issued, pre, t5);
      } else {
        const int hh = w >> 2;
        for (int rt = rank; rt < I.nrt && okt; rt += span) {
          const int r = rt * kRT + 32 * (w & 3) + lane;
          const bool act = hh * 8 < T && r < N;
          const size_t o = (size_t)r * T + hh * 8;
          // this thread's 8 elements of the state, loaded before the wait
          float cf[8], ef[8], bf[8];
          double Rf[8];
          if (act) {
            load8(c + o, cf);
            load8(e + o, ef);
            load8(b + o, bf);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const double2 v = *reinterpret_cast<const double2*>(I.R + o + 2 * j);
              Rf[2 * j] = v.x;
              Rf[2 * j + 1] = v.y;
            }
          }
          float U[8];
          okt = tc5_read<GT>(a, I, t5, xsi, U);
          if (okt && act) {
            float cn8[8], en8[8];
            uint64_t sg = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const CT Rr = CT(Rf[i]), cc = cf[i], ee = ef[i];
              const CT f = wcoef * Rr * U[i] + bf[i];
              const CT c2 = cc * cc;
              const CT cn = cc + dt * ((CT(-1) + p - c2) * cc + Kj * ee * f);
              const CT en = ee + dt * (-beta * (c2 - tau) * ee);
              cn8[i] = cn;
              en8[i] = en;
              bxput<GT, CT, PAIR, TC, TC5>(Xn, r, hh * 8 + i, twp,
                                           ((I.field == CS_FIELD_CN) ? Rr * cn : (cn > CT(0) ? Rr : CT(0))) * xsc);
              sg |= (uint64_t)(cn > CT(0) ? 1 : 0) << (8 * i);
            }
            *reinterpret_cast<float4*>(c + o) = make_float4(cn8[0], cn8[1], cn8[2], cn8[3]);
            *reinterpret_cast<float4*>(c + o + 4) = make_float4(cn8[4], cn8[5], cn8[6], cn8[7]);
            *reinterpret_cast<float4*>(e + o) = make_float4(en8[0], en8[1], en8[2], en8[3]);
            *reinterpret_cast<float4*>(e + o + 4) = make_float4(en8[4], en8[5], en8[6], en8[7]);
            if (last) *reinterpret_cast<uint64_t*>(I.sigma + o) = sg;
          }
        }
      }
      ok = run_sync(span, okt, vote, vpar);
      CT* tmp = Xc; Xc = Xn; Xn = tmp;
      continue;
    }
    for (int rt = rank; rt < I.nrt && ok; rt += span) {
      constexpr int kU = 8;
      const int ne = kRT * T;
      if constexpr (TC) {
        // Tensor-core form (T <= 16, so the kRT T elements of a row tile are at
        // most kU per consumer thread): each consumer thread loads the state of
        // its kU elements of the row tile
        // before the product and updates them after it, so the loads' latency
        // (the state is in global memory) is hidden behind the product
        // (measured on GB300: the update had been 45% of the kernel's time).
        constexpr int kUT = kBWarps * 32;
        const int tid = threadIdx.x;
        CT cv[kU], ev[kU], bv[kU];
        double Rd[kU];
        if (tid < kUT) {
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int idx = u * kUT + tid;
            const int r = rt * kRT + idx / T;
            cv[u] = ev[u] = bv[u] = CT(0);
            Rd[u] = 0.0;
            if (idx < ne && r < N) {
              const size_t o = (size_t)r * T + idx % T;
              cv[u] = c[o];
              ev[u] = e[o];
              bv[u] = b[o];
              Rd[u] = I.R[o];
            }
          }
        }
        ok = __syncthreads_and(row_tile_product<GT, CT, MR, PAIR, TC>(a, I, Xc, rt, span, ring, slot, P, full,
                                                                      empty, gctr, issued, xsi, pre));
        if (tid < kUT) {
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int idx = u * kUT + tid;
            const int rl = idx / T, t = idx % T, r = rt * kRT + rl;
            if (idx < ne && r < N) {
              const size_t o = (size_t)r * T + t;
              const CT Rr = CT(Rd[u]), cc = cv[u], ee = ev[u];
              const CT f = wcoef * Rr * tile_sum<CT, PAIR>(P, rl, t, twp) + bv[u];
              const CT c2 = cc * cc;
              const CT cn = cc + dt * ((CT(-1) + p - c2) * cc + Kj * ee * f);
              const CT en = ee + dt * (-beta * (c2 - tau) * ee);
              c[o] = cn;
              e[o] = en;
              bxput<GT, CT, PAIR, TC, TC5>(Xn, r, t, twp,
                                      ((I.field == CS_FIELD_CN) ? Rr * cn : (cn > CT(0) ? Rr : CT(0))) * xsc);
              if (last) I.sigma[o] = cn > CT(0) ? 1 : 0;
            }
          }
        }
        __syncthreads();
        continue;
      }
      ok = __syncthreads_and(row_tile_product<GT, CT, MR, PAIR, TC>(a, I, Xc, rt, span, ring, slot, P, full, empty,
                                                                    gctr, issued, xsi, pre));
      // the row tile's update, kU elements per thread at a time: every load of
      // the state (global memory, L2-resident) is issued before the first
      // update, so the L2 latency is paid once per kU elements (measured on
      // GB300: 9% less time per batch than one element at a time)
      for (int base = 0; base < ne; base += kU * kBThreads) {
        CT cv[kU], ev[kU], bv[kU], Rv[kU], Uv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int idx = base + u * kBThreads + threadIdx.x;
          const int rl = idx / T, t = idx % T, r = rt * kRT + rl;
          cv[u] = ev[u] = bv[u] = Rv[u] = Uv[u] = CT(0);
          if (idx < ne && r < N) {
            const size_t o = (size_t)r * T + t;
            cv[u] = c[o];
            ev[u] = e[o];
            bv[u] = b[o];
            Rv[u] = CT(I.R[o]);
            Uv[u] = tile_sum<CT, PAIR>(P, rl, t, twp) * row_scale<GT, CT>(I.gscale, r);
          }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int idx = base + u * kBThreads + threadIdx.x;
          const int rl = idx / T, t = idx % T, r = rt * kRT + rl;
          if (idx < ne && r < N) {
            const size_t o = (size_t)r * T + t;
            const CT Rr = Rv[u], cc = cv[u], ee = ev[u];
            const CT f = wcoef * Rr * Uv[u] + bv[u];
            const CT c2 = cc * cc;
            const CT cn = cc + dt * ((CT(-1) + p - c2) * cc + Kj * ee * f);
            const CT en = ee + dt * (-beta * (c2 - tau) * ee);
            c[o] = cn;
            e[o] = en;
            bxput<GT, CT, PAIR, TC, TC5>(Xn, r, t, twp,
                                    ((I.field == CS_FIELD_CN) ? Rr * cn : (cn > CT(0) ? Rr : CT(0))) * xsc);
            if (last) I.sigma[o] = cn > CT(0) ? 1 : 0;
          }
        }
      }
      __syncthreads();
    }
    ok = run_sync(span, ok, vote, vpar);
    CT* tmp = Xc; Xc = Xn; Xn = tmp;
  }
  return ok;
}

template <typename GT, typename CT, int MR, bool PAIR, bool TC, bool TC5>
__global__ void __launch_bounds__(kBThreads, 1) euler_batch_kernel(BArgs<CT> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const size_t slot = b_slot_bytes(a.twp, sizeof(GT), sizeof(CT), a.tps);
  unsigned char* ring = smem_raw;
  CT* P = reinterpret_cast<CT*>(smem_raw + (size_t)a.slots * slot);
  uint64_t* full =
      reinterpret_cast<uint64_t*>(smem_raw + (size_t)a.slots * slot + b_part_bytes(a.twp, sizeof(CT), PAIR));
  uint64_t* empty = full + a.slots;
  __shared__ int s_next;   // this CTA's own pops
  __shared__ int s_bcast;  // rank 0: the cluster's pops (read by every CTA of the cluster)
  __shared__ int s_vote[2];
  // tcgen05 form: accumulator barriers and the TMEM address
  __shared__ uint64_t s_acc[5];
  __shared__ uint32_t s_tmem;
  Tc5 t5;
  t5.accfull = s_acc;
  t5.accfree = s_acc + 2;
  t5.fin = s_acc + 4;
  t5.NN = 2 * a.twp;
  t5.idesc = std::is_same<GT, __nv_bfloat16>::value ? tc5::idesc_bf16_f32(128, t5.NN) : tc5::idesc_f16_f32(128, t5.NN);
  // four accumulators of NN columns in each of two sets (a power of two >= 32)
  const uint32_t tcols = t5.NN * 8 <= 32 ? 32u : (uint32_t)(t5.NN * 8);
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.slots; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, TC5 ? 1 : kBWarps);  // tcgen05: the commit after the slot's MMAs
    }
    if (TC5) {
      mbar_init(t5.accfull, 1);
      mbar_init(t5.accfull + 1, 1);
      mbar_init(t5.accfree, kBWarps);
      mbar_init(t5.accfree + 1, kBWarps);
      mbar_init(t5.fin, 1);
    }
    fence_mbar_init();
  }
  if (TC5 && threadIdx.x < 32) {
    tc5::tmem_alloc(&s_tmem, tcols);
    tc5::tmem_relinquish();
  }
  if (TC5) tc5::fence_before_sync();
  __syncthreads();
  if (TC5) {
    tc5::fence_after_sync();
    t5.tmem = s_tmem;
  }
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  unsigned gctr = 0;
  unsigned vpar = 0;
  unsigned issued[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // producer: 1 + last ring use issued per slot
  bool ok = true;
  // The large problems come first in the queue: while the cluster's pops return
  // large problems it runs them together; the first small one goes to rank 0,
  // and from then on every CTA pops and runs small problems alone.
  bool together = a.n_large > 0;
  while (ok) {
    int qi;
    if (together) {
      cl.sync();  // every CTA has read the previous pop
      if (rank == 0 && threadIdx.x == 0) s_bcast = ld_volatile(a.err) != 0 ? a.n : atomicAdd(a.queue, 1);
      cl.sync();
      qi = *cl.map_shared_rank(&s_bcast, 0);
      if (qi >= a.n) break;
      if (qi < a.n_large) {
        const BInst<CT> I = a.insts[a.order[qi]];
        ok = run_instance<GT, CT, MR, PAIR, TC, TC5>(a, I, rank, a.cc, ring, slot, P, full, empty, gctr, issued,
                                                     s_vote, vpar, t5);
        continue;
      }
      together = false;
      if (rank != 0) continue;  // pops its own next
    } else {
      if (threadIdx.x == 0) s_next = ld_volatile(a.err) != 0 ? a.n : atomicAdd(a.queue, 1);
      __syncthreads();
      qi = s_next;
      __syncthreads();
      if (qi >= a.n) break;
    }
    const BInst<CT> I = a.insts[a.order[qi]];
    ok = run_instance<GT, CT, MR, PAIR, TC, TC5>(a, I, 0, 1, ring, slot, P, full, empty, gctr, issued, s_vote, vpar,
                                                 t5);
  }
  // After a timeout, let any copy still in flight land before the CTA exits;
  // in the tcgen05 form, let every MMA issued complete, then free the TMEM.
  if (threadIdx.x == kBWarps * 32) {
    if (!ok)
      for (int s = 0; s < a.slots; ++s)
        if (issued[s] > 0) mbar_wait(full + s, (issued[s] - 1) / a.slots & 1u, a.timeout_cycles);
    if (TC5) {
      tc5::commit(t5.fin);
      mbar_wait(t5.fin, 0u, a.timeout_cycles);
    }
  }
  if (TC5) tc5::fence_before_sync();
  __syncthreads();
  if (TC5 && threadIdx.x < 32) {
    tc5::fence_after_sync();
    tc5::tmem_dealloc(t5.tmem, tcols);
  }
  // no CTA leaves while another of its cluster may still read its shared memory
  cl.sync();
}

// Ring shape of a launch: column tiles per slot (tps) and slots.  Unless the
// launch fixes them (L.tps, L.slots), the most column tiles (4, 2, 1) that
// still leave 3 slots (measured: one 32-column tile per slot leaves too little
// work between ring handoffs), and as many slots as fit (at most 8).
inline bool batch_ring(const BatchLaunch& L, int twp, size_t gbytes, size_t cbytes, size_t fixed, size_t cap,
                       int* tps_out, int* slots_out, size_t* smem_out) {
  auto need = [&](int tps, int slots) {
    return (size_t)slots * b_slot_bytes(twp, gbytes, cbytes, tps) + fixed + 2 * (size_t)slots * sizeof(uint64_t);
  };
  int tps = L.tps, slots = L.slots;
  if (tps == 0) {
    for (tps = 4; tps >= 1; tps >>= 1) {
      slots = 8;
      while (slots > 2 && need(tps, slots) > cap) --slots;
      if (slots >= 3 || tps == 1) break;
    }
    if (L.slots > 0) slots = L.slots;
  } else if (slots == 0) {
    slots = 8;
    while (slots > 2 && need(tps, slots) > cap) --slots;
  }
  if (tps != 1 && tps != 2 && tps != 4) return false;
  if (slots < 2 || slots > 8 || need(tps, slots) > cap) return false;
  *tps_out = tps;
  *slots_out = slots;
  *smem_out = need(tps, slots);
  return true;
}

template <typename GT, typename CT, int MR, bool PAIR, bool TC = false, bool TC5 = false>
cudaError_t launch_batch_typed(const BatchLaunch& L, cudaStream_t st) {
  const int twp = round4(L.T);
  auto fn = euler_batch_kernel<GT, CT, MR, PAIR, TC, TC5>;
  int optin = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  const size_t fixed = b_part_bytes(twp, sizeof(CT), PAIR);
  const size_t cap = (size_t)optin - fa.sharedSizeBytes;
  int tps = 0, slots = 0;
  size_t smem = 0;
  if (!batch_ring(L, twp, sizeof(GT), sizeof(CT), fixed, cap, &tps, &slots, &smem))
    return cudaErrorInvalidConfiguration;
  const int cc = L.cc > 0 ? L.cc : 1;
  if (cc != 1 && cc != 2 && cc != 4 && cc != 8) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  BArgs<CT> a;
  a.insts = reinterpret_cast<const BInst<CT>*>(L.insts);
  a.order = L.order;
  a.n = L.n;
  a.T = L.T;
  a.twp = twp;
  a.slots = slots;
  a.tps = tps;
  a.queue = L.queue;
  a.outer = L.outer;
  a.err = L.err;
  a.timeout_cycles = L.timeout_cycles;
  a.cc = cc;
  a.n_large = cc > 1 ? std::min(L.n_large, L.n) : 0;
  a.step_cap = L.step_cap;
  a.test_skip = L.test_skip;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kBThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // clusters: no more than are resident at once (the rest would only wait for
  // the queue to drain), nor than the queue has items for
  int resident = L.ctas;  // one CTA per SM
  if (cc > 1) {
    cfg.gridDim = dim3(cc);
    e = cudaOccupancyMaxActiveClusters(&resident, fn, &cfg);
    if (e != cudaSuccess) return e;
    if (resident < 1) return cudaErrorInvalidConfiguration;
  }
  const int items = a.n_large + (L.n - a.n_large + cc - 1) / cc;
  const int nclu = std::max(1, std::min({resident, std::max(1, L.ctas / cc), items}));
  cfg.gridDim = dim3(nclu * cc);
  e = cudaMemsetAsync(L.queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, fn, a);
}

template <typename GT, typename CT>
cudaError_t launch_batch_mr(const BatchLaunch& L, cudaStream_t st) {
  const int twp = round4(L.T);
  if constexpr (tc_type<GT>::value && std::is_same<CT, float>::value) {
    // the tensor-core forms (batch_tc_kind): tcgen05, or mma.sync with MR
    // carrying the n-tiles of 8 trials
    const int kind = batch_tc_kind(L.prm->precision, L.T, L.prm->tensor_form);
    if (kind == 2) {
      if (twp == 8) return launch_batch_typed<GT, CT, 1, false, false, true>(L, st);
      return launch_batch_typed<GT, CT, 2, false, false, true>(L, st);
    }
    if (kind == 1) {
      if (twp == 8) return launch_batch_typed<GT, CT, 1, false, true>(L, st);
      return launch_batch_typed<GT, CT, 2, false, true>(L, st);
    }
  }
  if constexpr (std::is_same<CT, float>::value) {
    // the wide form (packed FMAs) for trial blocks of 8, 16, 32 or 64
    if (twp == 8 || twp == 16 || twp == 32 || twp == 64) return launch_batch_typed<GT, CT, 8, true>(L, st);
  }
  int CG = 1;
  while (CG * 4 < twp) CG <<= 1;
  const int RG = std::min(16, 32 / CG);
  switch (16 / RG) {
    case 1: return launch_batch_typed<GT, CT, 1, false>(L, st);
    case 2: return launch_batch_typed<GT, CT, 2, false>(L, st);
    case 4: return launch_batch_typed<GT, CT, 4, false>(L, st);
    default: return launch_batch_typed<GT, CT, 8, false>(L, st);
  }
}

}  // namespace

int batch_row_tiles(int64_t N) { return (int)((N + kRT - 1) / kRT); }

size_t batch_inst_bytes() {
  return sizeof(BInst<double>) > sizeof(BInst<float>) ? sizeof(BInst<double>) : sizeof(BInst<float>);
}

int64_t tiled_elems(int64_t N, int64_t Npad) {
  const int64_t nrt = (N + kRT - 1) / kRT;
  return nrt * kRT * Npad;
}

int batch_tc_kind(int precision, int trials, int tensor_form) {
  if (tensor_form == 1 || !(precision == CS_P_BF16 || precision == CS_P_FP16) || !(trials == 8 || trials == 16))
    return 0;
  return tensor_form == 3 ? 1 : 2;
}

cudaError_t launch_store_tiled(ProblemDev& P, int precision, int frag) {
  if (P.gt_prec == precision && P.Gt && P.gt_frag == frag) return cudaSuccess;
  if (P.Gt) { dev_free(P.Gt, P.stream); P.Gt = nullptr; P.gt_prec = -1; }
  const size_t gb = storage_bytes(precision);
  const int64_t elems = tiled_elems(P.N, P.Npad);
  cudaError_t e = dev_alloc(&P.Gt, (size_t)elems * gb, P.stream);
  if (e != cudaSuccess) return e;
  const int N = (int)P.N, nrt = (int)((P.N + kRT - 1) / kRT), nkc = (int)(P.Npad / kKC);
  const int blocks = P.num_sms * 4;
  float* sc = P.gscale;
  switch (precision) {
    case CS_P_FP64: store_tiled_kernel<double><<<blocks, 256, 0, P.stream>>>(P.G, (double*)P.Gt, N, nrt, nkc, sc, 0); break;
    case CS_P_FP32: store_tiled_kernel<float><<<blocks, 256, 0, P.stream>>>(P.G, (float*)P.Gt, N, nrt, nkc, sc, 0); break;
    case CS_P_BF16:
      store_tiled_kernel<__nv_bfloat16><<<blocks, 256, 0, P.stream>>>(P.G, (__nv_bfloat16*)P.Gt, N, nrt, nkc, sc, frag);
      break;
    case CS_P_FP16:
      store_tiled_kernel<__half><<<blocks, 256, 0, P.stream>>>(P.G, (__half*)P.Gt, N, nrt, nkc, sc, frag);
      break;
    case CS_P_FP8:
      if ((e = ensure_row_scales(P)) != cudaSuccess) return e;
      store_tiled_kernel<__nv_fp8_e4m3><<<blocks, 256, 0, P.stream>>>(P.G, (__nv_fp8_e4m3*)P.Gt, N, nrt, nkc,
                                                                      P.gscale, 0);
      break;
    default: return cudaErrorInvalidValue;
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    P.gt_prec = precision;
    P.gt_frag = frag;
  }
  return e;
}

// Host description of one problem for the batched kernel, written into `dst`
// (a BInst of the precision's compute type): its buffers, its threshold term
// theta of this outer iteration, its instance number and its run parameters.
template <typename CT>
static void fill_inst(BInst<CT>& I, const ProblemDev& P, const SolveDev& S, const cs_params& prm, double theta,
                      int inst) {
  I.N = (int)P.N; I.nrt = (int)((P.N + kRT - 1) / kRT); I.nkc = (int)(P.Npad / kKC);
  I.Gt = P.Gt; I.gscale = P.gscale; I.R = S.R; I.hz = P.hz; I.g = P.g;
  I.X0 = (CT*)S.X0; I.X1 = (CT*)S.X1; I.state = (CT*)S.state; I.sigma = S.sigma;
  I.theta = theta; I.inst = inst;
  I.n_steps = prm.n_steps; I.pump_kind = prm.pump_kind; I.field = prm.field; I.init_kind = prm.init_kind;
  I.self_term = prm.self_term;
  I.dt = prm.dt; I.p0 = prm.p0; I.p1 = prm.p1; I.p_thr = prm.p_thr; I.d = prm.d; I.t0 = prm.t0;
  I.width = prm.width; I.beta = prm.beta; I.tau = prm.tau; I.Kj = prm.K * prm.j; I.init_scale = prm.init_scale;
  I.seed = prm.seed;
}

void fill_batch_inst(void* dst, const ProblemDev& P, const SolveDev& S, const cs_params& prm, double theta,
                     int inst) {
  if (prm.precision == CS_P_FP64) {
    BInst<double> I;
    fill_inst(I, P, S, prm, theta, inst);
    *reinterpret_cast<BInst<double>*>(dst) = I;
  } else {
    BInst<float> I;
    fill_inst(I, P, S, prm, theta, inst);
    *reinterpret_cast<BInst<float>*>(dst) = I;
  }
}

cudaError_t launch_euler_batch(const BatchLaunch& L, cudaStream_t st) {
  switch (L.prm->precision) {
    case CS_P_FP64: return launch_batch_mr<double, double>(L, st);
    case CS_P_FP32: return launch_batch_mr<float, float>(L, st);
    case CS_P_BF16: return launch_batch_mr<__nv_bfloat16, float>(L, st);
    case CS_P_FP16: return launch_batch_mr<__half, float>(L, st);
    case CS_P_FP8: return launch_batch_mr<__nv_fp8_e4m3, float>(L, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cs
