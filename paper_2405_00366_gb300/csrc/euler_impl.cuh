// Host side of one CIM run: the planner that picks the work split of the
// persistent Euler kernel (euler_kernel.cuh) for N, T and this GPU, the
// optional autotuner, and the launcher.
#pragma once

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "euler_kernel.cuh"

namespace cs {
namespace {
struct Plan {
  int C, NC, RPC, RPC_pad, ORW, kq, kch, slots, RW, RG, MR, WK, ldg;
  bool stream, wide, tc, tc5;
  size_t smem, slot_bytes, xoff;
};

template <typename CT>
using EulerFn = void (*)(EulerArgs<CT>);

template <typename GT, typename CT, bool STREAM, bool WIDE, bool TC = false>
EulerFn<CT> kernel_for_s(int MR) {
  switch (MR) {
    case 1: return euler_kernel<GT, CT, 1, STREAM, WIDE, TC, false>;
    case 2: return euler_kernel<GT, CT, 2, STREAM, WIDE, TC, false>;
    case 3: return euler_kernel<GT, CT, 3, STREAM, WIDE, TC, false>;
    case 4: return euler_kernel<GT, CT, 4, STREAM, WIDE, TC, false>;
    case 5: return euler_kernel<GT, CT, 5, STREAM, WIDE, TC, false>;
    case 6: return euler_kernel<GT, CT, 6, STREAM, WIDE, TC, false>;
    case 7: return euler_kernel<GT, CT, 7, STREAM, WIDE, TC, false>;
    default: return euler_kernel<GT, CT, 8, STREAM, WIDE, TC, false>;
  }
}

// Streaming (G_off tiles from memory every step) is built for the reduced
// storage types only; FP64 problems must fit on chip.  The wide split is built
// for FP32 compute only.
template <typename GT> struct streamable { static constexpr bool value = !std::is_same<GT, double>::value; };
template <typename CT> struct widenable { static constexpr bool value = std::is_same<CT, float>::value; };
// The tensor-core forms: streamed FP16 / BF16 G_off with FP32 compute, and
// resident FP32 G_off (three FP16 MMAs on split operands).
template <typename GT, typename CT> struct tensorable {
  static constexpr bool value = tc_type<GT>::value && std::is_same<CT, float>::value;
};
template <typename GT, typename CT> struct h3able {
  static constexpr bool value = std::is_same<GT, float>::value && std::is_same<CT, float>::value;
};

template <typename GT, typename CT, bool WIDE>
EulerFn<CT> kernel_for_w(int MR, bool stream) {
  if constexpr (streamable<GT>::value) {
    if (stream) return kernel_for_s<GT, CT, true, WIDE>(MR);
  }
  return kernel_for_s<GT, CT, false, WIDE>(MR);
}

template <typename GT, typename CT>
EulerFn<CT> kernel_for(int MR, bool stream, bool wide, bool tc, bool tc5 = false) {
  if constexpr (h3able<GT, CT>::value) {
    if (tc5) return euler_kernel<GT, CT, 1, false, true, true, true>;
  }
  if constexpr (tensorable<GT, CT>::value) {
    if (tc) return kernel_for_s<GT, CT, true, true, true>(MR);
  }
  if constexpr (h3able<GT, CT>::value) {
    if (tc) return kernel_for_s<GT, CT, false, true, true>(MR);
  }
  if constexpr (widenable<CT>::value) {
    if (wide) return kernel_for_w<GT, CT, true>(MR, stream);
  }
  return kernel_for_w<GT, CT, false>(MR, stream);
}

// Work split for N and T on this GPU.  For each cluster size C in {1, 2, 4, 8}
// (or only the caller's hint) and each split of the consumer warps, take the
// largest number of clusters that is resident at once with the footprint it
// implies (rows per lane MR, ring slots), first with G_off resident in shared
// memory and, if that cannot fit, with G_off tiles streamed from memory every
// step.  Keep the plan with the lowest estimate of one step per CTA, in clocks:
//  * wide split (FP32, all trial blocks of one width in {8, 16, 32, 64}): the
//    larger of the FMA rate (128 per clock at 67%, the rate measured on GB300
//    for this loop alone), shared-memory wavefronts (1 per clock, at 90%: per
//    four k a warp loads 4 X and MR G quads, each one wavefront per half-warp,
//    for 8 MR packed FMAs) and streamed G bytes at 22 per clock (one SM's share
//    of HBM), plus the k-warp reduction;
//  * narrow split (every other case; measured at about 45% of FFMA issue):
//    FMAs at 128 per clock / 0.45, or streamed G bytes;
//  * tensor-core forms (tensor_form != 1): streamed 16-bit G_off with 8 trials,
//    the larger of two m16n8k16 MMAs per 16 x 16 tile at one per 2 clocks and
//    the streamed G bytes; resident FP32 G_off with blocks of 16/32/64 trials,
//    three MMAs per 16 x 8 x 16 tile at one per 2 clocks and 70% of that
//    (mma.sync rates measured on GB300), plus the k-warp reduction; and the
//    tcgen05 form (resident FP32 G_off, at most 64 rows per cluster): one
//    M = 128 MMA per 16-k block plus the epilogue's TMEM loads
//    (tensor_form = 3 keeps the mma.sync forms only);
// each plus X bytes at 44 per clock (measured: the X traffic of a step adds to
// its time rather than overlapping the product), a fixed cost per cluster rank
// for the reduction through distributed shared memory, and the step barrier: a
// grid barrier (about 1.8 us measured; cheaper when the grid is a single
// cluster).  FP64 FMAs count at 1/64 of the FP32 rate (GB300 issues about 2
// FP64 FMAs per clock per SM, measured).  For the autotuner, besides the
// largest number of clusters that fits, a single cluster is offered too: for
// small problems it can be the fastest split and can be far from it, beyond
// what this model resolves.
template <typename GT, typename CT>
cudaError_t make_plan(const ProblemDev& P, int T, int hint, int max_ctas, bool force_stream, int tensor_form, Plan* out,
                      std::vector<std::pair<double, Plan>>* cands = nullptr, bool single_cluster = false,
                      int nst = 4) {
  const int N = (int)P.N, nq = (int)(P.Npad / 4);
  const int sms = max_ctas > 0 ? std::min(max_ctas, P.num_sms) : P.num_sms;
  const int twmax = round4(std::min(T, kTChunk));
  const int nblk = (T + kTChunk - 1) / kTChunk;
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P.device);
  if (e != cudaSuccess) { g_where = "cudaDeviceGetAttribute(optin)"; return e; }
  // narrow split: lane column groups of four trials
  const int WCn = col_warps(twmax), WRn = kConsumerWarps / WCn;
  int CGn = 1;
  while (CGn * 4 < twmax / WCn) CGn <<= 1;
  // the wide split needs every trial block to be twmax wide, with twmax / 8 a
  // power of two (lane column groups)
  const bool wide_ok = widenable<CT>::value && (twmax == 8 || twmax == 16 || twmax == 32 || twmax == 64) &&
                       (T <= kTChunk || T % kTChunk == 0);
  // the 16-bit tensor-core form (streamed): one block of exactly eight trials;
  // the FP32 one (resident): blocks of one width in {16, 32, 64}
  const bool tc_ok = tensorable<GT, CT>::value && tensor_form != 1 && T == 8;
  const bool h3_ok = h3able<GT, CT>::value && tensor_form != 1 && twmax >= 16 && wide_ok;
  // the tcgen05 form (resident FP32 G_off): the same trial blocks, at most 64 rows per cluster
  const bool tc5_ok = h3able<GT, CT>::value && tensor_form != 1 && tensor_form != 3 && twmax >= 16 && wide_ok;
  // tensor_form: 0 any form, 1 FMA forms only, 2 tensor-core forms only, 3 mma.sync forms only,
  // 4 the tcgen05 form only
  double best_cost = 0.0;
  bool found = false;
  Plan bp{};
  const int csizes[] = {1, 2, 4, 8};
  for (int pass = force_stream ? 1 : 0; pass < 2 && !found; ++pass) {
    const bool stream = pass == 1;
    if (stream && !streamable<GT>::value) break;
    for (int C : csizes) {
      if (hint > 0 && C != hint) continue;
      if (C > nq || sms < C) continue;
      // variants: wide with WK = 1, 2, 4, 8 k-warps, narrow (WK = 0), the
      // mma.sync tensor-core forms with WK = 1, 2, 4, 8 (v = 5 .. 8) and the
      // tcgen05 form (resident only) with 16 KB (v = 9) or 32 KB (v = 10) X chunks
      for (int v = 0; v < 11; ++v) {
        const bool tc5 = v >= 9;
        const int xchunk = v == 10 ? 32768 : 16384;
        const bool tc = v >= 5;
        const int WK = tc5 ? 1 : (tc ? 1 << (v - 5) : (v < 4 ? 1 << v : 0));
        const bool wide = WK > 0;
        if (wide && !wide_ok) continue;
        if (tc5 && (stream || !tc5_ok)) continue;
        if (tc && !tc5 && !(stream ? tc_ok : h3_ok)) continue;
        if (!tc5 && tensor_form == 4) continue;
        if (tc && !tc5 && !stream && WK * (twmax / 16) > kConsumerWarps) continue;
        if (!tc && tensor_form >= 2) continue;
        Plan pl{};
        pl.C = C;
        pl.stream = stream;
        pl.wide = wide;
        pl.tc = tc;
        pl.tc5 = tc5;
        pl.WK = wide ? WK : 1;
        if (stream) {
          pl.kq = ((nq + C - 1) / C + 7) / 8 * 8;  // whole 32-column tiles per rank
          pl.kch = kStreamK;  // per slot; widened below to as many tiles as the ring allows
        } else {
          pl.kq = (nq + C - 1) / C;
          if (tc) pl.kq = (pl.kq + 3) / 4 * 4;  // whole blocks of 16 k per rank
          // 16 KB (or 32 KB) of X per bulk copy: each copy costs about 350 clocks of
          // the copy engine whatever its size up to 32 KB (measured on GB300), so
          // fewer, larger chunks stream X faster
          pl.kch = std::max(4, std::min(pl.kq * 4, (int)((xchunk / (twmax * sizeof(CT))) & ~(size_t)3)));
        }
        // resident G rows: an odd number of quads apart, so the rows a half-warp
        // reads start in different banks
        pl.ldg = (wide && pl.kq % 2 == 0) ? (pl.kq + 1) * 4 : pl.kq * 4;
        if (tc && !stream) pl.ldg = pl.kq * 4;  // the block in A-operand order, no padding
        const int WR = tc && !stream ? kConsumerWarps / (WK * (twmax / 16)) : (wide ? kConsumerWarps / WK : WRn);
        // rows per lane group: the wide split's row groups, or 16-row MMA tiles
        const int CGw = twmax / 4, RGw = tc ? 16 : (wide ? 32 / CGw : 1);
        // the largest number of clusters that fits, and a single cluster (whose
        // steps need only the hardware cluster barrier) when that differs
        bool took_largest = false;
        for (int NC = std::min(sms / C, N); NC >= 1; --NC) {
          if (took_largest && NC != 1) continue;
          pl.RPC = (N + NC - 1) / NC;
          pl.NC = (N + pl.RPC - 1) / pl.RPC;  // no cluster without rows
          if (pl.NC != NC && NC != std::min(sms / C, N)) continue;
          const int rw_need = (pl.RPC + WR - 1) / WR;
          if (tc5) {
            // one M = 128 MMA covers 64 rows (hi over lo); fewer clusters only need more rows
            if (pl.RPC > 64) break;
            pl.RG = 1;
            pl.MR = 1;
          } else if (wide) {
            pl.RG = RGw;
            pl.MR = (rw_need + RGw - 1) / RGw;
          } else {
            // row groups (a power of two that fits beside the column groups, aiming
            // at about four rows per lane) and rows per lane; leftover lanes split k
            int RG = 1;
            while (RG * 4 < rw_need && CGn * RG * 2 <= 32) RG <<= 1;
            pl.RG = RG;
            pl.MR = (rw_need + RG - 1) / RG;
          }
          if (pl.MR > kMaxRowsPerLane) break;  // fewer clusters only need more rows
          pl.RW = pl.RG * pl.MR;
          pl.RPC_pad = WR * pl.RW;
          if (tc5) {
            pl.RW = 8;
            pl.RPC_pad = 64;
          }
          pl.ORW = (pl.RPC + C - 1) / C;
          EulerFn<CT> fn = kernel_for<GT, CT>(pl.MR, stream, wide, tc, tc5);
          cudaFuncAttributes fa;
          e = cudaFuncGetAttributes(&fa, fn);
          if (e != cudaSuccess) { g_where = "cudaFuncGetAttributes"; return e; }
          const size_t cap = (size_t)optin - fa.sharedSizeBytes;
          const size_t gblock = stream ? 0 : (size_t)pl.RPC_pad * pl.ldg * sizeof(GT);
          const size_t kpart = (wide && !tc5) ? (size_t)WK * pl.RPC_pad * twmax * sizeof(float) : 0;
          // streamed plans: the most G_off tiles per slot (4, 2, 1) that leave 3
          // slots (measured: one tile per slot keeps too few bytes in flight)
          pl.slots = 0;
          for (int tps = stream ? 4 : 1; tps >= 1 && pl.slots == 0; tps >>= 1) {
            if (stream && (size_t)tps * kStreamK > (size_t)pl.kq * 4) continue;
            if (stream) pl.kch = kStreamK * tps;
            const size_t gtile = stream ? (size_t)tps * pl.RPC_pad * kStreamK * sizeof(GT) : 0;
            pl.xoff = align128(gtile);
            pl.slot_bytes = align128(pl.xoff + (size_t)pl.kch * twmax * sizeof(CT));
            const int min_slots = (stream && tps > 1) ? 3 : ((stream || tc5) ? 2 : 3);
            for (int slots = 8; slots >= min_slots; --slots) {
              if ((size_t)slots * pl.slot_bytes < kpart) break;  // the ring holds the k-warp partials
              pl.smem =
                  smem_layout(gblock, pl.slot_bytes, slots, pl.RPC_pad, twmax, pl.ORW, T, sizeof(CT), nst).total;
              if (pl.smem <= cap) { pl.slots = slots; break; }
            }
          }
          if (pl.slots == 0) break;  // fewer clusters only need more shared memory
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
          // FP64 FMAs issue at a small fraction of the FP32 rate on this GPU
          const double frate = std::is_same<CT, double>::value ? 2.0 : 128.0;
          const double fma = (double)pl.RPC_pad * pl.kq * 4 * T * (128.0 / frate);
          const double xbytes = (double)pl.kq * 4 * twmax * sizeof(CT) * nblk;
          // streamed G_off bytes, weighted up when a slot carries fewer than 4 tiles
          // (fewer bytes in flight per SM)
          const double gbytes =
              stream ? (double)pl.RPC_pad * pl.kq * 4 * sizeof(GT) * std::max(1.0, 128.0 / pl.kch) : 0.0;
          double cost;
          if (tc5) {
            // one M = 128 MMA per 16-k block (64 clocks at N = 128, about 45 at
            // N <= 64, measured on GB300) overlapping the X stream (about 360
            // clocks per bulk copy of up to 32 KB, measured), then the
            // epilogue's TMEM loads (four accumulators per 16 columns)
            const double nkb = pl.kq * 4 / 16.0;
            const double mma = nkb * nblk * (twmax >= 64 ? 64.0 : 48.0);
            const double copies = std::ceil(pl.kq * 4.0 / pl.kch) * nblk * 360.0;
            const double epi = nblk * (twmax / 16.0) * 400.0;
            cost = std::max(mma, copies) + epi + 256.0;
          } else if (tc && stream) {
            // MMAs (two per 16 x 16 tile of G_off: the two parts of X), taken at
            // one per two clocks per SM (measured on GB300), overlap the streamed bytes
            const double mmas = (double)pl.RPC_pad / 16.0 * pl.kq * 4 / 16.0 * 2.0;
            const double red = (double)WK * pl.RPC * twmax * nblk / kThreads * 4.0;
            cost = std::max(mmas * 2.0, gbytes / 22.0) + xbytes / 44.0 + red;
          } else if (tc) {
            // three m16n8k16 MMAs per 16 x 8 x 16 block, at one per two clocks per
            // SM and about 70% of that (measured on GB300 for this loop)
            const double mmas = (double)pl.RPC_pad / 16.0 * (twmax / 8) * nblk * (pl.kq * 4 / 16) * 3.0;
            const double red = (double)WK * pl.RPC * twmax * nblk / kThreads * 4.0;
            cost = mmas * 2.0 / 0.7 + xbytes / 44.0 + red;
          } else if (wide) {
            const double ffma2 = fma / 64.0;  // packed FMA warp instructions
            const double wf = ffma2 * (8.0 + 2.0 * pl.MR) / (8.0 * pl.MR);
            const double red = (double)WK * pl.RPC * twmax * nblk / kThreads * 4.0;
            cost = std::max(std::max(fma / 128.0 / 0.67, wf / 0.9), gbytes / 22.0) + xbytes / 44.0 + red;
          } else {
            cost = std::max(fma / 128.0 / 0.45, gbytes / 22.0) + xbytes / 44.0;
          }
          cost += 300.0 * C;
          // per-step grid barrier (about 1.8 us measured; less for one cluster)
          cost += pl.NC > 1 ? 3700.0 : 1200.0;
          if (cands) cands->emplace_back(cost, pl);
          if (!found || cost < best_cost) {
            best_cost = cost;
            bp = pl;
            found = true;
          }
          if (took_largest || pl.NC == 1 || !single_cluster) break;
          took_largest = true;
        }
      }
    }
  }
  if (!found) {
    g_where = tensor_form >= 2 ? "make_plan: no tensor-core work split of the requested kind for this shape"
                               : "make_plan: no work split fits";
    return cudaErrorInvalidConfiguration;
  }
  *out = bp;
  if (cands) std::stable_sort(cands->begin(), cands->end(), [](const std::pair<double, Plan>& x,
                                                                const std::pair<double, Plan>& y) {
    return x.first < y.first;
  });
  return cudaSuccess;
}

// Streamed G_off tiles for a plan, rebuilt when the precision or split changes.
template <typename GT>
cudaError_t ensure_cluster_tiles(ProblemDev& P, int precision, const Plan& pl) {
  if (P.Gt2 && P.gt2_prec == precision && P.gt2_rpc == pl.RPC && P.gt2_rpcpad == pl.RPC_pad && P.gt2_nc == pl.NC &&
      P.gt2_frag == (int)pl.tc)
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
                                                                        pl.NC, nkct, P.gscale, (int)pl.tc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  P.gt2_prec = precision;
  P.gt2_rpc = pl.RPC;
  P.gt2_rpcpad = pl.RPC_pad;
  P.gt2_nc = pl.NC;
  P.gt2_frag = (int)pl.tc;
  return cudaSuccess;
}

// One Euler launch of plan `pl` on the problem's stream: n_steps steps
// (prm.n_steps for a real run, fewer for a tuning run) of outer iteration `outer`.
template <typename GT, typename CT>
cudaError_t launch_plan(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                        long long timeout_cycles, const Plan& pl, int n_steps, bool record) {
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
  a.WK = pl.WK;
  a.ldg = pl.ldg;
  a.Gs = P.Gs; a.gscale = P.gscale; a.R = S.R; a.hz = P.hz;
  a.X0 = (CT*)S.X0; a.X1 = (CT*)S.X1;
  a.sigma = S.sigma;
  a.record_steps = (record && outer == 0) ? std::min(S.record_steps, n_steps) : 0;
  a.rec_c = S.rec_c; a.rec_e = S.rec_e;
  a.n_steps = n_steps; a.dt = prm.dt;
  a.pump_kind = prm.pump_kind; a.p0 = prm.p0; a.p1 = prm.p1; a.p_thr = prm.p_thr; a.d = prm.d;
  a.t0 = prm.t0; a.width = prm.width;
  a.beta = prm.beta; a.tau = prm.tau; a.Kj = prm.K * prm.j;
  a.theta = sqrt(prm.tau) * eta * eta / 4.0;
  a.field = prm.field; a.init_kind = prm.init_kind; a.init_scale = prm.init_scale;
  a.seed = prm.seed; a.instance = prm.instance; a.outer = outer;
  a.flags = S.bar; a.err = S.err; a.timeout_cycles = timeout_cycles;
  a.g = P.g;
  a.self_term = prm.self_term;
  a.readout = prm.readout;
  a.lam_read = eta * eta / 2.0;
  a.e_hist = S.e_hist;
  a.s_hist = S.s_hist;
  a.phantom = (unsigned)prm.test_phantom_ctas;
  S.plan_cluster = pl.C;
  S.plan_ctas = pl.C * pl.NC;
  S.plan_form = pl.tc5 ? 5 : (pl.tc ? 2 : (pl.wide ? 1 : 0));

  if (pl.C * pl.NC > kMaxEulerCtas) { g_where = "launch_plan: grid larger than the flag array"; return cudaErrorInvalidConfiguration; }
  EulerFn<CT> fn = kernel_for<GT, CT>(pl.MR, pl.stream, pl.wide, pl.tc, pl.tc5);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) { g_where = "cudaFuncSetAttribute(launch)"; return e; }
  // the per-CTA publication flags and the word after them (never written)
  e = cudaMemsetAsync(S.bar, 0, sizeof(unsigned) * ((size_t)pl.C * pl.NC + 1), P.stream);
  if (e != cudaSuccess) { g_where = "cudaMemsetAsync(flags)"; return e; }
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

// The fields that identify a plan among the planner's candidates.
inline std::string plan_tag(const Plan& p) {
  const int v[] = {p.C, p.NC, p.RPC, p.RPC_pad, p.ORW, p.kq, p.kch, p.slots, p.RW, p.RG, p.MR, p.WK, p.ldg,
                   (int)p.stream, (int)p.wide, (int)p.tc, (int)p.tc5};
  std::string s;
  for (int x : v) s += (s.empty() ? "" : " ") + std::to_string(x);
  return s;
}

// Autotuner: time the kTuneCands cheapest candidate splits of the cost model,
// plus the cheapest of each kernel form (FMA, mma.sync, tcgen05) not among them, on
// this GPU (kTuneSteps Euler steps each, twice, CUDA events on the problem's
// stream; the second run counts) and return the fastest.  The runs only write
// the solve's scratch (X, sigma), which the real run rewrites.
constexpr int kTuneCands = 4;
constexpr int kTuneSteps = 48;

template <typename GT, typename CT>
cudaError_t autotune_plan(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                          long long timeout_cycles, const std::vector<std::pair<double, Plan>>& cands, Plan* out) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  const int steps = std::min(prm.n_steps, kTuneSteps);
  std::vector<size_t> pick;
  bool form_seen[3] = {false, false, false};
  for (size_t c = 0; c < cands.size(); ++c) {
    const int f = cands[c].second.tc5 ? 2 : (cands[c].second.tc ? 1 : 0);
    if ((int)pick.size() < kTuneCands || !form_seen[f]) {
      pick.push_back(c);
      form_seen[f] = true;
    }
  }
  for (size_t pi = 0; pi < pick.size() && e == cudaSuccess; ++pi) {
    const size_t c = pick[pi];
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, P.stream);
      if (e == cudaSuccess) e = launch_plan<GT, CT>(P, S, prm, outer, eta, timeout_cycles, cands[c].second, steps,
                                                    false);
      if (e == cudaSuccess) e = cudaEventRecord(e1, P.stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e == cudaSuccess && (pi == 0 || ms < best)) {
      best = ms;
      *out = cands[c].second;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) g_where = "autotuning run";
  return e;
}

template <typename GT, typename CT>
cudaError_t launch_typed(ProblemDev& P, SolveDev& S, const cs_params& prm, int outer, double eta,
                         long long timeout_cycles, bool plan_only) {
  // plans depend only on the shape, the caller's limits and the device; one
  // cache per process (so every thread and every solve of a shape agrees)
  struct Key {
    int64_t N;
    int T, hint, cap, strm, dev, tune, notc, best;
    bool operator<(const Key& o) const {
      return std::tie(N, T, hint, cap, strm, dev, tune, notc, best) <
             std::tie(o.N, o.T, o.hint, o.cap, o.strm, o.dev, o.tune, o.notc, o.best);
    }
  };
  static std::mutex mu;
  static std::map<Key, Plan> cache;
  const Key key{P.N, S.trials, prm.cluster_size, prm.max_ctas, prm.stream_g, P.device, prm.autotune,
                prm.tensor_form, prm.readout};
  Plan pl;
  bool hit = false;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) { pl = it->second; hit = true; }
  }
  if (!hit) {
    std::vector<std::pair<double, Plan>> cands;
    cudaError_t e = make_plan<GT, CT>(P, S.trials, prm.cluster_size, prm.max_ctas, prm.stream_g == 1,
                                      prm.tensor_form, &pl, &cands, prm.autotune != 0,
                                      prm.readout == CS_READOUT_BEST ? 5 : 4);
    if (e != cudaSuccess) return e;
    if (prm.autotune && cands.size() > 1) {
      // a choice persisted by an earlier process counts if it is still one of
      // the candidates; otherwise time them
      const std::string dkey = "euler|" + tune_device_tag(P.device) + "|p" + std::to_string(prm.precision) + "|N" +
                               std::to_string(P.N) + "|T" + std::to_string(S.trials) + "|h" +
                               std::to_string(prm.cluster_size) + "|c" + std::to_string(prm.max_ctas) + "|s" +
                               std::to_string(prm.stream_g) + "|f" + std::to_string(prm.tensor_form) + "|r" +
                               std::to_string(prm.readout);
      std::string stored;
      bool found = false;
      if (tune_lookup(dkey, &stored))
        for (const auto& c : cands)
          if (plan_tag(c.second) == stored) {
            pl = c.second;
            found = true;
            break;
          }
      if (found) {
        tune_note(false);
      } else {
        e = autotune_plan<GT, CT>(P, S, prm, outer, eta, timeout_cycles, cands, &pl);
        if (e != cudaSuccess) return e;
        tune_note(true);
        tune_store(dkey, plan_tag(pl));
      }
    }
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = pl;
  }
  if (plan_only) {
    if (pl.stream) {
      const cudaError_t e = ensure_cluster_tiles<GT>(P, prm.precision, pl);
      if (e != cudaSuccess) g_where = "streamed G_off tiles";
      return e;
    }
    return cudaSuccess;
  }
  return launch_plan<GT, CT>(P, S, prm, outer, eta, timeout_cycles, pl, prm.n_steps, true);
}

}  // namespace

}  // namespace cs
