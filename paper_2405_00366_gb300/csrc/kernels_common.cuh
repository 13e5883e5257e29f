// Device helpers shared by the Euler kernels: sizes, the pump schedule in the
// compute type, and widening loads of four consecutive storage values.
#pragma once

#include "common.cuh"

namespace cs {

__host__ __device__ __forceinline__ size_t align128(size_t b) { return (b + 127) & ~(size_t)127; }
__host__ __device__ __forceinline__ int round4(int v) { return (v + 3) & ~3; }

// Pump rate at step n of a run of S steps, in the compute type: the linear ramp
// p0 + (p1 - p0) n / S or the sigmoid of Eq. pumprateGACS at t = n dt.
template <typename CT>
__device__ __forceinline__ CT pump_at(int n, int S, int kind, double p0, double p1, double p_thr, double d, double dt,
                                      double t0, double width) {
  if (kind == CS_PUMP_LINEAR) return CT(p0) + CT(p1 - p0) * (CT(n) / CT(S));
  const CT t = CT(n) * CT(dt);
  return CT(p_thr - d) + CT(2.0 * d) / (CT(1) + exp(-(t - CT(t0)) / CT(width)));
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
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.y));
  out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}
template <>
__device__ __forceinline__ void load4<float, __half>(const __half* p, float out[4]) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
  out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}

template <>
__device__ __forceinline__ void load4<float, __nv_fp8_e4m3>(const __nv_fp8_e4m3* p, float out[4]) {
  const uint32_t v = *reinterpret_cast<const uint32_t*>(p);
  const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(v & 0xffffu), __NV_E4M3);
  const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(v >> 16), __NV_E4M3);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
  out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}

// A double rounded to a storage type (round to nearest; FP8 saturates to finite).
template <typename GT> __device__ __forceinline__ GT to_storage(double v);
template <> __device__ __forceinline__ double to_storage<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_storage<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_storage<__nv_bfloat16>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ __half to_storage<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __nv_fp8_e4m3 to_storage<__nv_fp8_e4m3>(double v) {
  return __nv_fp8_e4m3((float)v);
}

// Scale of row r of G_off in its storage type (1 unless the type is row-scaled).
template <typename GT, typename CT>
__device__ __forceinline__ CT row_scale(const float* gscale, int r) {
  if constexpr (row_scaled<GT>::value) return CT(gscale[r]);
  return CT(1);
}

// Two FP32 values in one 64-bit register, and the packed FMA of sm_100 and
// later (fma.rn.f32x2: two independent round-to-nearest FMAs, each exactly
// fmaf), which issues two FMAs per instruction.
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 unpack2(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ void fma2(uint64_t& acc, uint64_t a, uint64_t b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

// G_off quad (four consecutive k of one row) as two k-pairs.
template <typename GT>
__device__ __forceinline__ ulonglong2 load_gpairs(const GT* p) {
  float v[4];
  load4<float, GT>(p, v);
  return make_ulonglong2(pack2(v[0], v[1]), pack2(v[2], v[3]));
}
template <>
__device__ __forceinline__ ulonglong2 load_gpairs<float>(const float* p) {
  return *reinterpret_cast<const ulonglong2*>(p);
}

// Offset of X[k][t] in a block of twp trials: k-pair interleaved for the wide
// split ([k/2][t][k%2], so that (X[k][t], X[k+1][t]) is one 64-bit operand of
// the packed FMA), plain row-major [k][t] otherwise.  Any run of an even number
// of k rows starting at an even k is contiguous in both.
template <bool PAIR>
__device__ __forceinline__ size_t xoff(int k, int t, int twp) {
  return PAIR ? ((size_t)(k >> 1) * twp + t) * 2 + (k & 1) : (size_t)k * twp + t;
}

}  // namespace cs
