// Shared device helpers of the CUDA path: numeric conversions, the device
// error word, acquire/release accesses, block reductions and the
// counter-based generator of the initial amplitudes.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "../../include/cs.h"

namespace cs {

// ------------------------------------------------------------------ conversions
template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<double>(double v) { return (float)v; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f32<__nv_fp8_e4m3>(__nv_fp8_e4m3 v) { return float(v); }

// Storage types whose values carry a per-row scale (the row's largest |G_off|
// over the format's largest finite value): only FP8.
template <typename GT> struct row_scaled { static constexpr bool value = false; };
template <> struct row_scaled<__nv_fp8_e4m3> { static constexpr bool value = true; };

// widen a storage value to the compute type CT
template <typename CT, typename GT> __device__ __forceinline__ CT widen(GT v) { return (CT)to_f32(v); }
template <> __device__ __forceinline__ double widen<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float widen<float, float>(float v) { return v; }

// ------------------------------------------------------------------ error word
// Device error codes written into the per-solve error word (first writer wins).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_NONFINITE = 2, DEV_BADARG = 3 };

__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// ------------------------------------------------------------------ reductions
// Deterministic block sum (fixed tree order) of one double per thread.
// `scratch` must hold blockDim.x / 32 doubles.  Result valid in every thread.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += scratch[i];
  return s;
}

// ------------------------------------------------------------------ generator
// SplitMix64 finaliser (Steele, Lea & Flood 2014), golden-ratio increment.
__host__ __device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// Key of one CIM run: chained finaliser over (seed, instance, trial, outer).
__host__ __device__ __forceinline__ uint64_t run_key(uint64_t seed, uint64_t inst,
                                                     uint64_t trial, uint64_t outer) {
  uint64_t k = splitmix64_mix(seed);
  k = splitmix64_mix(k + kGamma * (inst + 1));
  k = splitmix64_mix(k + kGamma * (trial + 1));
  k = splitmix64_mix(k + kGamma * (outer + 1));
  return k;
}

// Uniform double in [0, 1) for spin r and lane (0 or 1) of a run key.
__device__ __forceinline__ double run_uniform(uint64_t key, uint64_t r, uint64_t lane) {
  const uint64_t z = splitmix64_mix(key + kGamma * (2 * r + lane + 1));
  return (double)(z >> 11) * 0x1.0p-53;
}

// Initial amplitude of spin r: U(-s, s) or N(0, s^2) by Box-Muller.
__device__ __forceinline__ double initial_amplitude(uint64_t key, uint64_t r, int kind, double s) {
  const double u1 = run_uniform(key, r, 0);
  if (kind == CS_INIT_UNIFORM) return s * (2.0 * u1 - 1.0);
  const double u2 = run_uniform(key, r, 1);
  return s * sqrt(-2.0 * log1p(-u1)) * cospi(2.0 * u2);
}

}  // namespace cs
