// Warp-level tensor-core MMA (mma.sync m16n8k16, FP32 accumulation) and the
// 16-bit types the tensor-core forms of the coupling product use.
//
// Operand order (PTX ISA, m16n8k16 with 16-bit inputs), lane L = 4 g + i:
//  A (16 x 16): registers {A[g][2i..2i+1], A[g+8][2i..2i+1], A[g][2i+8..], A[g+8][2i+8..]};
//  B (16 x 8):  registers {B[2i..2i+1][g], B[2i+8..2i+9][g]};
//  D (16 x 8):  {D[g][2i], D[g][2i+1], D[g+8][2i], D[g+8][2i+1]}.
// The tensor-core forms give both operands the same renaming of the summation
// index (MMA k 2i, 2i + 1, 2i + 8, 2i + 9 <- k 4i .. 4i + 3 of the block), so
// that a lane's A operand is one 16-byte load and its B operand one 8-byte load.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

namespace cs {
namespace {

// 16-bit storage types the tensor-core forms take as the A operand directly,
// with the shift s of the lo part of X (X = hi + 2^-s lo)
template <typename GT> struct tc_type { static constexpr bool value = false; };
template <> struct tc_type<__half> { static constexpr bool value = true; static constexpr int kLoShift = 11; };
template <> struct tc_type<__nv_bfloat16> { static constexpr bool value = true; static constexpr int kLoShift = 8; };
// 16-bit type and lo shift of the two parts of X in a tensor-core form: the
// storage type's own for 16-bit G_off, FP16 for FP32 G_off
template <typename GT> struct tc_x { using type = GT; static constexpr int kLoShift = tc_type<GT>::kLoShift; };
template <> struct tc_x<float> { using type = __half; static constexpr int kLoShift = 11; };

// d += A B for one 16 x 8 x 16 tile (A and B of the same 16-bit type GT)
template <typename GT>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint4& a, const uint2& b) {
  if constexpr (std::is_same<GT, __half>::value) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
  } else {
    static_assert(std::is_same<GT, __nv_bfloat16>::value, "FP16 or BF16 operands");
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
  }
}

// Index (in 16-bit elements) of X[k][t] part p (0 hi, 1 lo) in a block of twp
// trials stored as [k / 16][part][t][k % 16].
__host__ __device__ __forceinline__ size_t tc_xidx(int k, int t, int twp, int p) {
  return (((size_t)(k >> 4) * 2 + p) * twp + t) * 16 + (k & 15);
}

// Element e (0..7) of lane L's 16 bytes in a 16 x 16 A-operand block: its row
// and column inside the block.
__host__ __device__ __forceinline__ void tc_arow_col(int L, int e, int& r, int& k) {
  r = (L >> 2) + 8 * ((e >> 1) & 1);
  k = 4 * (L & 3) + 2 * (e >> 2) + (e & 1);
}

}  // namespace
}  // namespace cs
