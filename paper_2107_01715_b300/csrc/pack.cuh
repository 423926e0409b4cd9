// pack.cuh -- conversions and packed FP32x2 arithmetic shared by the kernels
// that write activation maps (the tensor-core layer epilogues and the leaf
// conv1 pass).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace bcts {

// Epilogue arithmetic on column pairs: the packed FP32x2 add / multiply-add
// (IEEE round-to-nearest per lane, the same results as the scalar operations),
// and conversions that clamp negative values to zero as they round, so the
// ReLU costs no instruction of its own.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
// max(a, 0) and max(b, 0) as bf16, a in the low half
__device__ __forceinline__ uint32_t relu_bf16x2(float2 a) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %2, %1;" : "=r"(r) : "f"(a.x), "f"(a.y));
  return r;
}
// max(., 0) of a.x, a.y, b.x, b.y as saturated E4M3 codes, bytes 0..3 in that order
__device__ __forceinline__ uint32_t relu_e4m3x4(float2 a, float2 b) {
  uint32_t r;
  asm("{\n\t.reg .b16 l, h;\n\t"
      "cvt.rn.satfinite.relu.e4m3x2.f32 l, %2, %1;\n\t"
      "cvt.rn.satfinite.relu.e4m3x2.f32 h, %4, %3;\n\t"
      "mov.b32 %0, {l, h};\n\t}"
      : "=r"(r)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

}  // namespace bcts
