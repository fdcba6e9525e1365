// hydro_fp.cuh -- FP64 <-> FP32 conversions by integer operations and the
// error-free FP32 pair operations shared by the mixed-precision kernels.
// GB300 runs FP64 arithmetic and f32 <-> f64 conversions at about 2 per clock
// per SM, the integer and FP32 pipes at 64-128, so these stay off the FP64 pipe.
#pragma once
#include <cuda_runtime.h>

namespace hydro {

// FP64 -> FP32: round to nearest on the magnitude (ties away from zero);
// values below the FP32 normal range become signed zero, larger finite values
// infinity, NaN stays NaN.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned lo = (unsigned)__double2loint(x), hi = (unsigned)__double2hiint(x);
  const unsigned mag = hi & 0x7fffffffu;
  unsigned r = __funnelshift_l(lo, hi, 3) + ((lo >> 28) & 1u) - 0xC0000000u;
  if (mag - 0x38100000u >= 0x0FE00000u) {
    r = mag < 0x38100000u ? 0u : ((mag > 0x7ff00000u || (mag == 0x7ff00000u && lo)) ? 0x7fc00000u : 0x7f800000u);
  }
  return __uint_as_float(r | (hi & 0x80000000u));
}

// FP32 -> FP64, exact (FP32 subnormals become zero).
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f), mag = b & 0x7fffffffu;
  unsigned hi = (mag >> 3) + 0x38000000u, lo = b << 29;
  if (mag - 0x00800000u >= 0x7f000000u) {
    const bool small = mag < 0x00800000u;
    hi = small ? 0u : (0x7ff00000u | (mag >> 3));
    lo = small ? 0u : lo;
  }
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)lo);
}

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum1(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// (h, l) = (ah + al) * (bh + bl) to about 2^-46.
__device__ __forceinline__ void pair_mul1(float ah, float al, float bh, float bl, float& h, float& l) {
  h = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -h);
  l = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
}

// (h, l) = (ah + al) + (bh + bl)
__device__ __forceinline__ void pair_add1(float ah, float al, float bh, float bl, float& h, float& l) {
  float e;
  two_sum1(ah, bh, h, e);
  l = __fadd_rn(e, __fadd_rn(al, bl));
}

}  // namespace hydro
