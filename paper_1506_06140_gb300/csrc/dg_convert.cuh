// FP64 <-> FP32 conversions with integer instructions.  GB300 issues FP64
// conversions on its narrow FP64 pipe (2 per clock per SM), so kernels that
// convert every weight of a cell use these instead.
#pragma once
#include <cuda_runtime.h>

namespace dgi {

// FP64 -> FP32, rounded to nearest (ties away from zero), with integer
// instructions only: GB300 runs FP64 conversions on its narrow FP64 pipe.
// Adding half an FP32 ulp to the bit pattern before truncating the low 29
// mantissa bits rounds the magnitude (a carry moves into the exponent as it
// should).  |d| below 2^-126 gives 0; |d| must stay below 2^127.
__device__ __forceinline__ float f32_round(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d) + (1ull << 28);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7FFu;  // biased FP64 exponent; FP32 bias is 896 lower
  const unsigned fb = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  return e > 896u ? __uint_as_float(fb) : 0.0f;
}

// FP32 -> FP64 exactly with integer instructions (normal floats and zero;
// FP32 subnormals, below 2^-126, give 0)
__device__ __forceinline__ double f64_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  const unsigned lo = u << 29;
  const unsigned long long b = ((unsigned long long)hi << 32) | lo;
  return e != 0u ? __longlong_as_double((long long)b) : 0.0;
}

}  // namespace dgi
