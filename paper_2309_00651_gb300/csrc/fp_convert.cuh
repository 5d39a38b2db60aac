// FP64 <-> FP32 conversions written from the IEEE-754 binary64/binary32 layouts with integer
// operations (the reduced-rate FP64 pipe of this part stays out of the contraction kernels).
#pragma once
#include <cuda_runtime.h>

namespace hfx {
namespace ace {

// FP64 -> FP32, round to nearest even, from the IEEE-754 binary64/binary32 layouts with integer
// operations: keep sign, rebias the exponent (1023 -> 127), round the 52-bit fraction to 23
// bits.  Magnitudes below 2^-126 flush to zero, above the FP32 range go to infinity.  (Measured
// faster inside the contraction kernel than the hardware conversion.)
__device__ __forceinline__ float f64_to_f32_rn(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned mag = hi & 0x7fffffffu;
  unsigned f = ((mag - 0x38000000u) << 3) | (lo >> 29);  // (e - 896) << 23 | top 23 fraction bits
  const unsigned rem = lo & 0x1fffffffu;                  // the 29 dropped bits
  f += (rem > 0x10000000u) | ((rem == 0x10000000u) & (f & 1u));
  f = (mag < 0x38100000u) ? 0u : f;             // e < 897: below the FP32 normal range
  f = (mag >= 0x47f00000u) ? 0x7f800000u : f;   // e > 1150: beyond it
  return __uint_as_float(f | (hi & 0x80000000u));
}

// FP32 -> FP64, exact for normal numbers (and +-0): keep sign, rebias the exponent
// (127 -> 1023), widen the fraction.  FP32 subnormals flush to zero, infinities and NaNs map to
// infinity.  Integer operations only, so the reduced-rate FP64 pipe is not touched.
__device__ __forceinline__ double f32_to_f64_exact(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned mag = u & 0x7fffffffu;
  unsigned hi = ((mag >> 3) + 0x38000000u) | (u & 0x80000000u);  // (e + 896) << 20 | top 20 fraction bits
  unsigned lo = mag << 29;                                         // low 3 fraction bits
  const bool tiny = mag < 0x00800000u, huge = mag >= 0x7f800000u;
  hi = tiny ? (u & 0x80000000u) : (huge ? (0x7ff00000u | (u & 0x80000000u)) : hi);
  lo = (tiny || huge) ? 0u : lo;
  return __hiloint2double((int)hi, (int)lo);
}

}  // namespace ace
}  // namespace hfx
