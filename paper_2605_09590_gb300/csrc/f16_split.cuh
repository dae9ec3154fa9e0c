// FP16 head + remainder operands of the tensor-core Gram products: a float
// scaled by a power of two splits into an FP16 head (rounded to nearest) and
// the FP16 of what remains, so that head + remainder carries about 22
// significant bits into a kind::f16 MMA with FP32 accumulation.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>
#include <string.h>

namespace pico {

// Power-of-two scale 2^(14 - e) for a bound = m 2^e (m in [0.5, 1)): a value
// of magnitude at most `bound` times the scale stays below 2^14 (FP16 holds
// up to 65504), and the scale itself is exact in FP32.  A zero or non-finite
// bound gives 1.
__host__ __device__ __forceinline__ float pow2_scale(double bound) {
  if (!(bound > 0.0) || !(bound < 1e300)) return 1.f;
  int e = 0;
  (void)frexp(bound, &e);
  int k = 14 - e;
  k = k > 100 ? 100 : (k < -100 ? -100 : k);
  return ldexpf(1.f, k);
}
// The same from a float bound, from its exponent bits (FP32 only)
__device__ __forceinline__ float pow2_scale_f(float bound) {
  if (!(bound > 0.f) || !(bound <= 3.0e38f)) return 1.f;
  const int eb = (int)((__float_as_uint(bound) >> 23) & 0xff);
  const int e = eb == 0 ? -126 : eb - 126;  // bound = m 2^e, m in [0.5, 1) (subnormals: at most 2^-126)
  int k = 14 - e;
  k = k > 100 ? 100 : (k < -100 ? -100 : k);
  return __int_as_float((127 + k) << 23);
}

__device__ __forceinline__ uint32_t h2_bits(__half2 h) {
  uint32_t u;
  memcpy(&u, &h, sizeof(u));
  return u;
}
// four FP32 values -> FP16 heads and FP16 remainders, each packed as four
// halves in a uint2 (element 0 in the low half)
__device__ __forceinline__ void split_f16x4(float a0, float a1, float a2, float a3, uint2& hi, uint2& lo) {
  const __half2 h01 = __floats2half2_rn(a0, a1), h23 = __floats2half2_rn(a2, a3);
  const float2 f01 = __half22float2(h01), f23 = __half22float2(h23);
  hi = make_uint2(h2_bits(h01), h2_bits(h23));
  lo = make_uint2(h2_bits(__floats2half2_rn(a0 - f01.x, a1 - f01.y)),
                  h2_bits(__floats2half2_rn(a2 - f23.x, a3 - f23.y)));
}

}  // namespace pico
