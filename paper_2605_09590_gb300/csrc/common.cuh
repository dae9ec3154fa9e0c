// Shared device helpers of the PICO CUDA library: complex arithmetic,
// the counter-based SplitMix64 draws, and deterministic reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pico {

// ---------------------------------------------------------------------------
// complex64 helpers (float2 = {re, im})
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * b
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmul_cb(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// acc + conj(a) * b
__device__ __forceinline__ float2 cfma_c(float2 acc, float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}
// Re(conj(a) * b)
__device__ __forceinline__ float cdot_re(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): output i of a generator seeded with
// state s is mix64(s + GAMMA * (i + 1)).  Probe p under `seed` uses the key
// splitmix64(seed, p); element e of that probe uses words 2e and 2e+1 of the
// key's own stream.
// ---------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t state, uint64_t i) {
  return mix64(state + kGamma * (i + 1ull));
}
// uniform on [0,1) and (0,1] from the top 24 bits (exact in float32)
__device__ __forceinline__ float unif24(uint64_t h) { return (float)(uint32_t)(h >> 40) * 5.9604644775390625e-8f; }
__device__ __forceinline__ float unif24_open0(uint64_t h) {
  return ((float)(uint32_t)(h >> 40) + 1.0f) * 5.9604644775390625e-8f;
}

enum ProbeKind { kProbePhase = 0, kProbeRademacher = 1, kProbeGauss = 2 };

// Probe value of element e (Sec. 2.2.4: random phase, real Rademacher, complex Gaussian)
__device__ __forceinline__ float2 draw_probe(uint64_t key, uint64_t e, int kind) {
  const uint64_t h0 = splitmix64(key, 2ull * e);
  if (kind == kProbePhase) {
    float s, c;
    sincospif(2.0f * unif24(h0), &s, &c);
    return make_float2(c, s);
  }
  if (kind == kProbeRademacher) return make_float2((h0 >> 63) ? -1.0f : 1.0f, 0.0f);
  const uint64_t h1 = splitmix64(key, 2ull * e + 1ull);
  const float r = sqrtf(-logf(unif24_open0(h0)));
  float s, c;
  sincospif(2.0f * unif24(h1), &s, &c);
  return make_float2(r * c, r * s);
}

// CN(0, sigma^2) draw of element e (PMR noise, polar Box-Muller)
__device__ __forceinline__ float2 draw_cnoise(uint64_t key, uint64_t e, float sigma) {
  const uint64_t h0 = splitmix64(key, 2ull * e);
  const uint64_t h1 = splitmix64(key, 2ull * e + 1ull);
  const float r = sigma * sqrtf(-logf(unif24_open0(h0)));
  float s, c;
  sincospif(2.0f * unif24(h1), &s, &c);
  return make_float2(r * c, r * s);
}

// ---------------------------------------------------------------------------
// Deterministic reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Float-float values hi + lo (|lo| <= ulp(hi) / 2): sums carried to about 44
// bits on the FP32 pipes, for inner products in latency-bound kernels where the
// FP64 pipe (a small fraction of the FP32 rate on this part) would set the
// pace.  The product of two floats is exact as hi + lo with one FMA (Dekker
// 1971); the sum takes Knuth's TwoSum of the high parts (exact rounding error)
// and adds the low parts once.  Explicit _rn intrinsics: no contraction.
struct ffloat {
  float hi, lo;
};
__device__ __forceinline__ ffloat ff_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ffloat ff_add(ffloat a, ffloat b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, t);
  return {h, __fsub_rn(t, __fsub_rn(h, s))};
}
// Re(conj(a) b) of two complex floats, both products exact before the sum
__device__ __forceinline__ ffloat ff_dot2(float2 a, float2 b) { return ff_add(ff_prod(a.x, b.x), ff_prod(a.y, b.y)); }
// xor-butterfly warp sum (the exact TwoSum error makes ff_add commutative
// bit for bit, so every lane ends with the same value)
__device__ __forceinline__ ffloat warp_sum_ff(ffloat v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = ff_add(v, ffloat{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  return v;
}

// Block-wide sum of one double per thread, fixed order; valid in thread 0.
// `scratch` needs blockDim.x/32 doubles of shared memory.
__device__ __forceinline__ double block_sum_d(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum_d(v);
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < nw ? scratch[lane] : 0.0;
    r = warp_sum_d(r);
  }
  __syncthreads();
  return r;
}

// Sum of n partials in a fixed order, evaluated by one full warp (all lanes
// get the result).  Every caller with the same inputs gets the same bits.
__device__ __forceinline__ double warp_sum_parts(const double* __restrict__ p, int n) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  for (int i = lane; i < n; i += 32) v += p[i];
  return warp_sum_d(v);
}

}  // namespace pico
