// Building blocks of the two-pass shared-memory FFTs used by the spiral
// (Toeplitz / gridding) kernels.
//
// A length-L transform (L = P1 * P2) is split as index n = n1 + P1 n2 and
// frequency k = k2 + P2 k1:
//   pass "a": one job per (line, n1) holds the P2 samples n1 + P1 n2 in registers;
//   pass "b": one job per (line, k2) holds the P1 values of frequency group k2.
// Forward: a-jobs run DFT_P2 and multiply W_L^(n1 k2), b-jobs run DFT_P1 and
// end with X[k2 + P2 k1].  Inverse: b-jobs run the inverse DFT_P1 and the
// conjugate twiddle, a-jobs the inverse DFT_P2 and end with x[n1 + P1 n2].
//
// Two shared-memory layouts:
//   column layout  buf[k2][n1][16 lines]   (lines = 16 adjacent image columns)
//   row layout     buf[line][k2][n1 + pad] (lines = 16 image rows; pad keeps the
//                                           stride odd for conflict-free access)
#pragma once
#include "common.cuh"
#include "dft_codelets.cuh"

namespace pico {

constexpr int kLines = 16;

template <int P1, int P2>
struct Split {
  static constexpr int L = P1 * P2;
  static constexpr int NT = (kLines * (P1 > P2 ? P1 : P2) + 31) / 32 * 32;
  static constexpr int LD = P1 + ((P1 % 2 == 0) ? 1 : 0);
  static constexpr size_t col_buf = (size_t)L * kLines * sizeof(float2);
  static constexpr size_t row_buf = (size_t)kLines * P2 * LD * sizeof(float2);
};

// ---- column layout (LS lines per block, kLines unless stated) ----
template <int P, int SIGN, int NZ>
__device__ __forceinline__ void dft_nz(float2 (&z)[P]);
template <int P1, int P2, int SIGN, int NZ = P2, int LS = kLines>
__device__ __forceinline__ void cola_store(float2 (&z)[P2], int n1, int ln, float2* buf, const float2* tws) {
  dft_nz<P2, SIGN, NZ>(z);
#pragma unroll
  for (int k = 0; k < P2; ++k) {
    const float2 w = tws[n1 * k];
    buf[(k * P1 + n1) * LS + ln] = k == 0 ? z[0] : (SIGN < 0 ? cmul(z[k], w) : cmul_cb(z[k], w));
  }
}
template <int P1, int P2, int LS = kLines>
__device__ __forceinline__ void colb_load(float2 (&y)[P1], int k2, int ln, const float2* buf) {
#pragma unroll
  for (int m = 0; m < P1; ++m) y[m] = buf[(k2 * P1 + m) * LS + ln];
}
template <int P1, int P2, int LS = kLines>
__device__ __forceinline__ void colb_store(const float2 (&y)[P1], int k2, int ln, float2* buf) {
#pragma unroll
  for (int m = 0; m < P1; ++m) buf[(k2 * P1 + m) * LS + ln] = y[m];
}
// inverse DFT_P1 of a b-job and the conjugate twiddle, stored for the a-jobs
template <int P1, int P2, int LS = kLines>
__device__ __forceinline__ void colb_inv_store(float2 (&y)[P1], int k2, int ln, float2* buf, const float2* tws) {
  DFT<P1, 1>::run(y);
#pragma unroll
  for (int m = 0; m < P1; ++m) buf[(k2 * P1 + m) * LS + ln] = m == 0 ? y[0] : cmul_cb(y[m], tws[m * k2]);
}
template <int P1, int P2, int SIGN, int LS = kLines>
__device__ __forceinline__ void cola_load(float2 (&z)[P2], int n1, int ln, const float2* buf) {
#pragma unroll
  for (int k = 0; k < P2; ++k) z[k] = buf[(k * P1 + n1) * LS + ln];
  DFT<P2, SIGN>::run(z);
}

// DFT_P of which only the first NZ inputs can be non-zero (zero-padded lines)
template <int P, int SIGN, int NZ>
__device__ __forceinline__ void dft_nz(float2 (&z)[P]) {
  if constexpr (NZ == P) {
    DFT<P, SIGN>::run(z);
  } else {
    DFTZ<P, SIGN, NZ>::run(z);
  }
}

// ---- row layout ----
template <int P1, int P2, int SIGN, int NZ = P2>
__device__ __forceinline__ void rowa_store(float2 (&z)[P2], int n1, int ln, float2* buf, const float2* tws) {
  constexpr int LD = Split<P1, P2>::LD;
  dft_nz<P2, SIGN, NZ>(z);
#pragma unroll
  for (int k = 0; k < P2; ++k) {
    const float2 w = tws[n1 * k];
    buf[(ln * P2 + k) * LD + n1] = k == 0 ? z[0] : (SIGN < 0 ? cmul(z[k], w) : cmul_cb(z[k], w));
  }
}
template <int P1, int P2, int SIGN>
__device__ __forceinline__ void rowb_load(float2 (&y)[P1], int k2, int ln, const float2* buf) {
  constexpr int LD = Split<P1, P2>::LD;
#pragma unroll
  for (int m = 0; m < P1; ++m) y[m] = buf[(ln * P2 + k2) * LD + m];
  DFT<P1, SIGN>::run(y);
}
template <int P1, int P2>
__device__ __forceinline__ void rowb_inv_store(float2 (&y)[P1], int k2, int ln, float2* buf, const float2* tws) {
  constexpr int LD = Split<P1, P2>::LD;
  DFT<P1, 1>::run(y);
#pragma unroll
  for (int m = 0; m < P1; ++m) buf[(ln * P2 + k2) * LD + m] = m == 0 ? y[0] : cmul_cb(y[m], tws[m * k2]);
}
template <int P1, int P2>
__device__ __forceinline__ void rowa_inv_load(float2 (&z)[P2], int n1, int ln, const float2* buf) {
  constexpr int LD = Split<P1, P2>::LD;
#pragma unroll
  for (int k = 0; k < P2; ++k) z[k] = buf[(ln * P2 + k) * LD + n1];
  DFT<P2, 1>::run(z);
}

}  // namespace pico
