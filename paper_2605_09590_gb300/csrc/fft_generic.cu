// Batched in-place 1-D FFTs along the rows or the columns of stacks of
// row-major planes (used by the forward / adjoint encoding operators and the
// spiral set-up).  Unnormalised: X_k = sum_n x_n exp(SIGN 2 pi i n k / L).
#include "cart_sizes.h"
#include "fft_blocks.cuh"
#include "kernels.cuh"

namespace pico {

namespace {

// rows of length L (row stride L); blockIdx.x: 16-row tile, blockIdx.y: plane
template <int P1, int P2, int SIGN>
__global__ void __launch_bounds__(Split<P1, P2>::NT, 1)
    k_lines_rows(float2* __restrict__ data, const float2* tw, int nrows, int64_t plane_stride) {
  constexpr int L = P1 * P2;
  constexpr int NT = Split<P1, P2>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* tws = buf + kLines * P2 * Split<P1, P2>::LD;
  const int t = threadIdx.x;
  for (int i = t; i < L; i += NT) tws[i] = tw[i];
  __syncthreads();
  float2* __restrict__ plane = data + (size_t)blockIdx.y * plane_stride;
  const int ra = t / P1, n1 = t % P1;
  const int rb = t / P2, k2 = t % P2;
  const int ya = blockIdx.x * kLines + ra, yb = blockIdx.x * kLines + rb;
  if (t < kLines * P1) {
    float2 z[P2];
    const float2* row = plane + (size_t)(ya < nrows ? ya : 0) * L;
#pragma unroll
    for (int n2 = 0; n2 < P2; ++n2) z[n2] = ya < nrows ? row[n1 + P1 * n2] : make_float2(0.f, 0.f);
    rowa_store<P1, P2, SIGN>(z, n1, ra, buf, tws);
  }
  __syncthreads();
  if (t < kLines * P2 && yb < nrows) {
    float2 y[P1];
    rowb_load<P1, P2, SIGN>(y, k2, rb, buf);
    float2* row = plane + (size_t)yb * L;
#pragma unroll
    for (int k1 = 0; k1 < P1; ++k1) row[k2 + P2 * k1] = y[k1];
  }
}

// columns of length L (row stride ncols); blockIdx.x: 16-column tile, blockIdx.y: plane
template <int P1, int P2, int SIGN>
__global__ void __launch_bounds__(Split<P1, P2>::NT, 1)
    k_lines_cols(float2* __restrict__ data, const float2* tw, int ncols, int64_t plane_stride) {
  constexpr int L = P1 * P2;
  constexpr int NT = Split<P1, P2>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* tws = buf + L * kLines;
  const int t = threadIdx.x;
  for (int i = t; i < L; i += NT) tws[i] = tw[i];
  __syncthreads();
  float2* __restrict__ plane = data + (size_t)blockIdx.y * plane_stride;
  const int ln = t % kLines, job = t / kLines;
  const int x = blockIdx.x * kLines + ln;
  const bool xv = x < ncols;
  if (job < P1) {
    float2 z[P2];
#pragma unroll
    for (int n2 = 0; n2 < P2; ++n2) z[n2] = xv ? plane[(size_t)(job + P1 * n2) * ncols + x] : make_float2(0.f, 0.f);
    cola_store<P1, P2, SIGN>(z, job, ln, buf, tws);
  }
  __syncthreads();
  if (job < P2 && xv) {
    float2 y[P1];
    colb_load<P1, P2>(y, job, ln, buf);
    DFT<P1, SIGN>::run(y);
#pragma unroll
    for (int k1 = 0; k1 < P1; ++k1) plane[(size_t)(job + P2 * k1) * ncols + x] = y[k1];
  }
}

template <int P1, int P2>
void lines_rows_t(float2* data, const float2* tw, int nrows, int planes, int64_t stride, int sign, cudaStream_t s) {
  using Sp = Split<P1, P2>;
  constexpr int L = P1 * P2;
  const size_t sm = Sp::row_buf + L * sizeof(float2);
  auto k = sign < 0 ? k_lines_rows<P1, P2, -1> : k_lines_rows<P1, P2, 1>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k<<<dim3((nrows + kLines - 1) / kLines, planes), Sp::NT, sm, s>>>(data, tw, nrows, stride);
}

template <int P1, int P2>
void lines_cols_t(float2* data, const float2* tw, int ncols, int planes, int64_t stride, int sign, cudaStream_t s) {
  using Sp = Split<P1, P2>;
  constexpr int L = P1 * P2;
  const size_t sm = Sp::col_buf + L * sizeof(float2);
  auto k = sign < 0 ? k_lines_cols<P1, P2, -1> : k_lines_cols<P1, P2, 1>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k<<<dim3((ncols + kLines - 1) / kLines, planes), Sp::NT, sm, s>>>(data, tw, ncols, stride);
}

}  // namespace

#define PICO_LINE_SIZES(X) PICO_SIZES(X) X(480, 30, 16)

bool fft_length_supported(int L) {
#define PICO_CASE(N, A, B) \
  if (L == N) return true;
  PICO_LINE_SIZES(PICO_CASE)
#undef PICO_CASE
  return false;
}

bool launch_fft_rows(int L, float2* data, const float2* tw, int nrows, int planes, int64_t plane_stride, int sign,
                     cudaStream_t s) {
#define PICO_CASE(N, A, B)                                          \
  if (L == N) {                                                     \
    lines_rows_t<A, B>(data, tw, nrows, planes, plane_stride, sign, s); \
    return true;                                                    \
  }
  PICO_LINE_SIZES(PICO_CASE)
#undef PICO_CASE
  return false;
}

bool launch_fft_cols(int L, float2* data, const float2* tw, int ncols, int planes, int64_t plane_stride, int sign,
                     cudaStream_t s) {
#define PICO_CASE(N, A, B)                                          \
  if (L == N) {                                                     \
    lines_cols_t<A, B>(data, tw, ncols, planes, plane_stride, sign, s); \
    return true;                                                    \
  }
  PICO_LINE_SIZES(PICO_CASE)
#undef PICO_CASE
  return false;
}

}  // namespace pico
