// Host-side dispatch of the Cartesian column/row kernels by transform length.
#include "kernels.cuh"
#include "cart_sizes.h"

namespace pico {

template <int N1, int N2>
void launch_col_normal_t(const CartOp&, const float2*, float2*, int, float, const CgArgs*, int, cudaStream_t);
template <int N1, int N2>
void launch_col_pmr_t(const CartOp&, float2*, int, uint64_t, int64_t, float, cudaStream_t, const float2*);
template <int M1, int M2>
void launch_row_adjoint_t(const CartOp&, const float2*, float2*, int, cudaStream_t);

static bool split_of(int n, int* a, int* b) {
#define PICO_SPLIT(N, A, B) \
  if (n == N) {             \
    *a = A;                 \
    *b = B;                 \
    return true;            \
  }
  PICO_SIZES(PICO_SPLIT)
#undef PICO_SPLIT
  return false;
}

bool cart_supported(int ny, int nx, int* N1, int* N2, int* M1, int* M2) {
  // the column operator needs an FFT split of ny; the row transform (PMR adjoint)
  // one of nx, reported as M1 = M2 = 0 when absent
  if (!split_of(nx, M1, M2)) *M1 = *M2 = 0;
  return split_of(ny, N1, N2);
}


void launch_cart_apply(const CartOp& op, const float2* x, float2* y, int nb, float lam, cudaStream_t s) {
#define PICO_CASE(N, A, B) \
  if (op.N1 == A && op.N2 == B) return launch_col_normal_t<A, B>(op, x, y, nb, lam, nullptr, 0, s);
  PICO_SIZES(PICO_CASE)
#undef PICO_CASE
}

void launch_cart_cg_normal(const CartOp& op, const CgArgs& a, int nb, int it, float lam, cudaStream_t s) {
#define PICO_CASE(N, A, B) \
  if (op.N1 == A && op.N2 == B) return launch_col_normal_t<A, B>(op, nullptr, nullptr, nb, lam, &a, it, s);
  PICO_SIZES(PICO_CASE)
#undef PICO_CASE
}

void launch_cart_pmr_cols(const CartOp& op, float2* G, int nb, uint64_t seed, int64_t rep_begin, float sigma,
                          cudaStream_t s, const float2* data) {
#define PICO_CASE(N, A, B) \
  if (op.N1 == A && op.N2 == B) return launch_col_pmr_t<A, B>(op, G, nb, seed, rep_begin, sigma, s, data);
  PICO_SIZES(PICO_CASE)
#undef PICO_CASE
}

void launch_cart_rows_adjoint(const CartOp& op, const float2* G, float2* out, int nb, cudaStream_t s) {
#define PICO_CASE(N, A, B) \
  if (op.M1 == A && op.M2 == B) return launch_row_adjoint_t<A, B>(op, G, out, nb, s);
  PICO_SIZES(PICO_CASE)
#undef PICO_CASE
}

}  // namespace pico
