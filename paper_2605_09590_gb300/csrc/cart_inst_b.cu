// Explicit instantiations of the Cartesian kernels, lengths 160..384.
#include "cart_impl.cuh"
#include "cart_sizes.h"
namespace pico {
#define PICO_INST(N, A, B)                                                                                    \
  template void launch_col_normal_t<A, B>(const CartOp&, const float2*, float2*, int, float, const CgArgs*, int, \
                                          cudaStream_t);                                                      \
  template void launch_col_pmr_t<A, B>(const CartOp&, float2*, int, uint64_t, int64_t, float, cudaStream_t, \
                                       const float2*);                                                        \
  template void launch_row_adjoint_t<A, B>(const CartOp&, const float2*, float2*, int, cudaStream_t);
PICO_SIZES_B(PICO_INST)
}  // namespace pico
