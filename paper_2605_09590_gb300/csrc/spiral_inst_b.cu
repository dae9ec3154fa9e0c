// Explicit instantiations of the spiral (Toeplitz / gridding) kernel launchers.
#include "spiral_impl.cuh"
#include "spiral_sizes.h"
namespace pico {
#define PICO_INST(LL, A, B)                                                                                  \
  template void launch_toep_normal_t<A, B>(const SpiralOp&, const float2*, float2*, float2*, int, float,     \
                                           const CgArgs*, int, cudaStream_t);                                \
  template void launch_fft2_t<A, B>(float2*, const float2*, int, int, bool, cudaStream_t);                   \
  template void launch_grid_cols_adjoint_t<A, B>(const SpiralOp&, const float2*, float2*, int, cudaStream_t);
PICO_GRID_SIZES_B(PICO_INST)
}  // namespace pico
