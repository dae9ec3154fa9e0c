// Element-wise and interpolation kernels of the forward encoding operator
// A x (Sec. 2.1.1, Eq. 1 after pre-whitening, Eq. 3):
//   Cartesian: y_c = M F (S_c x), orthonormal 2-D DFT, zero off the mask;
//   spiral:    y_c[m] = (1/n) sum_r (S_c x)[r] e^{-2 pi i k_m . r / n}, evaluated as a
//              Kaiser-Bessel NUFFT: deapodise, centre on the 2n grid, 2-D FFT,
//              interpolate the W x W neighbourhood of every sample.
#include "common.cuh"
#include "kernels.cuh"

namespace pico {

namespace {

__global__ void k_cart_smul(const float2* __restrict__ x, const float2* __restrict__ S, float2* __restrict__ G,
                            int nc, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int bc = blockIdx.y, b = bc / nc, c = bc % nc;
  G[(size_t)bc * n + i] = cmul(S[(size_t)c * n + i], x[(size_t)b * n + i]);
}

__global__ void k_cart_mask_scale(float2* __restrict__ G, const uint8_t* __restrict__ mask, int ny, int nx,
                                  float scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)ny * nx;
  if (i >= n) return;
  const int ky = (int)(i / nx);
  float2* g = G + (size_t)blockIdx.y * n + i;
  *g = mask[ky] ? cscale(*g, scale) : make_float2(0.f, 0.f);
}

// centred, deapodised coil image on the 2n grid (zero outside the image)
__global__ void k_spiral_pad(SpiralOp op, const float2* __restrict__ x, float2* __restrict__ G) {
  const int L = op.L, n = op.n;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)L * L) return;
  const int bc = blockIdx.y, b = bc / op.nc, c = bc % op.nc;
  const int gy = (int)(i / L), gx = (int)(i % L);
  const int y = (gy + n / 2) % L, xx = (gx + n / 2) % L;
  float2 v = make_float2(0.f, 0.f);
  if (y < n && xx < n) {
    const size_t r = (size_t)y * n + xx;
    v = cscale(cmul(op.smaps[(size_t)c * n * n + r], x[(size_t)b * n * n + r]), op.deapod[xx] * op.deapod[y]);
  }
  G[(size_t)bc * L * L + i] = v;
}

// y[b][c][m] = conj(e^{i pi (kx + ky)}) sum_{|g - u_m| <= W/2} G[b][c][g] phi(g - u_m)
__global__ void k_nufft_interp(SpiralOp op, const float2* __restrict__ G, float2* __restrict__ y) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= op.M) return;
  const int bc = blockIdx.y;
  const int L = op.L;
  const float hw = op.halfw;
  const float2 u = op.u[m];
  const float2* __restrict__ g = G + (size_t)bc * L * L;
  const int x0 = (int)ceilf(u.x - hw), x1 = (int)floorf(u.x + hw);
  const int y0 = (int)ceilf(u.y - hw), y1 = (int)floorf(u.y + hw);
  float2 acc = make_float2(0.f, 0.f);
  for (int gy = y0; gy <= y1; ++gy) {
    const float dy = (float)gy - u.y;
    const float ay = fmaxf(0.f, 1.f - (dy / hw) * (dy / hw));
    const float wy = cyl_bessel_i0f(op.beta * sqrtf(ay)) * op.inv_i0beta;
    const int ry = ((gy % L) + L) % L;
    for (int gx = x0; gx <= x1; ++gx) {
      const float dx = (float)gx - u.x;
      const float ax = fmaxf(0.f, 1.f - (dx / hw) * (dx / hw));
      const float w = wy * cyl_bessel_i0f(op.beta * sqrtf(ax)) * op.inv_i0beta;
      const float2 v = g[(size_t)ry * L + ((gx % L) + L) % L];
      acc.x = fmaf(w, v.x, acc.x);
      acc.y = fmaf(w, v.y, acc.y);
    }
  }
  y[(size_t)bc * op.M + m] = cmul_cb(acc, op.cphase[m]);
}

}  // namespace

void launch_cart_smul(const float2* x, const float2* S, float2* G, int nb, int nc, int64_t n, cudaStream_t s) {
  k_cart_smul<<<dim3((unsigned)((n + 255) / 256), nb * nc), 256, 0, s>>>(x, S, G, nc, n);
}
void launch_cart_mask_scale(float2* G, const uint8_t* mask, int planes, int ny, int nx, float scale, cudaStream_t s) {
  const int64_t n = (int64_t)ny * nx;
  k_cart_mask_scale<<<dim3((unsigned)((n + 255) / 256), planes), 256, 0, s>>>(G, mask, ny, nx, scale);
}
void launch_spiral_pad(const SpiralOp& op, const float2* x, float2* G, int nb, cudaStream_t s) {
  const int64_t cnt = (int64_t)op.L * op.L;
  k_spiral_pad<<<dim3((unsigned)((cnt + 255) / 256), nb * op.nc), 256, 0, s>>>(op, x, G);
}
void launch_nufft_interp(const SpiralOp& op, const float2* G, float2* y, int nb, cudaStream_t s) {
  k_nufft_interp<<<dim3((unsigned)((op.M + 127) / 128), nb * op.nc), 128, 0, s>>>(op, G, y);
}

// Pre-whitening S' = L^-1 S (Eq. 3) per voxel, FP64 accumulation, in place:
// each thread reads all coils of its voxel before writing any.
__global__ void k_whiten(float2* __restrict__ S, const double2* __restrict__ Li, int nc, int64_t n) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  double2 col[kWhitenMaxCoils];
  for (int k = 0; k < nc; ++k) {
    const float2 a = S[(size_t)k * n + v];
    col[k] = make_double2(a.x, a.y);
  }
  for (int i = 0; i < nc; ++i) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k <= i; ++k) {
      const double2 l = Li[i * nc + k], x = col[k];
      re += l.x * x.x - l.y * x.y;
      im += l.x * x.y + l.y * x.x;
    }
    S[(size_t)i * n + v] = make_float2((float)re, (float)im);
  }
}

void launch_whiten(float2* S, const double2* Li, int nc, int64_t n, cudaStream_t s) {
  k_whiten<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(S, Li, nc, n);
}

}  // namespace pico
