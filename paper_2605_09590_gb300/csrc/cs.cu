// Kernels of the nonlinear compressed-sensing path (Sec. 2.2.5 with an
// L1-wavelet FISTA reconstruction): periodised orthonormal 2-D DWT passes,
// the element-wise FISTA steps, the complex soft threshold and its R-linear
// tangent, the reverse-sweep updates of the VJP, and the 2-D-mask helpers of
// the forward / adjoint encoding operator.
#include "common.cuh"
#include "kernels.cuh"

namespace pico {

namespace {

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---- DWT passes on the top-left nyl x nxl region of n-strided images ----
// analysis along rows: a[k] = sum_m h[m] x[(2k+m) mod nxl], d[k] = sum_m g[m] x[...]; [a | d]
__global__ void k_dwt_rows_fwd(const float2* __restrict__ in, float2* __restrict__ out, int n, int nyl, int nxl,
                               int64_t img, Wavelet w) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int half = nxl / 2;
  if (t >= (int64_t)nyl * half) return;
  const int y = (int)(t / half), k = (int)(t % half);
  const float2* row = in + (size_t)blockIdx.y * img + (size_t)y * n;
  float2 a = make_float2(0.f, 0.f), d = a;
  for (int m = 0; m < w.L; ++m) {
    int j = 2 * k + m;
    if (j >= nxl) j -= nxl;
    const float2 v = row[j];
    a.x = fmaf(w.h[m], v.x, a.x);
    a.y = fmaf(w.h[m], v.y, a.y);
    d.x = fmaf(w.g[m], v.x, d.x);
    d.y = fmaf(w.g[m], v.y, d.y);
  }
  float2* o = out + (size_t)blockIdx.y * img + (size_t)y * n;
  o[k] = a;
  o[half + k] = d;
}

__global__ void k_dwt_cols_fwd(const float2* __restrict__ in, float2* __restrict__ out, int n, int nyl, int nxl,
                               int64_t img, Wavelet w) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int half = nyl / 2;
  if (t >= (int64_t)half * nxl) return;
  const int k = (int)(t / nxl), x = (int)(t % nxl);
  const float2* base = in + (size_t)blockIdx.y * img + x;
  float2 a = make_float2(0.f, 0.f), d = a;
  for (int m = 0; m < w.L; ++m) {
    int j = 2 * k + m;
    if (j >= nyl) j -= nyl;
    const float2 v = base[(size_t)j * n];
    a.x = fmaf(w.h[m], v.x, a.x);
    a.y = fmaf(w.h[m], v.y, a.y);
    d.x = fmaf(w.g[m], v.x, d.x);
    d.y = fmaf(w.g[m], v.y, d.y);
  }
  float2* o = out + (size_t)blockIdx.y * img + x;
  o[(size_t)k * n] = a;
  o[(size_t)(half + k) * n] = d;
}

// synthesis (transpose of the analysis): x[i] = sum over taps m with (i - m) even of
// h[m] a[k] + g[m] d[k], k = ((i - m) mod len) / 2  (gather form, no atomics)
__global__ void k_dwt_rows_inv(const float2* __restrict__ in, float2* __restrict__ out, int n, int nyl, int nxl,
                               int64_t img, Wavelet w) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nyl * nxl) return;
  const int y = (int)(t / nxl), i = (int)(t % nxl);
  const int half = nxl / 2;
  const float2* row = in + (size_t)blockIdx.y * img + (size_t)y * n;
  float2 acc = make_float2(0.f, 0.f);
  for (int m = (i & 1); m < w.L; m += 2) {
    int j = i - m;
    while (j < 0) j += nxl;
    const int k = j / 2;
    const float2 a = row[k], d = row[half + k];
    acc.x = fmaf(w.h[m], a.x, fmaf(w.g[m], d.x, acc.x));
    acc.y = fmaf(w.h[m], a.y, fmaf(w.g[m], d.y, acc.y));
  }
  out[(size_t)blockIdx.y * img + (size_t)y * n + i] = acc;
}

__global__ void k_dwt_cols_inv(const float2* __restrict__ in, float2* __restrict__ out, int n, int nyl, int nxl,
                               int64_t img, Wavelet w) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nyl * nxl) return;
  const int i = (int)(t / nxl), x = (int)(t % nxl);
  const int half = nyl / 2;
  const float2* base = in + (size_t)blockIdx.y * img + x;
  float2 acc = make_float2(0.f, 0.f);
  for (int m = (i & 1); m < w.L; m += 2) {
    int j = i - m;
    while (j < 0) j += nyl;
    const int k = j / 2;
    const float2 a = base[(size_t)k * n], d = base[(size_t)(half + k) * n];
    acc.x = fmaf(w.h[m], a.x, fmaf(w.g[m], d.x, acc.x));
    acc.y = fmaf(w.h[m], a.y, fmaf(w.g[m], d.y, acc.y));
  }
  out[(size_t)blockIdx.y * img + (size_t)i * n + x] = acc;
}

__global__ void k_copy_region(const float2* __restrict__ in, float2* __restrict__ out, int n, int nyl, int nxl,
                              int64_t img) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nyl * nxl) return;
  const int y = (int)(t / nxl), x = (int)(t % nxl);
  const size_t o = (size_t)blockIdx.y * img + (size_t)y * n + x;
  out[o] = in[o];
}

// ---- element-wise FISTA / Jacobian steps (image index i, batch b = blockIdx.y) ----
__device__ __forceinline__ float2 soft1(float2 c, float tau) {
  const float a = sqrtf(c.x * c.x + c.y * c.y);
  if (!(a > tau)) return make_float2(0.f, 0.f);
  return cscale(c, 1.f - tau / a);
}
__device__ __forceinline__ float2 soft_tan1(float2 c, float tau, float2 dc) {
  const float a = sqrtf(c.x * c.x + c.y * c.y);
  if (!(a > tau)) return make_float2(0.f, 0.f);
  const float2 u = cscale(c, 1.f / a);
  const float re = cdot_re(u, dc);  // Re(conj(u) dc)
  const float s = 1.f - tau / a, q = (tau / a) * re;
  return make_float2(fmaf(s, dc.x, q * u.x), fmaf(s, dc.y, q * u.y));
}

// y = z - (Mz - rhs) / Lc ; rhs broadcast when rhs_stride == 0
__global__ void k_cs_gradstep(const float2* __restrict__ z, const float2* __restrict__ Mz,
                              const float2* __restrict__ rhs, int64_t rhs_stride, float inv_lc, float2* __restrict__ y,
                              int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t o = (size_t)blockIdx.y * n + i;
  const float2 r = rhs ? rhs[(size_t)blockIdx.y * rhs_stride + i] : make_float2(0.f, 0.f);
  const float2 zz = z[o], mz = Mz[o];
  y[o] = make_float2(fmaf(-inv_lc, mz.x - r.x, zz.x), fmaf(-inv_lc, mz.y - r.y, zz.y));
}

// primal: threshold the coefficients (batch b = blockIdx.y); `keep` (one image) stores them
// as the linearisation point of the Jacobian
__global__ void k_cs_soft(const float2* c, float2* __restrict__ keep, float2* out, float tau, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t o = (size_t)blockIdx.y * n + i;
  const float2 v = c[o];
  if (keep) keep[i] = v;
  out[o] = soft1(v, tau);
}

// x[b] += alpha y (y one image, broadcast over the batch)
__global__ void k_axpy_bcast(float2* __restrict__ x, const float2* __restrict__ y, float alpha, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t o = (size_t)blockIdx.y * n + i;
  const float2 a = x[o], b = y[i];
  x[o] = make_float2(fmaf(alpha, b.x, a.x), fmaf(alpha, b.y, a.y));
}

// tangent of the soft threshold at the stored coefficients (broadcast over the batch), in place
__global__ void k_cs_soft_tan(const float2* __restrict__ at, float2* __restrict__ dc, float tau, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t o = (size_t)blockIdx.y * n + i;
  dc[o] = soft_tan1(at[i], tau, dc[o]);
}

// z = xn + c (xn - x); x = xn
__global__ void k_cs_momentum(const float2* __restrict__ xn, float2* __restrict__ x, float2* __restrict__ z, float c,
                              int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t o = (size_t)blockIdx.y * n + i;
  const float2 a = xn[o], b = x[o];
  z[o] = make_float2(fmaf(c, a.x - b.x, a.x), fmaf(c, a.y - b.y, a.y));
  x[o] = a;
}

// reverse sweep, first half: xk1 = xbn + (1 + c) zb ; xbn = -c zb
__global__ void k_vjp_a(float2* __restrict__ xbn, const float2* __restrict__ zb, float2* __restrict__ xk1, float c,
                        int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t o = (size_t)blockIdx.y * n + i;
  const float2 z = zb[o], xb = xbn[o];
  xk1[o] = make_float2(fmaf(1.f + c, z.x, xb.x), fmaf(1.f + c, z.y, xb.y));
  xbn[o] = make_float2(-c * z.x, -c * z.y);
}

// reverse sweep, second half: zb = yb - M yb / Lc ; ysum += yb
__global__ void k_vjp_b(const float2* __restrict__ yb, const float2* __restrict__ Myb, float inv_lc,
                        float2* __restrict__ zb, float2* __restrict__ ysum, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t o = (size_t)blockIdx.y * n + i;
  const float2 y = yb[o], m = Myb[o];
  zb[o] = make_float2(fmaf(-inv_lc, m.x, y.x), fmaf(-inv_lc, m.y, y.y));
  const float2 s = ysum[o];
  ysum[o] = make_float2(s.x + y.x, s.y + y.y);
}

__global__ void k_scale(float2* __restrict__ x, float s, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t o = (size_t)blockIdx.y * n + i;
  x[o] = cscale(x[o], s);
}

// 2-D mask: out = mask2d . in . scale (k-space planes)
__global__ void k_mask2d(const float2* __restrict__ in, float2* __restrict__ out, const uint8_t* __restrict__ mask,
                         float scale, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t o = (size_t)blockIdx.y * n + i;
  out[o] = mask[i] ? cscale(in[o], scale) : make_float2(0.f, 0.f);
}

// x[b] = sum_c conj(S_c) . G[b][c]
__global__ void k_coil_combine(const float2* __restrict__ G, const float2* __restrict__ S, int nc,
                               float2* __restrict__ x, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = blockIdx.y;
  float2 acc = make_float2(0.f, 0.f);
  for (int c = 0; c < nc; ++c) acc = cfma_c(acc, S[(size_t)c * n + i], G[((size_t)b * nc + c) * n + i]);
  x[(size_t)b * n + i] = acc;
}

// CN(0, sigma^2) noise on the sampled positions of a 2-D mask, element index (c * ny + ky) * nx + kx
__global__ void k_noise_kspace2d(float2* __restrict__ G, const uint8_t* __restrict__ mask, int nc, int64_t n,
                                 uint64_t seed, int64_t rep_begin, float sigma) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int bc = blockIdx.y, b = bc / nc, c = bc % nc;
  float2 v = make_float2(0.f, 0.f);
  if (mask[i]) {
    const uint64_t key = splitmix64(seed, (uint64_t)(rep_begin + b));
    v = draw_cnoise(key, (uint64_t)c * (uint64_t)n + (uint64_t)i, sigma);
  }
  G[(size_t)bc * n + i] = v;
}

}  // namespace

// The first analysis level covers the whole image, so it reads x directly (x may equal coef).
void launch_dwt(const float2* x, float2* coef, float2* tmp, int n, int levels, int nb, const Wavelet& w,
                cudaStream_t s) {
  const int64_t img = (int64_t)n * n;
  for (int l = 0; l < levels; ++l) {
    const int m = n >> l;
    k_dwt_rows_fwd<<<dim3(blocks((int64_t)m * (m / 2)), nb), 256, 0, s>>>(l == 0 ? x : coef, tmp, n, m, m, img, w);
    k_dwt_cols_fwd<<<dim3(blocks((int64_t)(m / 2) * m), nb), 256, 0, s>>>(tmp, coef, n, m, m, img, w);
  }
}

// Synthesis runs in place on x; with x == coef no copy is needed.
void launch_idwt(const float2* coef, float2* x, float2* tmp, int n, int levels, int nb, const Wavelet& w,
                 cudaStream_t s) {
  const int64_t img = (int64_t)n * n;
  if (coef != x) k_copy_region<<<dim3(blocks(img), nb), 256, 0, s>>>(coef, x, n, n, n, img);
  for (int l = levels - 1; l >= 0; --l) {
    const int m = n >> l;
    k_dwt_cols_inv<<<dim3(blocks((int64_t)m * m), nb), 256, 0, s>>>(x, tmp, n, m, m, img, w);
    k_dwt_rows_inv<<<dim3(blocks((int64_t)m * m), nb), 256, 0, s>>>(tmp, x, n, m, m, img, w);
  }
}

int dwt_kernels(int levels) { return 2 * levels; }
int idwt_kernels(int levels, bool in_place) { return 2 * levels + (in_place ? 0 : 1); }

void launch_cs_gradstep(const float2* z, const float2* Mz, const float2* rhs, int64_t rhs_stride, float inv_lc,
                        float2* y, int64_t n, int nb, cudaStream_t s) {
  k_cs_gradstep<<<dim3(blocks(n), nb), 256, 0, s>>>(z, Mz, rhs, rhs_stride, inv_lc, y, n);
}
void launch_cs_soft(const float2* c, float2* keep, float2* out, float tau, int64_t n, int nb, cudaStream_t s) {
  k_cs_soft<<<dim3(blocks(n), nb), 256, 0, s>>>(c, keep, out, tau, n);
}
void launch_axpy_bcast(float2* x, const float2* y, float alpha, int64_t n, int nb, cudaStream_t s) {
  k_axpy_bcast<<<dim3(blocks(n), nb), 256, 0, s>>>(x, y, alpha, n);
}
void launch_cs_soft_tan(const float2* at, float2* dc, float tau, int64_t n, int nb, cudaStream_t s) {
  k_cs_soft_tan<<<dim3(blocks(n), nb), 256, 0, s>>>(at, dc, tau, n);
}
void launch_cs_momentum(const float2* xn, float2* x, float2* z, float c, int64_t n, int nb, cudaStream_t s) {
  k_cs_momentum<<<dim3(blocks(n), nb), 256, 0, s>>>(xn, x, z, c, n);
}
void launch_vjp_a(float2* xbn, const float2* zb, float2* xk1, float c, int64_t n, int nb, cudaStream_t s) {
  k_vjp_a<<<dim3(blocks(n), nb), 256, 0, s>>>(xbn, zb, xk1, c, n);
}
void launch_vjp_b(const float2* yb, const float2* Myb, float inv_lc, float2* zb, float2* ysum, int64_t n, int nb,
                  cudaStream_t s) {
  k_vjp_b<<<dim3(blocks(n), nb), 256, 0, s>>>(yb, Myb, inv_lc, zb, ysum, n);
}
void launch_scale(float2* x, float sc, int64_t n, int nb, cudaStream_t s) {
  k_scale<<<dim3(blocks(n), nb), 256, 0, s>>>(x, sc, n);
}
void launch_mask2d(const float2* in, float2* out, const uint8_t* mask, float scale, int64_t n, int planes,
                   cudaStream_t s) {
  k_mask2d<<<dim3(blocks(n), planes), 256, 0, s>>>(in, out, mask, scale, n);
}
void launch_coil_combine(const float2* G, const float2* S, int nc, float2* x, int64_t n, int nb, cudaStream_t s) {
  k_coil_combine<<<dim3(blocks(n), nb), 256, 0, s>>>(G, S, nc, x, n);
}
void launch_noise_kspace2d(float2* G, const uint8_t* mask, int nc, int64_t n, int nb, uint64_t seed,
                           int64_t rep_begin, float sigma, cudaStream_t s) {
  k_noise_kspace2d<<<dim3(blocks(n), nb * nc), 256, 0, s>>>(G, mask, nc, n, seed, rep_begin, sigma);
}

}  // namespace pico
