// Spiral set-up kernels (Toeplitz point-spread kernel), Kaiser-Bessel gridding
// of PMR noise, and host dispatch of the templated spiral passes.
#include "common.cuh"
#include "kernels.cuh"
#include "spiral_sizes.h"

namespace pico {

template <int P1, int P2>
void launch_toep_normal_t(const SpiralOp&, const float2*, float2*, float2*, int, float, const CgArgs*, int,
                          cudaStream_t);
template <int P1, int P2>
void launch_fft2_t(float2*, const float2*, int, int, bool, cudaStream_t);
template <int P1, int P2>
void launch_grid_cols_adjoint_t(const SpiralOp&, const float2*, float2*, int, cudaStream_t);

namespace {

constexpr int kStrip = 8;     // consecutive dx per thread in the kernel sum
constexpr int kChunk = 256;   // samples staged in shared memory at a time

// h(d) = sum_m e^{+2 pi i (kx_m dx + ky_m dy) / n} on the circular 2n grid
// (scaled later).  Grid row gy holds dy = gy (gy < n) or gy - 2n (gy > n);
// row/column n is zero.  One thread: one row, kStrip consecutive columns; the
// phase of the first column is reduced in FP64, the rest follow by rotation;
// each chunk of kChunk samples is summed in FP32 (at most kChunk unit-modulus
// terms) and the chunk sums are accumulated in FP64 in sample order -- FP64
// arithmetic runs at a small fraction of the FP32 rate on this part.
__global__ void __launch_bounds__(256) k_toep_h(const float* __restrict__ traj, int64_t M, int n, float2* c) {
  __shared__ float2 s_k[kChunk];
  __shared__ float2 s_rot[kChunk];
  const int L = 2 * n;
  const int strips = L / kStrip;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = tid < (int64_t)L * strips;
  const int gy = active ? (int)(tid / strips) : 0;
  const int gx0 = active ? (int)(tid % strips) * kStrip : 0;
  const int dy = gy < n ? gy : gy - L;
  const int dx0 = gx0 < n ? gx0 : gx0 - L;
  double accx[kStrip], accy[kStrip];
#pragma unroll
  for (int j = 0; j < kStrip; ++j) accx[j] = accy[j] = 0.0;
  for (int64_t m0 = 0; m0 < M; m0 += kChunk) {
    __syncthreads();
    for (int i = threadIdx.x; i < kChunk; i += blockDim.x) {
      const int64_t m = m0 + i;
      float2 kk = make_float2(0.f, 0.f), rot = make_float2(1.f, 0.f);
      if (m < M) {
        kk = make_float2(traj[2 * m], traj[2 * m + 1]);
        double fr = (double)kk.x / (double)n;
        fr -= floor(fr);
        float s, cs;
        sincospif(2.0f * (float)fr, &s, &cs);
        rot = make_float2(cs, s);
      }
      s_k[i] = kk;
      s_rot[i] = rot;
    }
    __syncthreads();
    const int cnt = (int)((M - m0) < kChunk ? (M - m0) : kChunk);
    if (active) {
      float fx[kStrip], fy[kStrip];
#pragma unroll
      for (int j = 0; j < kStrip; ++j) fx[j] = fy[j] = 0.f;
      for (int i = 0; i < cnt; ++i) {
        const float2 kk = s_k[i];
        double ph = ((double)kk.x * dx0 + (double)kk.y * dy) / (double)n;
        ph -= floor(ph);
        float s, cs;
        sincospif(2.0f * (float)ph, &s, &cs);
        float2 w = make_float2(cs, s);
        const float2 r = s_rot[i];
#pragma unroll
        for (int j = 0; j < kStrip; ++j) {
          fx[j] += w.x;
          fy[j] += w.y;
          w = cmul(w, r);
        }
      }
#pragma unroll
      for (int j = 0; j < kStrip; ++j) {
        accx[j] += (double)fx[j];
        accy[j] += (double)fy[j];
      }
    }
  }
  if (!active) return;
#pragma unroll
  for (int j = 0; j < kStrip; ++j) {
    const int gx = gx0 + j;
    const bool zero = gy == n || gx == n;
    c[(size_t)gy * L + gx] = zero ? make_float2(0.f, 0.f) : make_float2((float)accx[j], (float)accy[j]);
  }
}

__global__ void k_toep_finalize(const float2* c, int64_t count, float scale, float* T) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) T[i] = c[i].x * scale;
}

// Gather-form Kaiser-Bessel gridding of PMR noise onto the 2n grid.
// CTA: one 16x16 grid tile, one replica, kCoilGroup coils; thread = grid point.
// The kernel is separable, phi(dx) phi(dy), and its 1-D weights at the integer
// offsets of a sample's window (kMaxTaps of them, zero outside |d| <= W/2)
// depend on the trajectory alone: k_grid_table evaluates them once per
// sample at set-up.  Per staged chunk of a tile's samples the block copies
// their weights and draws their noise (every thread one (sample, coil) pair),
// then every grid point looks its two weights up -- no Bessel evaluation in
// the gridding itself.
constexpr int kCoilGroup = 4;
constexpr int kMaxTaps = 10;  // window integers for kb_width <= 8, plus one

__global__ void k_grid_table(SpiralOp op, float* __restrict__ gw, int2* __restrict__ go) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= op.M) return;
  const int L = op.L;
  const float hw = op.halfw;
  const int ntaps = min(kMaxTaps, (int)(2.f * hw) + 2);
  const float2 u = op.u[m];
  const int ix0 = (int)floorf(u.x - hw), iy0 = (int)floorf(u.y - hw);
  for (int k = 0; k < kMaxTaps; ++k) {
    float wx = 0.f, wy = 0.f;
    if (k < ntaps) {
      const float dx = (float)(ix0 + k) - u.x, dy = (float)(iy0 + k) - u.y;
      if (fabsf(dx) <= hw) wx = cyl_bessel_i0f(op.beta * sqrtf(fmaxf(0.f, 1.f - (dx / hw) * (dx / hw)))) * op.inv_i0beta;
      if (fabsf(dy) <= hw) wy = cyl_bessel_i0f(op.beta * sqrtf(fmaxf(0.f, 1.f - (dy / hw) * (dy / hw)))) * op.inv_i0beta;
    }
    gw[m * 2 * kMaxTaps + k] = wx;
    gw[m * 2 * kMaxTaps + kMaxTaps + k] = wy;
  }
  go[m] = make_int2(((ix0 % L) + L) % L, ((iy0 % L) + L) % L);
}

__global__ void __launch_bounds__(256) k_grid_pmr(SpiralOp op, float2* __restrict__ Q, uint64_t seed,
                                                  int64_t rep_begin, float sigma, const float2* __restrict__ data) {
  __shared__ float s_wx[kChunk][kMaxTaps];
  __shared__ float s_wy[kChunk][kMaxTaps];
  __shared__ int2 s_o[kChunk];               // wrapped first grid index of each window (x, y)
  __shared__ int s_m[kChunk];                // sample index
  __shared__ float2 s_w[kChunk][kCoilGroup];
  const int L = op.L;
  const int tiles_x = L / 16;
  const int tile = blockIdx.x;
  const int b = blockIdx.y;
  const int c0 = blockIdx.z * kCoilGroup;
  const int ty = tile / tiles_x, tx = tile % tiles_x;
  const int gy = ty * 16 + threadIdx.x / 16, gx = tx * 16 + threadIdx.x % 16;
  const uint64_t key = splitmix64(seed, (uint64_t)(rep_begin + b));
  const int beg = op.tile_ptr[tile], end = op.tile_ptr[tile + 1];
  float2 acc[kCoilGroup];
#pragma unroll
  for (int g = 0; g < kCoilGroup; ++g) acc[g] = make_float2(0.f, 0.f);
  const float hw = op.halfw;
  const int ntaps = min(kMaxTaps, (int)(2.f * hw) + 2);
  for (int p0 = beg; p0 < end; p0 += kChunk) {
    __syncthreads();
    const int cnt = min(kChunk, end - p0);
    if ((int)threadIdx.x < cnt) {
      const int m = op.tile_idx[p0 + threadIdx.x];
      s_m[threadIdx.x] = m;
      s_o[threadIdx.x] = op.go[m];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt * 2 * kMaxTaps; j += blockDim.x) {
      const int i = j / (2 * kMaxTaps), k = j - i * (2 * kMaxTaps);
      const float w = op.gw[(size_t)s_m[i] * (2 * kMaxTaps) + k];
      if (k < kMaxTaps)
        s_wx[i][k] = w;
      else
        s_wy[i][k - kMaxTaps] = w;
    }
    for (int j = threadIdx.x; j < cnt * kCoilGroup; j += blockDim.x) {
      const int i = j / kCoilGroup, g = j - i * kCoilGroup;
      const int m = s_m[i], c = c0 + g;
      float2 v = make_float2(0.f, 0.f);
      if (c < op.nc) {
        const uint64_t e = (uint64_t)c * (uint64_t)op.M + (uint64_t)m;
        v = cmul(data ? data[(size_t)b * op.nc * op.M + e] : draw_cnoise(key, e, sigma), op.cphase[m]);
      }
      s_w[i][g] = v;
    }
    __syncthreads();
    for (int i = 0; i < cnt; ++i) {
      const int2 o = s_o[i];
      int kx = gx - o.x, ky = gy - o.y;
      if (kx < 0) kx += L;
      if (ky < 0) ky += L;
      if (kx < ntaps && ky < ntaps) {
        const float wgt = s_wx[i][kx] * s_wy[i][ky];
        if (wgt != 0.f) {
#pragma unroll
          for (int g = 0; g < kCoilGroup; ++g) {
            acc[g].x = fmaf(wgt, s_w[i][g].x, acc[g].x);
            acc[g].y = fmaf(wgt, s_w[i][g].y, acc[g].y);
          }
        }
      }
    }
  }
#pragma unroll
  for (int g = 0; g < kCoilGroup; ++g) {
    const int c = c0 + g;
    if (c < op.nc) Q[(((size_t)b * op.nc + c) * L + gy) * L + gx] = acc[g];
  }
}

}  // namespace

bool spiral_supported(int n, int* P1, int* P2) {
#define PICO_SPLIT(LL, A, B) \
  if (2 * n == LL) {         \
    *P1 = A;                 \
    *P2 = B;                 \
    return n % kStrip == 0;  \
  }
  PICO_GRID_SIZES(PICO_SPLIT)
#undef PICO_SPLIT
  return false;
}

bool grid_split(int L, int* P1, int* P2) {
#define PICO_SPLIT(LL, A, B) \
  if (L == LL) {             \
    *P1 = A;                 \
    *P2 = B;                 \
    return true;             \
  }
  PICO_GRID_SIZES(PICO_SPLIT)
#undef PICO_SPLIT
  return false;
}

void launch_toep_h(const float* traj, int64_t M, int n, float2* c, cudaStream_t s) {
  const int64_t threads = (int64_t)(2 * n) * (2 * n / kStrip);
  k_toep_h<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(traj, M, n, c);
}

void launch_toep_fft2(const SpiralOp& op, float2* c, cudaStream_t s) {
#define PICO_CASE(LL, A, B)                               \
  if (op.P1 == A && op.P2 == B) {                         \
    launch_fft2_t<A, B>(c, op.tw2, 1, -1, true, s);       \
    launch_fft2_t<A, B>(c, op.tw2, 1, -1, false, s);      \
    return;                                               \
  }
  PICO_GRID_SIZES(PICO_CASE)
#undef PICO_CASE
}

void launch_toep_finalize(const float2* c, int L, float scale, float* T, cudaStream_t s) {
  const int64_t cnt = (int64_t)L * L;
  k_toep_finalize<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(c, cnt, scale, T);
}

void launch_toep_apply(const SpiralOp& op, const float2* x, float2* y, float2* G, int nb, float lam, cudaStream_t s) {
#define PICO_CASE(LL, A, B) \
  if (op.P1 == A && op.P2 == B) return launch_toep_normal_t<A, B>(op, x, y, G, nb, lam, nullptr, 0, s);
  PICO_GRID_SIZES(PICO_CASE)
#undef PICO_CASE
}

void launch_toep_cg_normal(const SpiralOp& op, const CgArgs& a, float2* G, int nb, int it, float lam,
                           cudaStream_t s) {
#define PICO_CASE(LL, A, B) \
  if (op.P1 == A && op.P2 == B) return launch_toep_normal_t<A, B>(op, nullptr, nullptr, G, nb, lam, &a, it, s);
  PICO_GRID_SIZES(PICO_CASE)
#undef PICO_CASE
}

size_t grid_table_floats(int64_t M) { return (size_t)M * 2 * kMaxTaps; }

void launch_grid_table(const SpiralOp& op, float* gw, int2* go, cudaStream_t s) {
  if (op.M > 0) k_grid_table<<<(unsigned)((op.M + 255) / 256), 256, 0, s>>>(op, gw, go);
}

void launch_grid_pmr(const SpiralOp& op, float2* Q, int nb, uint64_t seed, int64_t rep_begin, float sigma,
                     cudaStream_t s, const float2* data) {
  const int tiles = (op.L / 16) * (op.L / 16);
  const dim3 grid(tiles, nb, (op.nc + kCoilGroup - 1) / kCoilGroup);
  k_grid_pmr<<<grid, 256, 0, s>>>(op, Q, seed, rep_begin, sigma, data);
}

void launch_grid_adjoint_rest(const SpiralOp& op, float2* Q, float2* out, int nb, cudaStream_t s) {
#define PICO_CASE(LL, A, B)                                        \
  if (op.P1 == A && op.P2 == B) {                                  \
    launch_fft2_t<A, B>(Q, op.tw2, nb * op.nc, 1, true, s);        \
    launch_grid_cols_adjoint_t<A, B>(op, Q, out, nb, s);           \
    return;                                                        \
  }
  PICO_GRID_SIZES(PICO_CASE)
#undef PICO_CASE
}

}  // namespace pico
