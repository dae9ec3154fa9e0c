// Cartesian SENSE operators on the GPU (kernel templates).
//
// With a phase-encode-only mask the normal operator factorises over readout
// columns (Sec. 2.1.3 operator A^H A with A = M F S; F = F_y (x) F_x and the
// mask acts on ky only, so F^H M F = (F_y^H M_y F_y) (x) I):
//     (A^H A p)[:, x] = sum_c conj(S_c[:, x]) . F_y^H M_y F_y (S_c[:, x] . p[:, x]).
// One CTA owns NC adjacent columns of one image and runs, per coil, a length-ny
// FFT / mask / inverse FFT on each column without leaving the SM.
//
// Column FFT (length N = N1 * N2, index n = n1 + N1 n2, frequency k = k2 + N2 k1):
//   "row jobs"  (one per n1 and column) hold the N2 samples n1 + N1 n2 in registers,
//               run DFT_N2 over n2 and apply the twiddle W_N^(n1 k2);
//   "freq jobs" (one per k2 and column) run DFT_N1 over n1, apply the mask to the
//               frequencies k2 + N2 k1, run the inverse DFT_N1 and the conjugate twiddle;
//   the row jobs finish with the inverse DFT_N2 and the conj(S) coil combine.
// Shared memory is touched twice per FFT pair; the data layout [k2][n1][col]
// keeps every access conflict-free.
#pragma once
#include "common.cuh"
#include "dft_codelets.cuh"
#include "kernels.cuh"

namespace pico {

constexpr int kColTile = 16;  // columns per CTA
constexpr int kRowTile = 16;  // rows per CTA of the row transforms

template <int N1, int N2>
struct ColShape {
  static constexpr int N = N1 * N2;
  // threads: one per (column, job), rounded up to whole warps
  static constexpr int NT = (kColTile * (N1 > N2 ? N1 : N2) + 31) / 32 * 32;
  static constexpr size_t smem = (size_t)N * kColTile * sizeof(float2) + (size_t)N * sizeof(float2) + N * sizeof(float);
};

template <int M1, int M2>
struct RowShape {
  static constexpr int M = M1 * M2;
  static constexpr int PAD = (M1 % 2 == 0) ? 1 : 0;  // odd stride => conflict-free 64-bit accesses
  static constexpr int NT = (kRowTile * (M1 > M2 ? M1 : M2) + 31) / 32 * 32;
  static constexpr size_t smem = (size_t)kRowTile * M2 * (M1 + PAD) * sizeof(float2) + (size_t)M * sizeof(float2);
};

__device__ __forceinline__ const double* cg_rr(const CgArgs& a, int b, int it) {
  return a.rr_part + ((size_t)b * (a.itmax + 1) + it) * a.PB;
}
__device__ __forceinline__ double* cg_pq(const CgArgs& a, int b, int it) {
  return a.pq_part + ((size_t)b * a.itmax + it) * a.PA;
}

// ---------------------------------------------------------------------------
// Normal operator q = (A^H A + lam) p on column tiles.
// CG = true fuses the CG direction update p = r + beta p (beta from the
// per-iteration r^H r partials) and emits the p^H q partial of this tile.
// ---------------------------------------------------------------------------
template <int N1, int N2, bool CG>
__global__ void __launch_bounds__(ColShape<N1, N2>::NT, 1)
    k_col_normal(CartOp op, const float2* __restrict__ xin, float2* __restrict__ yout, float lam, CgArgs a,
                 int it) {
  constexpr int N = N1 * N2;
  constexpr int NT = ColShape<N1, N2>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);  // [N2][N1][kColTile]
  float2* tws = buf + N * kColTile;                 // [N]
  float* ym = reinterpret_cast<float*>(tws + N);    // [N]
  __shared__ double red[(NT + 31) / 32];
  __shared__ float sh_beta;
  __shared__ int sh_done;

  const int t = threadIdx.x;
  const int col = t % kColTile, job = t / kColTile;
  const int b = blockIdx.y;
  const int nx = op.nx;
  const int colg = blockIdx.x * kColTile + col;
  const bool cval = colg < nx;

  for (int i = t; i < N; i += NT) {
    tws[i] = op.tw[i];
    ym[i] = op.ymul[i];
  }
  if (CG) {
    if (t < 32) {
      const double rr = warp_sum_parts(cg_rr(a, b, it), a.PB);
      const double rr0 = warp_sum_parts(cg_rr(a, b, 0), a.PB);
      const double rrp = it > 0 ? warp_sum_parts(cg_rr(a, b, it - 1), a.PB) : 1.0;
      if (t == 0) {
        sh_done = !(rr > a.rtol2 * rr0);
        sh_beta = it > 0 ? (float)(rr / rrp) : 0.f;
      }
    }
  }
  __syncthreads();
  if (CG && sh_done) return;

  const size_t img = (size_t)b * op.ny * nx;
  const bool rowjob = job < N1;
  const bool freqjob = job < N2;
  const int n1 = job, k2 = job;

  float2 p[N2], acc[N2];
  if (rowjob) {
    const float beta = CG ? sh_beta : 0.f;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      const size_t idx = img + (size_t)(n1 + N1 * n2) * nx + colg;
      float2 v = make_float2(0.f, 0.f);
      if (cval) {
        if (CG) {
          const float2 r = a.R[idx];
          if (it > 0) {
            const float2 po = a.P[idx];
            v = make_float2(fmaf(beta, po.x, r.x), fmaf(beta, po.y, r.y));
          } else {
            v = r;
          }
          a.P[idx] = v;
        } else {
          v = xin[idx];
        }
      }
      p[n2] = v;
      acc[n2] = make_float2(0.f, 0.f);
    }
  }

  for (int c = 0; c < op.nc; ++c) {
    const float2* __restrict__ S = op.smaps + (size_t)c * op.ny * nx;
    float2 s[N2];
    if (rowjob) {
      float2 z[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) {
        s[n2] = cval ? __ldg(S + (size_t)(n1 + N1 * n2) * nx + colg) : make_float2(0.f, 0.f);
        z[n2] = cmul(s[n2], p[n2]);
      }
      DFT<N2, -1>::run(z);
#pragma unroll
      for (int k = 0; k < N2; ++k) buf[(k * N1 + n1) * kColTile + col] = k == 0 ? z[0] : cmul(z[k], tws[n1 * k]);
    }
    __syncthreads();
    if (freqjob) {
      float2 y[N1];
#pragma unroll
      for (int m = 0; m < N1; ++m) y[m] = buf[(k2 * N1 + m) * kColTile + col];
      DFT<N1, -1>::run(y);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) y[k1] = cscale(y[k1], ym[k2 + N2 * k1]);
      DFT<N1, 1>::run(y);
#pragma unroll
      for (int m = 0; m < N1; ++m) buf[(k2 * N1 + m) * kColTile + col] = m == 0 ? y[0] : cmul_cb(y[m], tws[m * k2]);
    }
    __syncthreads();
    if (rowjob) {
      float2 z[N2];
#pragma unroll
      for (int k = 0; k < N2; ++k) z[k] = buf[(k * N1 + n1) * kColTile + col];
      DFT<N2, 1>::run(z);
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) acc[n2] = cfma_c(acc[n2], s[n2], z[n2]);
    }
  }

  float pq = 0.f;
  if (rowjob && cval) {
    float2* __restrict__ out = CG ? a.Q : yout;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      const size_t idx = img + (size_t)(n1 + N1 * n2) * nx + colg;
      const float2 q = make_float2(fmaf(lam, p[n2].x, acc[n2].x), fmaf(lam, p[n2].y, acc[n2].y));
      out[idx] = q;
      pq += cdot_re(p[n2], q);
    }
  }
  if (CG) {
    const double tot = block_sum_d((double)pq, red);
    if (t == 0) cg_pq(a, b, it)[blockIdx.x] = tot;
  }
}

// ---------------------------------------------------------------------------
// PMR adjoint, column half: for replica b and coil c draw whitened k-space
// noise on the sampled lines, inverse-transform along y:
//     G[b][c][y][kx] = (1/sqrt(ny nx)) sum_ky mask(ky) n(c, ky, kx) e^{+2 pi i ky y / ny}
// Noise element index e = (c * ny + ky) * nx + kx of replica rep_begin + b.
// ---------------------------------------------------------------------------
template <int N1, int N2>
__global__ void __launch_bounds__(ColShape<N1, N2>::NT, 1)
    k_col_pmr(CartOp op, float2* __restrict__ G, uint64_t seed, int64_t rep_begin, float sigma, float scale) {
  constexpr int N = N1 * N2;
  constexpr int NT = ColShape<N1, N2>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* tws = buf + N * kColTile;

  const int t = threadIdx.x;
  const int col = t % kColTile, job = t / kColTile;
  const int bc = blockIdx.y;  // b * nc + c
  const int c = bc % op.nc, b = bc / op.nc;
  const int nx = op.nx, ny = op.ny;
  const int colg = blockIdx.x * kColTile + col;
  const bool cval = colg < nx;
  for (int i = t; i < N; i += NT) tws[i] = op.tw[i];
  __syncthreads();
  const int n1 = job, k2 = job;
  if (job < N2) {
    const uint64_t key = splitmix64(seed, (uint64_t)(rep_begin + b));
    float2 y[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const int ky = k2 + N2 * k1;
      float2 v = make_float2(0.f, 0.f);
      if (cval && op.mask[ky]) {
        const uint64_t e = ((uint64_t)c * ny + ky) * (uint64_t)nx + colg;
        v = draw_cnoise(key, e, sigma);
      }
      y[k1] = v;
    }
    DFT<N1, 1>::run(y);
#pragma unroll
    for (int m = 0; m < N1; ++m) buf[(k2 * N1 + m) * kColTile + col] = m == 0 ? y[0] : cmul_cb(y[m], tws[m * k2]);
  }
  __syncthreads();
  if (job < N1 && cval) {
    float2 z[N2];
#pragma unroll
    for (int k = 0; k < N2; ++k) z[k] = buf[(k * N1 + n1) * kColTile + col];
    DFT<N2, 1>::run(z);
    float2* __restrict__ g = G + ((size_t)b * op.nc + c) * (size_t)ny * nx;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) g[(size_t)(n1 + N1 * n2) * nx + colg] = cscale(z[n2], scale);
  }
}

// ---------------------------------------------------------------------------
// Row transform with conjugate coil combine:
//     out[b][y][x] = sum_c conj(S_c[y][x]) sum_kx G[b][c][y][kx] e^{+2 pi i kx x / M}
// Rows of length M = M1 * M2 (= nx).  "contiguous jobs" (k2) read the
// frequencies k2 + M2 k1 (coalesced), "strided jobs" (n1) own the outputs
// n1 + M1 n2 for every coil.
// ---------------------------------------------------------------------------
template <int M1, int M2>
__global__ void __launch_bounds__(RowShape<M1, M2>::NT, 1)
    k_row_adjoint(CartOp op, const float2* __restrict__ G, float2* __restrict__ out) {
  constexpr int M = M1 * M2;
  constexpr int NT = RowShape<M1, M2>::NT;
  constexpr int LD = M1 + RowShape<M1, M2>::PAD;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);  // [kRowTile][M2][LD]
  float2* tws = buf + kRowTile * M2 * LD;           // [M]
  const int t = threadIdx.x;
  const int b = blockIdx.y;
  const int ny = op.ny, nx = op.nx;
  for (int i = t; i < M; i += NT) tws[i] = op.twx[i];
  __syncthreads();

  // strided-job identity
  const int ra = t / M1, n1 = t % M1;
  const bool ajob = t < kRowTile * M1;
  const int ya = blockIdx.x * kRowTile + ra;
  const bool aval = ajob && ya < ny;
  // contiguous-job identity
  const int rb = t / M2, k2 = t % M2;
  const bool bjob = t < kRowTile * M2;
  const int yb = blockIdx.x * kRowTile + rb;
  const bool bval = bjob && yb < ny;

  float2 acc[M2];
#pragma unroll
  for (int n2 = 0; n2 < M2; ++n2) acc[n2] = make_float2(0.f, 0.f);

  for (int c = 0; c < op.nc; ++c) {
    if (bjob) {
      float2 y[M1];
      const float2* __restrict__ g = G + (((size_t)b * op.nc + c) * ny + (bval ? yb : 0)) * (size_t)nx;
#pragma unroll
      for (int k1 = 0; k1 < M1; ++k1) y[k1] = bval ? g[k2 + M2 * k1] : make_float2(0.f, 0.f);
      DFT<M1, 1>::run(y);
#pragma unroll
      for (int m = 0; m < M1; ++m) buf[(rb * M2 + k2) * LD + m] = m == 0 ? y[0] : cmul_cb(y[m], tws[m * k2]);
    }
    __syncthreads();
    if (ajob) {
      float2 z[M2];
#pragma unroll
      for (int k = 0; k < M2; ++k) z[k] = buf[(ra * M2 + k) * LD + n1];
      DFT<M2, 1>::run(z);
      if (aval) {
        const float2* __restrict__ S = op.smaps + ((size_t)c * ny + ya) * nx;
#pragma unroll
        for (int n2 = 0; n2 < M2; ++n2) acc[n2] = cfma_c(acc[n2], __ldg(S + n1 + M1 * n2), z[n2]);
      }
    }
    __syncthreads();
  }
  if (aval) {
    float2* __restrict__ o = out + ((size_t)b * ny + ya) * nx;
#pragma unroll
    for (int n2 = 0; n2 < M2; ++n2) o[n1 + M1 * n2] = acc[n2];
  }
}

// ---------------------------------------------------------------------------
// launchers (explicitly instantiated per size in the cart_inst_*.cu units)
// ---------------------------------------------------------------------------
template <int N1, int N2>
void launch_col_normal_t(const CartOp& op, const float2* x, float2* y, int nb, float lam, const CgArgs* a, int it,
                         cudaStream_t s) {
  using Sh = ColShape<N1, N2>;
  const dim3 grid((op.nx + kColTile - 1) / kColTile, nb);
  if (a) {
    auto k = k_col_normal<N1, N2, true>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
    k<<<grid, Sh::NT, Sh::smem, s>>>(op, nullptr, nullptr, lam, *a, it);
  } else {
    auto k = k_col_normal<N1, N2, false>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
    CgArgs dummy{};
    k<<<grid, Sh::NT, Sh::smem, s>>>(op, x, y, lam, dummy, 0);
  }
}

template <int N1, int N2>
void launch_col_pmr_t(const CartOp& op, float2* G, int nb, uint64_t seed, int64_t rep_begin, float sigma,
                      cudaStream_t s) {
  using Sh = ColShape<N1, N2>;
  const dim3 grid((op.nx + kColTile - 1) / kColTile, nb * op.nc);
  auto k = k_col_pmr<N1, N2>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
  const float scale = (float)(1.0 / sqrt((double)op.ny * (double)op.nx));
  k<<<grid, Sh::NT, Sh::smem, s>>>(op, G, seed, rep_begin, sigma, scale);
}

template <int M1, int M2>
void launch_row_adjoint_t(const CartOp& op, const float2* G, float2* out, int nb, cudaStream_t s) {
  using Sh = RowShape<M1, M2>;
  const dim3 grid((op.ny + kRowTile - 1) / kRowTile, nb);
  auto k = k_row_adjoint<M1, M2>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
  k<<<grid, Sh::NT, Sh::smem, s>>>(op, G, out);
}

}  // namespace pico
