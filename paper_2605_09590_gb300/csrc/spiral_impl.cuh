// Non-Cartesian (spiral) operators on the GPU (kernel templates).
//
// Normal operator by Toeplitz embedding (Sec. 3.2.2 / Sec. 3.3, Fessler 2005):
// for an N x N image and the exact NUDFT A_c = E diag(S_c),
//     A^H A x = sum_c conj(S_c) . crop_N IDFT_2N( T^ . DFT_2N( pad_2N(S_c . x) ) )
// where T^ = DFT_2N of the point-spread kernel h(d) = (1/N^2) sum_m e^{+2 pi i k_m.d/N},
// d in (-N, N)^2, placed circularly on the 2N grid (its DFT is real because h
// is Hermitian).  Three passes per normal operator, all on the 2N grid:
//   rows_fwd : per image row and coil, S_c . p zero-padded to 2N, row FFT  -> G[b][c][N][2N]
//   cols     : per grid column and coil, column FFT (rows >= N are zero), x T^,
//              inverse column FFT, rows < N written back in place
//   rows_inv : per image row, inverse row FFT of every coil, first N samples,
//              conj(S_c) coil combine, + lam p, p^H q partial
// The CG direction update p = r + beta p is fused into rows_fwd.
//
// PMR adjoint A^H n (Sec. 1; Kaiser-Bessel gridding, width W, oversampling 2):
//   grid     : gather-form gridding of CN(0, sigma^2) k-space noise drawn per
//              (replica, coil, sample) onto the 2N grid, no atomics
//   fft rows : inverse row FFT of the grid
//   cols_adj : inverse column FFT, centred crop, deapodisation, conj(S_c)
//              coil combine
#pragma once
#include "common.cuh"
#include "fft_blocks.cuh"
#include "kernels.cuh"
#include "tc_util.cuh"

namespace pico {

__device__ __forceinline__ const double* sp_rr(const CgArgs& a, int b, int it) {
  return a.rr_part + ((size_t)b * (a.itmax + 1) + it) * a.PB;
}
__device__ __forceinline__ double* sp_pq(const CgArgs& a, int b, int it) {
  return a.pq_part + ((size_t)b * a.itmax + it) * a.PA;
}

// CG scalars of iteration it (computed by warp 0): returns done flag and beta
__device__ __forceinline__ void cg_scalars(const CgArgs& a, int b, int it, int* sh_done, float* sh_beta) {
  if (threadIdx.x < 32) {
    const double rr = warp_sum_parts(sp_rr(a, b, it), a.PB);
    const double rr0 = warp_sum_parts(sp_rr(a, b, 0), a.PB);
    const double rrp = it > 0 ? warp_sum_parts(sp_rr(a, b, it - 1), a.PB) : 1.0;
    if (threadIdx.x == 0) {
      *sh_done = !(rr > a.rtol2 * rr0);
      *sh_beta = it > 0 ? (float)(rr / rrp) : 0.f;
    }
  }
}

// Row-pass blocks of RL image rows: RL = 16 (one block of up to 480 threads
// per SM) or RL = 4 (a quarter of the threads, four blocks per SM, so that
// the blocks' global loads and stores overlap one another's transforms).
template <int P1, int P2, int RL>
struct RowSplit {
  static constexpr int NT = (RL * (P1 > P2 ? P1 : P2) + 31) / 32 * 32;
  static constexpr int MINB = RL <= 4 ? 4 : RL <= 8 ? 2 : 1;
  static constexpr size_t buf = (size_t)RL * P2 * Split<P1, P2>::LD * sizeof(float2);
};

// ---------------------------------------------------------------------------
// Pass 1: rows of the image, forward transform of S_c . p padded to L = 2N
// ---------------------------------------------------------------------------
// PAD: the grid is 2N (Toeplitz embedding, image in the first half of each
// line); otherwise L = N (2-D Cartesian masks: plain 2-D DFT, no padding).
template <int P1, int P2, bool CG, bool PAD, int RL>
__global__ void __launch_bounds__(RowSplit<P1, P2, RL>::NT, RowSplit<P1, P2, RL>::MINB)
    k_toep_rows_fwd(SpiralOp op, const float2* __restrict__ xin, float2* __restrict__ G, CgArgs a, int it) {
  constexpr int NIN = PAD ? P2 / 2 : P2;  // samples n1 + P1 n2 inside the image: n2 < NIN
  constexpr int L = P1 * P2;
  constexpr int NT = RowSplit<P1, P2, RL>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* tws = buf + RL * P2 * Split<P1, P2>::LD;
  __shared__ float sh_beta;
  __shared__ int sh_done;
  const int t = threadIdx.x, b = blockIdx.y, N = op.n;
  for (int i = t; i < L; i += NT) tws[i] = op.tw2[i];
  if (CG) cg_scalars(a, b, it, &sh_done, &sh_beta);
  __syncthreads();
  if (CG && blockIdx.x == 0 && t == 0 && a.done) a.done[b] = sh_done;  // for the column pass
  if (CG && sh_done) return;

  const int ra = t / P1, n1 = t % P1;
  const bool ajob = t < RL * P1;
  const int ya = blockIdx.x * RL + ra;
  const bool aval = ajob && ya < N;
  const int rb = t / P2, k2 = t % P2;
  const bool bjob = t < RL * P2;
  const int yb = blockIdx.x * RL + rb;
  const bool bval = bjob && yb < N;
  const size_t img = (size_t)b * N * N;

  float2 p[P2];
  if (ajob) {
    const float beta = CG ? sh_beta : 0.f;
#pragma unroll
    for (int n2 = 0; n2 < P2; ++n2) {
      const int x = n1 + P1 * n2;
      float2 v = make_float2(0.f, 0.f);
      if (aval && n2 < NIN) {
        const size_t idx = img + (size_t)ya * N + x;
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
    }
  }
  for (int c = 0; c < op.nc; ++c) {
    if (ajob) {
      float2 z[P2];
      const float2* __restrict__ S = op.smaps + ((size_t)c * N + (aval ? ya : 0)) * N;
#pragma unroll
      for (int n2 = 0; n2 < P2; ++n2) {
        const int x = n1 + P1 * n2;
        z[n2] = (aval && n2 < NIN) ? cmul(__ldg(S + x), p[n2]) : make_float2(0.f, 0.f);
      }
      rowa_store<P1, P2, -1, NIN>(z, n1, ra, buf, tws);
    }
    __syncthreads();
    if (bval) {
      float2 y[P1];
      rowb_load<P1, P2, -1>(y, k2, rb, buf);
      float2* __restrict__ g = G + (((size_t)b * op.nc + c) * N + yb) * L;
#pragma unroll
      for (int k1 = 0; k1 < P1; ++k1) g[k2 + P2 * k1] = y[k1];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Pass 2: columns of the grid: FFT (rows >= N zero), x T^, inverse FFT, rows < N
// ---------------------------------------------------------------------------
// done: per-image stop flags of the CG iteration (nullptr outside CG); planes of
// converged images are skipped
template <int P1, int P2, bool PAD>
__global__ void __launch_bounds__(Split<P1, P2>::NT, 1)
    k_toep_cols(SpiralOp op, float2* __restrict__ G, const int* __restrict__ done) {
  constexpr int NIN = PAD ? P2 / 2 : P2;
  constexpr int L = P1 * P2;
  constexpr int NT = Split<P1, P2>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* tws = buf + L * kLines;
  const int t = threadIdx.x, N = op.n;
  if (done && done[blockIdx.y / op.nc]) return;
  for (int i = t; i < L; i += NT) tws[i] = op.tw2[i];
  __syncthreads();
  const int ln = t % kLines, job = t / kLines;
  const int kx = blockIdx.x * kLines + ln;  // grid column (always < L: L is a multiple of 16)
  float2* __restrict__ g = G + (size_t)blockIdx.y * N * L;  // (b, c) plane [N][L]
  const int n1 = job, k2 = job;
  if (job < P1) {
    float2 z[P2];
#pragma unroll
    for (int n2 = 0; n2 < P2; ++n2) {
      const int y = n1 + P1 * n2;  // rows >= N (n2 >= NIN) are the zero padding
      z[n2] = n2 < NIN ? g[(size_t)y * L + kx] : make_float2(0.f, 0.f);
    }
    cola_store<P1, P2, -1, NIN>(z, n1, ln, buf, tws);
  }
  __syncthreads();
  if (job < P2) {
    float2 y[P1];
    colb_load<P1, P2>(y, k2, ln, buf);
    DFT<P1, -1>::run(y);
#pragma unroll
    for (int k1 = 0; k1 < P1; ++k1) y[k1] = cscale(y[k1], __ldg(op.That + (size_t)(k2 + P2 * k1) * L + kx));
    colb_inv_store<P1, P2>(y, k2, ln, buf, tws);
  }
  __syncthreads();
  if (job < P1) {
    float2 z[P2];
    cola_load<P1, P2, 1>(z, n1, ln, buf);
#pragma unroll
    for (int n2 = 0; n2 < NIN; ++n2) g[(size_t)(n1 + P1 * n2) * L + kx] = z[n2];  // rows < N only
  }
}

// The same pass for splits with P1 > P2, persistent: each block walks work
// items (plane, group of P1 grid columns) and one thread brings the next
// item's N x P1 input values into a staging buffer with TMA tensor loads
// while the block transforms the current item, so the global-load latency of
// a plane no longer stalls every thread at its start.  With P1 columns per
// item the b-jobs (the heavy DFT_P1 pair and the T^ product) occupy all
// P2 x P1 threads; the light DFT_P2 a-jobs take P1 / P2 rounds.
template <int P1, int P2, bool PAD>
__global__ void __launch_bounds__(P1 * P2, (P1 * P2 <= 320 ? 2 : 1))
    k_toep_cols_w(SpiralOp op, const __grid_constant__ CUtensorMap mG, float2* __restrict__ G,
                  const int* __restrict__ done, int nplanes, int box_rows) {
  constexpr int NIN = PAD ? P2 / 2 : P2;
  constexpr int L = P1 * P2;
  constexpr int NT = L;
  constexpr int CL = P1;  // grid columns per item
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  const int t = threadIdx.x, N = op.n;          // N input rows per plane
  float2* stage = reinterpret_cast<float2*>(sm);  // [N][CL] input rows of the item
  float2* buf = stage + (size_t)N * CL;           // [k2][n1][CL]
  float2* tws = buf + (size_t)L * CL;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tws + L);
  int* arrived = reinterpret_cast<int*>(bar + 1);
  const int items = P2 * nplanes;
  const uint32_t bytes = (uint32_t)N * CL * sizeof(float2);
  if (t == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  for (int i = t; i < L; i += NT) tws[i] = op.tw2[i];
  __syncthreads();
  auto issue = [&](int w) {
    const int plane = w / P2, cg = w - plane * P2;
    tc::mbar_expect_tx(bar, bytes);
    for (int r0 = 0; r0 < N; r0 += box_rows) tc::tma_load_3d(stage + (size_t)r0 * CL, &mG, bar, cg * CL, r0, plane);
  };
  if (t == 0 && (int)blockIdx.x < items) issue(blockIdx.x);
  int phase = 0;
  for (int w = blockIdx.x; w < items; w += gridDim.x, phase ^= 1) {
    const int plane = w / P2, cg = w - plane * P2, x0 = cg * CL;
    // One thread decides whether the item's copy arrived and the block
    // follows that decision together.  On a timeout it records the error,
    // waits once more (bounded) for the copy still in flight into this
    // block's shared memory, and the whole block leaves at the same point.
    if (t == 0) {
      bool ok = tc::mbar_wait(bar, phase);
      if (!ok) {
        if (op.err) atomicCAS(op.err, 0, 10);
        tc::mbar_wait(bar, phase);
      }
      *arrived = ok ? 1 : 0;
    }
    __syncthreads();
    if (!*arrived) return;
    const bool skip = done && done[plane / op.nc];
    float2* __restrict__ g = G + (size_t)plane * N * L;  // (b, c) plane [N][L]
    if (!skip)
      for (int jj = t; jj < P1 * CL; jj += NT) {
        const int n1 = jj / CL, ln = jj - n1 * CL;
        float2 z[P2];
#pragma unroll
        for (int n2 = 0; n2 < P2; ++n2) z[n2] = n2 < NIN ? stage[(n1 + P1 * n2) * CL + ln] : make_float2(0.f, 0.f);
        cola_store<P1, P2, -1, NIN, CL>(z, n1, ln, buf, tws);
      }
    __syncthreads();  // the staging buffer is free: fetch the next item
    if (t == 0 && w + (int)gridDim.x < items) issue(w + gridDim.x);
    if (!skip) {
      {
        const int k2 = t / CL, ln = t - k2 * CL, kx = x0 + ln;
        float2 y[P1];
        colb_load<P1, P2, CL>(y, k2, ln, buf);
        DFT<P1, -1>::run(y);
#pragma unroll
        for (int k1 = 0; k1 < P1; ++k1) y[k1] = cscale(y[k1], __ldg(op.That + (size_t)(k2 + P2 * k1) * L + kx));
        colb_inv_store<P1, P2, CL>(y, k2, ln, buf, tws);
      }
      __syncthreads();
      for (int jj = t; jj < P1 * CL; jj += NT) {
        const int n1 = jj / CL, ln = jj - n1 * CL;
        float2 z[P2];
        cola_load<P1, P2, 1, CL>(z, n1, ln, buf);
#pragma unroll
        for (int n2 = 0; n2 < NIN; ++n2) g[(size_t)(n1 + P1 * n2) * L + x0 + ln] = z[n2];  // rows < N only
      }
    }
    __syncthreads();  // buf is rewritten by the next item
  }
}

// ---------------------------------------------------------------------------
// Pass 3: rows: inverse FFT per coil, first N samples, conj(S) combine, + lam p
// ---------------------------------------------------------------------------
template <int P1, int P2, bool CG, bool PAD, int RL>
__global__ void __launch_bounds__(RowSplit<P1, P2, RL>::NT, RowSplit<P1, P2, RL>::MINB)
    k_toep_rows_inv(SpiralOp op, const float2* __restrict__ G, const float2* __restrict__ xin,
                    float2* __restrict__ yout, float lam, CgArgs a, int it) {
  constexpr int NIN = PAD ? P2 / 2 : P2;
  constexpr int L = P1 * P2;
  constexpr int NT = RowSplit<P1, P2, RL>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* tws = buf + RL * P2 * Split<P1, P2>::LD;
  __shared__ double red[(NT + 31) / 32];
  __shared__ float sh_beta;
  __shared__ int sh_done;
  const int t = threadIdx.x, b = blockIdx.y, N = op.n;
  for (int i = t; i < L; i += NT) tws[i] = op.tw2[i];
  if (CG) cg_scalars(a, b, it, &sh_done, &sh_beta);
  __syncthreads();
  if (CG && sh_done) return;

  const int ra = t / P1, n1 = t % P1;
  const bool ajob = t < RL * P1;
  const int ya = blockIdx.x * RL + ra;
  const bool aval = ajob && ya < N;
  const int rb = t / P2, k2 = t % P2;
  const bool bjob = t < RL * P2;
  const int yb = blockIdx.x * RL + rb;
  const bool bval = bjob && yb < N;
  const size_t img = (size_t)b * N * N;

  float2 acc[NIN];
#pragma unroll
  for (int n2 = 0; n2 < NIN; ++n2) acc[n2] = make_float2(0.f, 0.f);
  for (int c = 0; c < op.nc; ++c) {
    if (bjob) {
      float2 y[P1];
      const float2* __restrict__ g = G + (((size_t)b * op.nc + c) * N + (bval ? yb : 0)) * L;
#pragma unroll
      for (int k1 = 0; k1 < P1; ++k1) y[k1] = bval ? g[k2 + P2 * k1] : make_float2(0.f, 0.f);
      rowb_inv_store<P1, P2>(y, k2, rb, buf, tws);
    }
    __syncthreads();
    if (ajob) {
      float2 z[P2];
      rowa_inv_load<P1, P2>(z, n1, ra, buf);
      if (aval) {
        const float2* __restrict__ S = op.smaps + ((size_t)c * N + ya) * N;
#pragma unroll
        for (int n2 = 0; n2 < NIN; ++n2) acc[n2] = cfma_c(acc[n2], __ldg(S + n1 + P1 * n2), z[n2]);
      }
    }
    __syncthreads();
  }
  float pq = 0.f;
  if (aval) {
    const float2* __restrict__ pin = CG ? a.P : xin;
    float2* __restrict__ out = CG ? a.Q : yout;
#pragma unroll
    for (int n2 = 0; n2 < NIN; ++n2) {
      const int x = n1 + P1 * n2;
      {
        const size_t idx = img + (size_t)ya * N + x;
        const float2 pv = pin[idx];
        const float2 q = make_float2(fmaf(lam, pv.x, acc[n2].x), fmaf(lam, pv.y, acc[n2].y));
        out[idx] = q;
        pq += cdot_re(pv, q);
      }
    }
  }
  if (CG) {
    const double tot = block_sum_d((double)pq, red);
    if (t == 0) sp_pq(a, b, it)[blockIdx.x] = tot;
  }
}

// ---------------------------------------------------------------------------
// Generic in-place FFTs of all rows / all columns of [planes][L][L] grids
// ---------------------------------------------------------------------------
template <int P1, int P2, int SIGN>
__global__ void __launch_bounds__(Split<P1, P2>::NT, 1) k_fft_rows(float2* __restrict__ data, const float2* tw2) {
  constexpr int L = P1 * P2;
  constexpr int NT = Split<P1, P2>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* tws = buf + kLines * P2 * Split<P1, P2>::LD;
  const int t = threadIdx.x;
  for (int i = t; i < L; i += NT) tws[i] = tw2[i];
  __syncthreads();
  float2* __restrict__ plane = data + (size_t)blockIdx.y * L * L;
  const int ra = t / P1, n1 = t % P1;
  const int rb = t / P2, k2 = t % P2;
  if (t < kLines * P1) {
    float2 z[P2];
    const float2* row = plane + (size_t)(blockIdx.x * kLines + ra) * L;
#pragma unroll
    for (int n2 = 0; n2 < P2; ++n2) z[n2] = row[n1 + P1 * n2];
    rowa_store<P1, P2, SIGN>(z, n1, ra, buf, tws);
  }
  __syncthreads();
  if (t < kLines * P2) {
    float2 y[P1];
    rowb_load<P1, P2, SIGN>(y, k2, rb, buf);
    float2* row = plane + (size_t)(blockIdx.x * kLines + rb) * L;
#pragma unroll
    for (int k1 = 0; k1 < P1; ++k1) row[k2 + P2 * k1] = y[k1];
  }
}

template <int P1, int P2, int SIGN>
__global__ void __launch_bounds__(Split<P1, P2>::NT, 1) k_fft_cols(float2* __restrict__ data, const float2* tw2) {
  constexpr int L = P1 * P2;
  constexpr int NT = Split<P1, P2>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* tws = buf + L * kLines;
  const int t = threadIdx.x;
  for (int i = t; i < L; i += NT) tws[i] = tw2[i];
  __syncthreads();
  float2* __restrict__ plane = data + (size_t)blockIdx.y * L * L;
  const int ln = t % kLines, job = t / kLines;
  const int kx = blockIdx.x * kLines + ln;
  if (job < P1) {
    float2 z[P2];
#pragma unroll
    for (int n2 = 0; n2 < P2; ++n2) z[n2] = plane[(size_t)(job + P1 * n2) * L + kx];
    cola_store<P1, P2, SIGN>(z, job, ln, buf, tws);
  }
  __syncthreads();
  if (job < P2) {
    float2 y[P1];
    colb_load<P1, P2>(y, job, ln, buf);
    DFT<P1, SIGN>::run(y);
#pragma unroll
    for (int k1 = 0; k1 < P1; ++k1) plane[(size_t)(job + P2 * k1) * L + kx] = y[k1];
  }
}

// ---------------------------------------------------------------------------
// PMR adjoint, last pass: inverse column FFT of the (row-transformed) grid,
// centred crop to the N x N image, deapodisation and conj(S_c) coil combine.
// Image column x reads grid column (x - N/2) mod L; image row y is grid row
// (y - N/2) mod L.  One CTA: 16 image columns of one replica, all coils.
// ---------------------------------------------------------------------------
template <int P1, int P2>
__global__ void __launch_bounds__(Split<P1, P2>::NT, 1)
    k_grid_cols_adjoint(SpiralOp op, const float2* __restrict__ Q, float2* __restrict__ out) {
  constexpr int L = P1 * P2;
  constexpr int NT = Split<P1, P2>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* tws = buf + L * kLines;
  const int t = threadIdx.x, N = op.n, b = blockIdx.y;
  for (int i = t; i < L; i += NT) tws[i] = op.tw2[i];
  __syncthreads();
  const int ln = t % kLines, job = t / kLines;
  const int x = blockIdx.x * kLines + ln;  // image column
  const bool xval = x < N;
  const int gx = ((x - N / 2) % L + L) % L;
  const float dax = xval ? op.deapod[x] : 0.f;
  float2 acc[P1];
#pragma unroll
  for (int k1 = 0; k1 < P1; ++k1) acc[k1] = make_float2(0.f, 0.f);
  for (int c = 0; c < op.nc; ++c) {
    const float2* __restrict__ q = Q + ((size_t)b * op.nc + c) * L * L;
    if (job < P1) {
      float2 z[P2];
#pragma unroll
      for (int n2 = 0; n2 < P2; ++n2) z[n2] = xval ? q[(size_t)(job + P1 * n2) * L + gx] : make_float2(0.f, 0.f);
      cola_store<P1, P2, 1>(z, job, ln, buf, tws);
    }
    __syncthreads();
    if (job < P2 && xval) {
      float2 y[P1];
      colb_load<P1, P2>(y, job, ln, buf);
      DFT<P1, 1>::run(y);
#pragma unroll
      for (int k1 = 0; k1 < P1; ++k1) {
        const int gy = job + P2 * k1;
        const int yy = (gy + N / 2) % L;  // image row of grid row gy
        if (yy < N) {
          const float2 s = __ldg(op.smaps + ((size_t)c * N + yy) * N + x);
          acc[k1] = cfma_c(acc[k1], s, cscale(y[k1], dax * op.deapod[yy]));
        }
      }
    }
    __syncthreads();
  }
  if (job < P2 && xval) {
#pragma unroll
    for (int k1 = 0; k1 < P1; ++k1) {
      const int gy = job + P2 * k1;
      const int yy = (gy + N / 2) % L;
      if (yy < N) out[((size_t)b * N + yy) * N + x] = acc[k1];
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// Row passes of RL image rows per block (grid: ceil(n / RL) row blocks per
// image; the p^H q partials of the inverse pass, one per row block, fill the
// context's ceil(n / RL) slots).
template <int P1, int P2, bool PAD, int RL>
void toep_rows_fwd_launch(const SpiralOp& op, const float2* x, float2* G, int nb, const CgArgs* a, int it,
                          cudaStream_t s) {
  using Rs = RowSplit<P1, P2, RL>;
  const size_t smr = Rs::buf + P1 * P2 * sizeof(float2);
  const dim3 grow((op.n + RL - 1) / RL, nb);
  if (a) {
    auto k1 = k_toep_rows_fwd<P1, P2, true, PAD, RL>;
    cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
    k1<<<grow, Rs::NT, smr, s>>>(op, nullptr, G, *a, it);
  } else {
    CgArgs dummy{};
    auto k1 = k_toep_rows_fwd<P1, P2, false, PAD, RL>;
    cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
    k1<<<grow, Rs::NT, smr, s>>>(op, x, G, dummy, 0);
  }
}
template <int P1, int P2, bool PAD, int RL>
void toep_rows_inv_launch(const SpiralOp& op, const float2* x, float2* y, const float2* G, int nb, float lam,
                          const CgArgs* a, int it, cudaStream_t s) {
  using Rs = RowSplit<P1, P2, RL>;
  const size_t smr = Rs::buf + P1 * P2 * sizeof(float2);
  const dim3 grow((op.n + RL - 1) / RL, nb);
  if (a) {
    auto k3 = k_toep_rows_inv<P1, P2, true, PAD, RL>;
    cudaFuncSetAttribute(k3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
    k3<<<grow, Rs::NT, smr, s>>>(op, G, nullptr, nullptr, lam, *a, it);
  } else {
    CgArgs dummy{};
    auto k3 = k_toep_rows_inv<P1, P2, false, PAD, RL>;
    cudaFuncSetAttribute(k3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
    k3<<<grow, Rs::NT, smr, s>>>(op, G, x, y, lam, dummy, 0);
  }
}

template <int P1, int P2, bool PAD>
void toep_normal_impl(const SpiralOp& op, const float2* x, float2* y, float2* G, int nb, float lam, const CgArgs* a,
                      int it, cudaStream_t s) {
  using Sp = Split<P1, P2>;
  constexpr int L = P1 * P2;
  const size_t smc = Sp::col_buf + L * sizeof(float2);
  if (op.row_lines == 4)
    toep_rows_fwd_launch<P1, P2, PAD, 4>(op, x, G, nb, a, it, s);
  else
    toep_rows_fwd_launch<P1, P2, PAD, kLines>(op, x, G, nb, a, it, s);
  // persistent column pass (P1 > P2): N rows staged per item, TMA boxes of at
  // most 256 rows, every TMA destination 128-byte aligned
  bool wide = false;
  if constexpr (P1 > P2) {
    const int box_rows = op.n <= 256 ? op.n : op.n / 2;
    CUtensorMap mG{};
    const size_t smw = 1024 + ((size_t)op.n * P1 + (size_t)L * P1 + L) * sizeof(float2) + 16;
    wide = op.n % box_rows == 0 && ((size_t)box_rows * P1 * 8) % 128 == 0 && smw <= 227 * 1024 &&
           encode_plane_map(&mG, G, op.n, L, (int64_t)nb * op.nc, P1, box_rows);
    if (wide) {
      auto k2 = k_toep_cols_w<P1, P2, PAD>;
      static thread_local int bps = 0;
      cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
      if (bps == 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k2, L, smw) != cudaSuccess) bps = 1;
      int dev = 0, nsm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      const int64_t items = (int64_t)P2 * nb * op.nc;
      const int grid = (int)std::min<int64_t>(items, (int64_t)std::max(1, bps) * std::max(1, nsm));
      k2<<<grid, L, smw, s>>>(op, mG, G, a ? a->done : nullptr, nb * op.nc, box_rows);
    }
  }
  if (!wide) {
    auto k2 = k_toep_cols<P1, P2, PAD>;
    cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
    k2<<<dim3(L / kLines, nb * op.nc), Sp::NT, smc, s>>>(op, G, a ? a->done : nullptr);
  }
  if (op.row_lines == 4)
    toep_rows_inv_launch<P1, P2, PAD, 4>(op, x, y, G, nb, lam, a, it, s);
  else
    toep_rows_inv_launch<P1, P2, PAD, kLines>(op, x, y, G, nb, lam, a, it, s);
}

template <int P1, int P2>
void launch_toep_normal_t(const SpiralOp& op, const float2* x, float2* y, float2* G, int nb, float lam,
                          const CgArgs* a, int it, cudaStream_t s) {
  if (op.L == 2 * op.n)
    toep_normal_impl<P1, P2, true>(op, x, y, G, nb, lam, a, it, s);
  else
    toep_normal_impl<P1, P2, false>(op, x, y, G, nb, lam, a, it, s);
}

template <int P1, int P2>
void launch_fft2_t(float2* data, const float2* tw2, int planes, int sign, bool rows, cudaStream_t s) {
  using Sp = Split<P1, P2>;
  constexpr int L = P1 * P2;
  if (rows) {
    const size_t sm = Sp::row_buf + L * sizeof(float2);
    auto k = sign < 0 ? k_fft_rows<P1, P2, -1> : k_fft_rows<P1, P2, 1>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k<<<dim3(L / kLines, planes), Sp::NT, sm, s>>>(data, tw2);
  } else {
    const size_t sm = Sp::col_buf + L * sizeof(float2);
    auto k = sign < 0 ? k_fft_cols<P1, P2, -1> : k_fft_cols<P1, P2, 1>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k<<<dim3(L / kLines, planes), Sp::NT, sm, s>>>(data, tw2);
  }
}

template <int P1, int P2>
void launch_grid_cols_adjoint_t(const SpiralOp& op, const float2* Q, float2* out, int nb, cudaStream_t s) {
  using Sp = Split<P1, P2>;
  constexpr int L = P1 * P2;
  const size_t sm = Sp::col_buf + L * sizeof(float2);
  auto k = k_grid_cols_adjoint<P1, P2>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k<<<dim3((op.n + kLines - 1) / kLines, nb), Sp::NT, sm, s>>>(op, Q, out);
}

}  // namespace pico
