// Batched conjugate gradients (Sec. 2.1.3, Eq. 6), PICO/PMR accumulation
// (Alg. 1; PMR), finalisation (Eqs. 10-11) and small vector helpers.
//
// All reductions are deterministic: per-thread FP32 partial over at most
// kVecPerThread products, FP64 from there on, fixed shuffle trees, and the
// per-block partials are summed in a fixed order by every consumer.
#include "common.cuh"
#include "kernels.cuh"

namespace pico {

namespace {

__device__ __forceinline__ const double* rr_at(const CgArgs& a, int b, int it) {
  return a.rr_part + ((size_t)b * (a.itmax + 1) + it) * a.PB;
}
__device__ __forceinline__ double* rr_at_w(const CgArgs& a, int b, int it) {
  return a.rr_part + ((size_t)b * (a.itmax + 1) + it) * a.PB;
}
__device__ __forceinline__ const double* pq_at(const CgArgs& a, int b, int it) {
  return a.pq_part + ((size_t)b * a.itmax + it) * a.PA;
}

// State of one system before CG update `it`: 0 update, 1 converged or
// stopped (||r||^2 <= rtol^2 ||r0||^2), 2 breakdown.  A non-finite residual
// (a NaN or Inf right-hand side or operator) is a breakdown, not convergence;
// so is p^H (M + lam) p <= 0.
__device__ __forceinline__ int cg_state_of(double rr, double rr0, double pq, double rtol2) {
  if (!isfinite(rr) || !isfinite(rr0)) return 2;
  if (!(rr > rtol2 * rr0)) return 1;
  if (!(pq > 0.0) || !isfinite(pq)) return 2;
  return 0;
}

// x = 0, r = probe(b), rr partial
__global__ void __launch_bounds__(kVecThreads) k_cg_init_probe(CgArgs a, uint64_t seed, int64_t probe_begin,
                                                               int kind) {
  __shared__ double scratch[kVecThreads / 32];
  const int b = blockIdx.y;
  const uint64_t key = splitmix64(seed, (uint64_t)(probe_begin + b));
  float2* X = a.X + (size_t)b * a.n;
  float2* R = a.R + (size_t)b * a.n;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < kVecPerThread; ++j) {
    const int64_t i = (int64_t)blockIdx.x * kVecPerBlock + j * kVecThreads + threadIdx.x;
    if (i < a.n) {
      const float2 v = draw_probe(key, (uint64_t)i, kind);
      R[i] = v;
      X[i] = make_float2(0.f, 0.f);
      acc += cdot_re(v, v);
    }
  }
  const double s = block_sum_d((double)acc, scratch);
  if (threadIdx.x == 0) rr_at_w(a, b, 0)[blockIdx.x] = s;
}

// x = 0, r already holds the right-hand side, rr partial
__global__ void __launch_bounds__(kVecThreads) k_cg_init_rhs(CgArgs a) {
  __shared__ double scratch[kVecThreads / 32];
  const int b = blockIdx.y;
  float2* X = a.X + (size_t)b * a.n;
  const float2* R = a.R + (size_t)b * a.n;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < kVecPerThread; ++j) {
    const int64_t i = (int64_t)blockIdx.x * kVecPerBlock + j * kVecThreads + threadIdx.x;
    if (i < a.n) {
      const float2 v = R[i];
      X[i] = make_float2(0.f, 0.f);
      acc += cdot_re(v, v);
    }
  }
  const double s = block_sum_d((double)acc, scratch);
  if (threadIdx.x == 0) rr_at_w(a, b, 0)[blockIdx.x] = s;
}

// alpha = rr/pq; x += alpha p; r -= alpha q; partial of the new r^H r
__global__ void __launch_bounds__(kVecThreads) k_cg_update(CgArgs a, int it) {
  __shared__ double scratch[kVecThreads / 32];
  __shared__ float sh_alpha;
  __shared__ int sh_state;  // 0 update, 1 converged/stopped, 2 breakdown
  const int b = blockIdx.y;
  if (threadIdx.x < 32) {
    const double rr = warp_sum_parts(rr_at(a, b, it), a.PB);
    const double rr0 = warp_sum_parts(rr_at(a, b, 0), a.PB);
    const double pq = warp_sum_parts(pq_at(a, b, it), a.PA);
    if (threadIdx.x == 0) {
      sh_state = cg_state_of(rr, rr0, pq, a.rtol2);
      sh_alpha = (float)(rr / pq);
    }
  }
  __syncthreads();
  if (sh_state == 1) {
    // converged (or stopped): carry this block's r^H r partial forward so that
    // every later iteration of this system sees the same, converged value
    if (threadIdx.x == 0) rr_at_w(a, b, it + 1)[blockIdx.x] = rr_at(a, b, it)[blockIdx.x];
    return;
  }
  if (sh_state == 2) {
    // CG breakdown: record it and make the probe look converged from here on.
    if (threadIdx.x == 0) {
      rr_at_w(a, b, it + 1)[blockIdx.x] = 0.0;
      if (blockIdx.x == 0) a.status[b] = 5;
    }
    return;
  }
  const float alpha = sh_alpha;
  float2* X = a.X + (size_t)b * a.n;
  float2* R = a.R + (size_t)b * a.n;
  const float2* P = a.P + (size_t)b * a.n;
  const float2* Q = a.Q + (size_t)b * a.n;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < kVecPerThread; ++j) {
    const int64_t i = (int64_t)blockIdx.x * kVecPerBlock + j * kVecThreads + threadIdx.x;
    if (i < a.n) {
      const float2 p = P[i], q = Q[i];
      float2 x = X[i], r = R[i];
      x.x = fmaf(alpha, p.x, x.x);
      x.y = fmaf(alpha, p.y, x.y);
      r.x = fmaf(-alpha, q.x, r.x);
      r.y = fmaf(-alpha, q.y, r.y);
      X[i] = x;
      R[i] = r;
      acc += cdot_re(r, r);
    }
  }
  const double s = block_sum_d((double)acc, scratch);
  if (threadIdx.x == 0) rr_at_w(a, b, it + 1)[blockIdx.x] = s;
}

// Per-system CG step of iteration it, once per system: state 0 update,
// 1 converged / stopped, 2 breakdown; alpha = rr / pq.
__global__ void k_cg_alpha(CgArgs a, int it, float* alpha, int* state) {
  const int b = blockIdx.x;
  const double rr = warp_sum_parts(rr_at(a, b, it), a.PB);
  const double rr0 = warp_sum_parts(rr_at(a, b, 0), a.PB);
  const double pq = warp_sum_parts(pq_at(a, b, it), a.PA);
  if (threadIdx.x == 0) {
    state[b] = cg_state_of(rr, rr0, pq, a.rtol2);
    alpha[b] = (float)(rr / pq);
  }
}

// x += alpha p; r -= alpha q with the per-system scalars of k_cg_alpha; two
// complex values per 16-byte access (n even), the same blocks of
// kVecPerBlock values and the same r^H r partials as k_cg_update.
__global__ void __launch_bounds__(kVecThreads) k_cg_update_v(CgArgs a, int it, const float* __restrict__ alpha_b,
                                                             const int* __restrict__ state_b) {
  __shared__ double scratch[kVecThreads / 32];
  const int b = blockIdx.y;
  const int st = state_b[b];
  if (st == 1) {
    if (threadIdx.x == 0) rr_at_w(a, b, it + 1)[blockIdx.x] = rr_at(a, b, it)[blockIdx.x];
    return;
  }
  if (st == 2) {
    if (threadIdx.x == 0) {
      rr_at_w(a, b, it + 1)[blockIdx.x] = 0.0;
      if (blockIdx.x == 0) a.status[b] = 5;
    }
    return;
  }
  const float alpha = alpha_b[b];
  float4* X = reinterpret_cast<float4*>(a.X + (size_t)b * a.n);
  float4* R = reinterpret_cast<float4*>(a.R + (size_t)b * a.n);
  const float4* P = reinterpret_cast<const float4*>(a.P + (size_t)b * a.n);
  const float4* Q = reinterpret_cast<const float4*>(a.Q + (size_t)b * a.n);
  const int64_t n4 = a.n / 2;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < kVecPerThread / 2; ++j) {
    const int64_t i = (int64_t)blockIdx.x * (kVecPerBlock / 2) + j * kVecThreads + threadIdx.x;
    if (i < n4) {
      const float4 p = P[i], q = Q[i];
      float4 x = X[i], r = R[i];
      x.x = fmaf(alpha, p.x, x.x);
      x.y = fmaf(alpha, p.y, x.y);
      x.z = fmaf(alpha, p.z, x.z);
      x.w = fmaf(alpha, p.w, x.w);
      r.x = fmaf(-alpha, q.x, r.x);
      r.y = fmaf(-alpha, q.y, r.y);
      r.z = fmaf(-alpha, q.z, r.z);
      r.w = fmaf(-alpha, q.w, r.w);
      X[i] = x;
      R[i] = r;
      acc += fmaf(r.x, r.x, r.y * r.y) + fmaf(r.z, r.z, r.w * r.w);
    }
  }
  const double s = block_sum_d((double)acc, scratch);
  if (threadIdx.x == 0) rr_at_w(a, b, it + 1)[blockIdx.x] = s;
}

// The same update with x advanced once per two iterations, for operators that
// keep the last two directions (the tensor-core Gram path): mode 0 (iteration
// it even) updates r only; mode 1 (it odd) applies the pending x += alpha_prev
// p_prev, then x += alpha p and r -= alpha q; mode 2 only applies the pending
// x update (after a solve that ended on an even iteration).  The x values are
// the same bits as with one update per iteration (the same two FMAs per value
// in the same order); one pass over x is saved per pair of iterations.
__global__ void __launch_bounds__(kVecThreads)
    k_cg_update_pair(CgArgs a, int it, const float* __restrict__ alpha_b, const int* __restrict__ state_b,
                     const float* __restrict__ alpha_prev_b, const int* __restrict__ state_prev_b,
                     const float2* __restrict__ p_prev, int mode) {
  __shared__ double scratch[kVecThreads / 32];
  const int b = blockIdx.y;
  const int st = mode == 2 ? 1 : state_b[b];
  const bool pend = mode != 0 && state_prev_b[b] == 0;
  const bool upd = st == 0;
  const float alpha = upd ? alpha_b[b] : 0.f, ap = pend ? alpha_prev_b[b] : 0.f;
  float4* X = reinterpret_cast<float4*>(a.X + (size_t)b * a.n);
  float4* R = reinterpret_cast<float4*>(a.R + (size_t)b * a.n);
  const float4* P = reinterpret_cast<const float4*>(a.P + (size_t)b * a.n);
  const float4* PP = reinterpret_cast<const float4*>(p_prev + (size_t)b * a.n);
  const float4* Q = reinterpret_cast<const float4*>(a.Q + (size_t)b * a.n);
  const int64_t n4 = a.n / 2;
  const bool xpass = pend || (upd && mode == 1);
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < kVecPerThread / 2; ++j) {
    const int64_t i = (int64_t)blockIdx.x * (kVecPerBlock / 2) + j * kVecThreads + threadIdx.x;
    if (i < n4) {
      if (xpass) {
        float4 x = X[i];
        if (pend) {
          const float4 p = PP[i];
          x.x = fmaf(ap, p.x, x.x);
          x.y = fmaf(ap, p.y, x.y);
          x.z = fmaf(ap, p.z, x.z);
          x.w = fmaf(ap, p.w, x.w);
        }
        if (upd && mode == 1) {
          const float4 p = P[i];
          x.x = fmaf(alpha, p.x, x.x);
          x.y = fmaf(alpha, p.y, x.y);
          x.z = fmaf(alpha, p.z, x.z);
          x.w = fmaf(alpha, p.w, x.w);
        }
        X[i] = x;
      }
      if (upd) {
        const float4 q = Q[i];
        float4 r = R[i];
        r.x = fmaf(-alpha, q.x, r.x);
        r.y = fmaf(-alpha, q.y, r.y);
        r.z = fmaf(-alpha, q.z, r.z);
        r.w = fmaf(-alpha, q.w, r.w);
        R[i] = r;
        acc += fmaf(r.x, r.x, r.y * r.y) + fmaf(r.z, r.z, r.w * r.w);
      }
    }
  }
  if (mode == 2) return;
  if (st == 1) {
    if (threadIdx.x == 0) rr_at_w(a, b, it + 1)[blockIdx.x] = rr_at(a, b, it)[blockIdx.x];
    return;
  }
  if (st == 2) {
    if (threadIdx.x == 0) {
      rr_at_w(a, b, it + 1)[blockIdx.x] = 0.0;
      if (blockIdx.x == 0) a.status[b] = 5;
    }
    return;
  }
  const double sum = block_sum_d((double)acc, scratch);
  if (threadIdx.x == 0) rr_at_w(a, b, it + 1)[blockIdx.x] = sum;
}

// flag = 1 when every system of the batch meets the stopping rule at iteration
// it (or has broken down, which zeroes its r^H r); cleared by any other
__global__ void k_cg_all_done(CgArgs a, int it, int* flag) {
  const int b = blockIdx.x;
  const double rr = warp_sum_parts(rr_at(a, b, it), a.PB);
  const double rr0 = warp_sum_parts(rr_at(a, b, 0), a.PB);
  if (threadIdx.x == 0 && rr > a.rtol2 * rr0) atomicExch(flag, 0);
}

// iterations performed and final relative residual per right-hand side
__global__ void k_cg_report(CgArgs a, int max_iter, int* iters, double* relres) {
  const int b = blockIdx.x;
  if (threadIdx.x >= 32) return;
  const double rr0 = warp_sum_parts(rr_at(a, b, 0), a.PB);
  int it = 0;
  double rr = rr0;
  while (it < max_iter) {
    if (!(rr > a.rtol2 * rr0)) break;
    // update `it` happened (or broke down); its result is rr(it+1)
    rr = warp_sum_parts(rr_at(a, b, it + 1), a.PB);
    ++it;
  }
  if (threadIdx.x == 0) {
    iters[b] = it;
    relres[b] = !isfinite(rr0) ? (double)NAN : rr0 > 0.0 ? sqrt(rr / rr0) : 0.0;
  }
}

// s += sum_b Re(conj(v_b) x_b), ss += sum_b (.)^2 ; fixed order over b
__global__ void __launch_bounds__(kVecThreads) k_accum_pico(const float2* __restrict__ X, int64_t n, int nb,
                                                            uint64_t seed, int64_t probe_begin, int kind,
                                                            double* __restrict__ sum, double* __restrict__ sumsq) {
  const int64_t i = (int64_t)blockIdx.x * kVecThreads + threadIdx.x;
  if (i >= n) return;
  double s = sum[i];
  double ss = sumsq ? sumsq[i] : 0.0;
  for (int b = 0; b < nb; ++b) {
    const uint64_t key = splitmix64(seed, (uint64_t)(probe_begin + b));
    const float2 v = draw_probe(key, (uint64_t)i, kind);
    const float d = cdot_re(v, X[(size_t)b * n + i]);
    s += (double)d;
    ss += (double)d * (double)d;
  }
  sum[i] = s;
  if (sumsq) sumsq[i] = ss;
}

// s += sum_b |x_b|^2 / sigma^2
__global__ void __launch_bounds__(kVecThreads) k_accum_pmr(const float2* __restrict__ X, int64_t n, int nb,
                                                           float inv_sigma2, double* __restrict__ sum,
                                                           double* __restrict__ sumsq) {
  const int64_t i = (int64_t)blockIdx.x * kVecThreads + threadIdx.x;
  if (i >= n) return;
  double s = sum[i];
  double ss = sumsq ? sumsq[i] : 0.0;
  for (int b = 0; b < nb; ++b) {
    const float2 x = X[(size_t)b * n + i];
    const float d = cdot_re(x, x) * inv_sigma2;
    s += (double)d;
    ss += (double)d * (double)d;
  }
  sum[i] = s;
  if (sumsq) sumsq[i] = ss;
}

// var = s / N ; stderr of the mean = sqrt((ss/N - (s/N)^2) / (N - 1))
__global__ void k_finalize(const double* sum, const double* sumsq, int64_t n, int64_t count, float* var,
                           float* se) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double m = sum[i] / (double)count;
  if (var) var[i] = (float)m;
  if (se) {
    double v = 0.0;
    if (sumsq && count > 1) v = fmax(sumsq[i] / (double)count - m * m, 0.0) / (double)(count - 1);
    se[i] = (float)sqrt(v);
  }
}

// partial sums over voxels of (s/N)^2 and the squared standard error of the mean
__global__ void __launch_bounds__(256) k_stderr_parts(const double* sum, const double* sumsq, int64_t n,
                                                      int64_t count, double* part) {
  __shared__ double scratch[8];
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const double m = sum[i] / (double)count;
    const double v = fmax(sumsq[i] / (double)count - m * m, 0.0) / (double)(count - 1);
    a += m * m;
    b += v;
  }
  const double ta = block_sum_d(a, scratch);
  const double tb = block_sum_d(b, scratch);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ta;
    part[2 * blockIdx.x + 1] = tb;
  }
}

__global__ void k_gfactor(const float* va, const float* vr, int64_t n, double R, float* g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  g[i] = (float)sqrt((double)va[i] / (R * (double)vr[i]));
}

__global__ void __launch_bounds__(kVecThreads) k_norm2_part(const float2* x, int64_t n, double* part) {
  __shared__ double scratch[kVecThreads / 32];
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < kVecPerThread; ++j) {
    const int64_t i = (int64_t)blockIdx.x * kVecPerBlock + j * kVecThreads + threadIdx.x;
    if (i < n) acc += cdot_re(x[i], x[i]);
  }
  const double s = block_sum_d((double)acc, scratch);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kVecThreads) k_scale_by_norm(const float2* y, float2* x, int64_t n,
                                                               const double* part, int nparts, double* norm_out) {
  __shared__ float sh_inv;
  if (threadIdx.x < 32) {
    const double s = warp_sum_parts(part, nparts);
    if (threadIdx.x == 0) {
      const double nr = sqrt(s);
      sh_inv = (float)(1.0 / nr);
      if (blockIdx.x == 0 && norm_out) *norm_out = nr;
    }
  }
  __syncthreads();
  const float inv = sh_inv;
#pragma unroll
  for (int j = 0; j < kVecPerThread; ++j) {
    const int64_t i = (int64_t)blockIdx.x * kVecPerBlock + j * kVecThreads + threadIdx.x;
    if (i < n) x[i] = cscale(y[i], inv);
  }
}

__global__ void k_fill_probe(float2* x, int64_t n, uint64_t seed, int64_t index, float scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t key = splitmix64(seed, (uint64_t)index);
  x[i] = cscale(draw_probe(key, (uint64_t)i, kProbePhase), scale);
}

inline int vec_blocks(int64_t n) { return (int)((n + kVecPerBlock - 1) / kVecPerBlock); }

}  // namespace

void launch_cg_init_probe(const CgArgs& a, int nb, uint64_t seed, int64_t probe_begin, int kind, cudaStream_t s) {
  k_cg_init_probe<<<dim3(a.PB, nb), kVecThreads, 0, s>>>(a, seed, probe_begin, kind);
}
void launch_cg_init_rhs(const CgArgs& a, int nb, cudaStream_t s) {
  k_cg_init_rhs<<<dim3(a.PB, nb), kVecThreads, 0, s>>>(a);
}
void launch_cg_update(const CgArgs& a, int nb, int it, cudaStream_t s) {
  k_cg_update<<<dim3(a.PB, nb), kVecThreads, 0, s>>>(a, it);
}
bool launch_cg_step(const CgArgs& a, int nb, int it, float* alpha, int* state, cudaStream_t s) {
  if (a.n % 2) return false;
  k_cg_alpha<<<nb, 32, 0, s>>>(a, it, alpha, state);
  k_cg_update_v<<<dim3(a.PB, nb), kVecThreads, 0, s>>>(a, it, alpha, state);
  return true;
}
bool launch_cg_step_pair(const CgArgs& a, int nb, int it, float* alpha, int* state, const float* alpha_prev,
                         const int* state_prev, const float2* p_prev, cudaStream_t s) {
  if (a.n % 2) return false;
  k_cg_alpha<<<nb, 32, 0, s>>>(a, it, alpha, state);
  k_cg_update_pair<<<dim3(a.PB, nb), kVecThreads, 0, s>>>(a, it, alpha, state, alpha_prev, state_prev, p_prev,
                                                          it & 1);
  return true;
}
void launch_cg_flush_pair(const CgArgs& a, int nb, const float* alpha_prev, const int* state_prev,
                          const float2* p_prev, cudaStream_t s) {
  if (nb > 0)
    k_cg_update_pair<<<dim3(a.PB, nb), kVecThreads, 0, s>>>(a, 0, alpha_prev, state_prev, alpha_prev, state_prev,
                                                            p_prev, 2);
}
void launch_cg_all_done(const CgArgs& a, int nb, int it, int* flag, cudaStream_t s) {
  cudaMemsetAsync(flag, 0xFF, sizeof(int), s);  // nonzero: all done unless a block clears it
  k_cg_all_done<<<nb, 32, 0, s>>>(a, it, flag);
}
void launch_cg_report(const CgArgs& a, int nb, int max_iter, int* iters, double* relres, cudaStream_t s) {
  k_cg_report<<<nb, 32, 0, s>>>(a, max_iter, iters, relres);
}
void launch_accum_pico(const float2* X, int64_t n, int nb, uint64_t seed, int64_t probe_begin, int kind,
                       double* sum, double* sumsq, cudaStream_t s) {
  k_accum_pico<<<(unsigned)((n + kVecThreads - 1) / kVecThreads), kVecThreads, 0, s>>>(X, n, nb, seed, probe_begin,
                                                                                        kind, sum, sumsq);
}
void launch_accum_pmr(const float2* X, int64_t n, int nb, float inv_sigma2, double* sum, double* sumsq,
                      cudaStream_t s) {
  k_accum_pmr<<<(unsigned)((n + kVecThreads - 1) / kVecThreads), kVecThreads, 0, s>>>(X, n, nb, inv_sigma2, sum,
                                                                                       sumsq);
}
void launch_finalize(const double* sum, const double* sumsq, int64_t n, int64_t count, float* var, float* se,
                     cudaStream_t s) {
  k_finalize<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sum, sumsq, n, count, var, se);
}
void launch_stderr_parts(const double* sum, const double* sumsq, int64_t n, int64_t count, double* part, int nblk,
                         cudaStream_t s) {
  k_stderr_parts<<<nblk, 256, 0, s>>>(sum, sumsq, n, count, part);
}
void launch_gfactor(const float* va, const float* vr, int64_t n, double R, float* g, cudaStream_t s) {
  k_gfactor<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(va, vr, n, R, g);
}
void launch_norm2_part(const float2* x, int64_t n, double* part, cudaStream_t s) {
  k_norm2_part<<<vec_blocks(n), kVecThreads, 0, s>>>(x, n, part);
}
void launch_scale_by_norm(const float2* y, float2* x, int64_t n, const double* part, int nparts, double* norm_out,
                          cudaStream_t s) {
  k_scale_by_norm<<<vec_blocks(n), kVecThreads, 0, s>>>(y, x, n, part, nparts, norm_out);
}
void launch_fill_probe(float2* x, int64_t n, uint64_t seed, int64_t index, float scale, cudaStream_t s) {
  k_fill_probe<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, seed, index, scale);
}

}  // namespace pico
