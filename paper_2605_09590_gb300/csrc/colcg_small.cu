// Per-column CG with the whole solve on chip, for small Cartesian images.
//
// With a phase-encode mask A^H A is block diagonal over the readout columns
// (Sec. 2.1.3 with F^H M F = (F_y^H M_y F_y) (x) I): column j of every image is
// acted on by the dense Hermitian ny x ny matrix
//   G_j[y, y'] = P[y - y'] sum_c conj(S_c[y, j]) S_c[y', j],
//   P[d] = (1/ny) sum_k m_k exp(2 pi i k d / ny),
// so CG on Eq. 6 splits into independent column systems (G_j + lam I) x_j = b_j.
// For ny <= 96 a block holds G_j (ny^2 complex64, at most 72 KB) and the CG
// vectors x, r, p, q of a group of images of that column in shared memory and
// runs every CG update of the solve in one launch: a latency-bound workload
// (64 x 64 images, 32 probes) then needs one kernel per solve instead of
// three per update.  Inner products take exact float products summed in
// float-float within a warp and FP64 across warps and columns (fixed-order
// reductions, so the result does not depend on the launch shape; the FP64
// pipe, a small fraction of the FP32 rate, would otherwise bound the solve);
// each column stops on its own test ||r_j|| <= rtol ||b_j||.
#include "common.cuh"
#include "kernels.cuh"

namespace pico {

namespace {

constexpr int kSmallThreads = 256;

// G_j of every column in the plain layout [nx][ny][ny] (row y, column y'),
// FP64 sums over the coils, then rounded to complex64.
__global__ void k_colcg_small_build(const float2* __restrict__ S, const double2* __restrict__ P, int nc, int ny,
                                    int nx, float2* __restrict__ G) {
  const int j = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ny * ny) return;
  const int y = t / ny, yp = t % ny;
  const int64_t n = (int64_t)ny * nx;
  double re = 0.0, im = 0.0;
  for (int c = 0; c < nc; ++c) {
    const float2 a = S[c * n + (int64_t)y * nx + j], b = S[c * n + (int64_t)yp * nx + j];
    re += (double)a.x * b.x + (double)a.y * b.y;  // conj(a) b
    im += (double)a.x * b.y - (double)a.y * b.x;
  }
  int d = y - yp;
  if (d < 0) d += ny;
  const double2 p = P[d];
  G[((size_t)j * ny + y) * ny + yp] = make_float2((float)(p.x * re - p.y * im), (float)(p.x * im + p.y * re));
}

// Sum over the NY rows of every image of a per-element value held by the
// thread that owns element e = k * kSmallThreads + tid (image e / NY, row
// e % NY): a warp's 32 elements belong to one image; warp sums (float-float)
// go to red[t][w] as doubles, then thread t adds its NY / 32 slots in order.
// `un[t]` undoes the power-of-two scaling of image t's values (sum * 2^un[t]).
template <int NY, int T>
__device__ __forceinline__ void image_sums(const ffloat (&v)[NY * T / kSmallThreads], double* red, const int* un,
                                           double* out) {
  constexpr int E = NY * T / kSmallThreads;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const ffloat s = warp_sum_ff(v[k]);
    const int e = k * kSmallThreads + threadIdx.x;
    if (lane == 0) red[(e / NY) * (NY / 32) + (e % NY) / 32] = (double)s.hi + (double)s.lo;
  }
  __syncthreads();
  if (threadIdx.x < T) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NY / 32; ++w) s += red[threadIdx.x * (NY / 32) + w];
    out[threadIdx.x] = s * __longlong_as_double((long long)(1023 + un[threadIdx.x]) << 52);  // exact: |un| <= 240
  }
  __syncthreads();
}

// Largest |component| over the NY rows of every image (same element ownership
// as image_sums); thread t < T gets its image's value.
template <int NY, int T>
__device__ __forceinline__ float image_max(const float (&v)[NY * T / kSmallThreads], float* red) {
  constexpr int E = NY * T / kSmallThreads;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < E; ++k) {
    float m = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int e = k * kSmallThreads + threadIdx.x;
    if (lane == 0) red[(e / NY) * (NY / 32) + (e % NY) / 32] = m;
  }
  __syncthreads();
  float m = 0.f;
  if (threadIdx.x < T)
    for (int w = 0; w < NY / 32; ++w) m = fmaxf(m, red[threadIdx.x * (NY / 32) + w]);
  __syncthreads();
  return m;
}

// Power-of-two scaling keeps the float-float products clear of FP32 underflow
// and overflow: values are multiplied by 2^e before the exact products and the
// sum by 2^-e afterwards (both exact in the normal range).
__device__ __forceinline__ int clamp_exp(int e) { return e < -120 ? -120 : (e > 120 ? 120 : e); }
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
// binary exponent e of a > 0 with a = m 2^e, m in [0.5, 1) (normal doubles;
// every value here is a sum of squares of floats, far above the subnormals)
__device__ __forceinline__ int exp_of(double a) {
  return (int)((__double_as_longlong(a) >> 52) & 0x7ff) - 1022;
}
// e with a * 2^e in [0.5, 1) (0 for zero or non-finite a)
__device__ __forceinline__ int inv_exp(double a) {
  if (!(a > 0.0) || !isfinite(a)) return 0;
  return clamp_exp(-exp_of(a));
}
// e with ||r|| * 2^e near 1, from rr = ||r||^2
__device__ __forceinline__ int inv_exp_sqrt(double rr) {
  if (!(rr > 0.0) || !isfinite(rr)) return 0;
  return clamp_exp(-(exp_of(rr) >> 1));
}

// Grid-wide barrier of a cooperative launch (all blocks resident): the last
// block to arrive resets the counter and advances the generation; the others
// wait for the generation to change, for at most about two seconds, after
// which the wait records error 11 and reports false (the caller then leaves
// its loop; the other blocks' own bounded waits end the same way).
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks, int* err, int* sh_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = gen;
    const unsigned g = *vgen;
    __threadfence();  // this block's partial sums are visible before it arrives
    bool ok = true;
    if (atomicAdd(count, 1u) == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      uint64_t t0;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      for (;;) {
        if (*vgen != g) break;
        uint64_t t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        if (t1 - t0 > 2000000000ull) {
          ok = false;
          if (err) atomicCAS(err, 0, 11);
          break;
        }
      }
    }
    __threadfence();
    *sh_ok = ok;
  }
  __syncthreads();
  return *sh_ok != 0;
}

// Block = (column j, images b0 .. b0 + T - 1).  rhs and x are natural-layout
// images [B][NY][nx]; rr0 / rr / iters receive the column's ||b_j||^2, final
// ||r_j||^2 and update count per image ([B][nx]).
// GLOBAL: CG on the whole image instead of per column -- the per-column sums
// of every image go to part_pq / part_rr ([B][nx]), a grid barrier of the
// cooperative launch follows, and every block adds an image's nx column sums
// in column order, so all blocks take the same alpha and beta (Eq. 6 CG with
// the operator applied column by column).
template <int NY, int T, bool GLOBAL>
__global__ void __launch_bounds__(kSmallThreads, 2) k_colcg_small(const float2* __restrict__ G, const float2* __restrict__ rhs,
                                                            float2* __restrict__ X, int nx, int nb, int max_iter,
                                                            double rtol2, float lam, double* __restrict__ rr0_out,
                                                            double* __restrict__ rr_out, int* __restrict__ iters_out,
                                                            int* __restrict__ status, double* __restrict__ part_pq,
                                                            double* __restrict__ part_rr, unsigned* __restrict__ bar,
                                                            int* __restrict__ err) {
  constexpr int E = NY * T / kSmallThreads;  // elements (image, row) per thread
  static_assert(NY % 32 == 0 && (NY * T) % kSmallThreads == 0, "tile shape");
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* Gs = reinterpret_cast<float2*>(smraw);  // [NY][NY]
  float2* ps = Gs + NY * NY;                      // [T][NY] direction
  double* red = reinterpret_cast<double*>(ps + T * NY);  // [T][NY / 32]
  double* sc = red + T * (NY / 32);               // rr0[T], rr[T], tmp[T]
  double* s_rr0 = sc;
  double* s_rr = sc + T;
  double* s_tmp = sc + 2 * T;
  float* s_alpha = reinterpret_cast<float*>(sc + 3 * T);
  float* s_beta = s_alpha + T;
  int* s_live = reinterpret_cast<int*>(s_beta + T);
  int* s_any = s_live + T;
  int* s_ok = s_any + 1;
  int* s_er = s_ok + 1;    // [T] scale exponent of r and p (from ||r||)
  int* s_eq = s_er + T;    // [T] scale exponent of q = (G_j + lam) p
  int* s_unpq = s_eq + T;  // [T] -(er + eq): undoes the scaling of p^H q
  int* s_unrr = s_unpq + T;  // [T] -2 er: undoes the scaling of r^H r
  int* s_eg = s_unrr + T;  // exponent that brings max(|G_j|, lam) to [0.5, 1)
  auto set_scales = [&](int t, double rr) {  // thread t < T, after s_rr[t] changes
    const int er = inv_exp_sqrt(rr), eq = clamp_exp(er + *s_eg);
    s_er[t] = er;
    s_eq[t] = eq;
    s_unpq[t] = -(er + eq);
    s_unrr[t] = -2 * er;
  };

  const int j = blockIdx.x, b0 = blockIdx.y * T, tid = threadIdx.x;
  const int64_t n = (int64_t)NY * nx;
  const unsigned nblocks = gridDim.x * gridDim.y;
  // GLOBAL: replace each image's column sum in `col` by the sum over all columns
  auto whole_image = [&](double* col, double* part) -> bool {
    if (!GLOBAL) return true;
    if (threadIdx.x < T && b0 + (int)threadIdx.x < nb) part[(size_t)(b0 + threadIdx.x) * nx + j] = col[threadIdx.x];
    const bool ok = grid_barrier(bar, bar + 1, nblocks, err, s_ok);
    // warp w adds the nx column sums of images w, w + 8, ...: lane l loads columns
    // l, l + 32, ... (from L2: other blocks wrote them since the last read), then
    // a fixed shuffle tree -- the same order in every block
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = w; t < T; t += kSmallThreads / 32) {
      double a = 0.0;
      if (b0 + t < nb) {
        const double* pp = part + (size_t)(b0 + t) * nx;
        for (int jj = lane; jj < nx; jj += 32) a += __ldcg(pp + jj);
      }
      a = warp_sum_d(a);
      if (lane == 0 && b0 + t < nb) col[t] = a;
    }
    __syncthreads();
    return ok;
  };
  float gmax = lam > 0.f ? lam : 0.f;
  for (int i = tid; i < NY * NY; i += kSmallThreads) {
    const float2 g = G[(size_t)j * NY * NY + i];
    Gs[i] = g;
    gmax = fmaxf(gmax, fmaxf(fabsf(g.x), fabsf(g.y)));
  }
  {
    float* redf = reinterpret_cast<float*>(red);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    if ((tid & 31) == 0) redf[tid >> 5] = gmax;
    __syncthreads();
    if (tid == 0) {
      float m = 0.f;
      for (int w = 0; w < kSmallThreads / 32; ++w) m = fmaxf(m, redf[w]);
      *s_eg = inv_exp(m);
    }
    __syncthreads();
  }
  // this thread's elements: image t = e / NY, row y = e % NY (a warp's 32 share t)
  float2 x[E], r[E], q[E];
  ffloat v[E];
  float am[E];
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int e = k * kSmallThreads + tid, t = e / NY, y = e % NY, b = b0 + t;
    r[k] = b < nb ? rhs[(size_t)b * n + (int64_t)y * nx + j] : make_float2(0.f, 0.f);
    x[k] = make_float2(0.f, 0.f);
    am[k] = fmaxf(fabsf(r[k].x), fabsf(r[k].y));
  }
  {  // ||b_j||^2 with b scaled by its largest component
    const float m = image_max<NY, T>(am, reinterpret_cast<float*>(red));
    if (tid < T) {
      s_er[tid] = inv_exp(m);
      s_unrr[tid] = -2 * s_er[tid];
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int t = (k * kSmallThreads + tid) / NY;
    const float f = pow2f(s_er[t]);
    const float2 rs = make_float2(r[k].x * f, r[k].y * f);
    v[k] = ff_dot2(rs, rs);
  }
  image_sums<NY, T>(v, red, s_unrr, s_rr0);
  if (tid < T && b0 + tid < nb) {  // this column's ||b_j||^2 (and ||r_j||^2 until an update)
    rr0_out[(size_t)(b0 + tid) * nx + j] = s_rr0[tid];
    rr_out[(size_t)(b0 + tid) * nx + j] = s_rr0[tid];
  }
  __syncthreads();
  bool alive = whole_image(s_rr0, part_rr);
  if (tid < T) {
    const double rr = s_rr0[tid];
    s_rr[tid] = rr;
    set_scales(tid, rr);
    s_beta[tid] = 0.f;
    if (b0 + tid < nb) {
      iters_out[(size_t)(b0 + tid) * nx + j] = 0;
      if (!isfinite(rr)) status[b0 + tid] = 5;  // a non-finite right-hand side: x stays 0
    }
  }
  __syncthreads();
  for (int it = 0; it < max_iter && alive; ++it) {
    // which systems take this update (block-uniform "any" decides whether to go on)
    if (tid == 0) *s_any = 0;
    __syncthreads();
    if (tid < T) {
      const double rr = s_rr[tid], rr0 = s_rr0[tid];
      const int live = b0 + tid < nb && isfinite(rr) && isfinite(rr0) && rr > rtol2 * rr0;
      s_live[tid] = live;
      if (live) *s_any = 1;
    }
    __syncthreads();
    // every block of a launch whose images all stopped leaves together; with
    // GLOBAL and several image groups the blocks keep the same number of
    // barriers by running the remaining updates as no-ops
    if (!*s_any && (!GLOBAL || gridDim.y == 1)) break;
    // p = r + beta p
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int e = k * kSmallThreads + tid, t = e / NY;
      if (s_live[t]) {
        const float bt = s_beta[t];
        const float2 po = it > 0 ? ps[e] : make_float2(0.f, 0.f);
        ps[e] = make_float2(fmaf(bt, po.x, r[k].x), fmaf(bt, po.y, r[k].y));
      }
    }
    __syncthreads();
    // q = (G_j + lam) p: q[y] = sum_y' G[y][y'] p[y'] = sum_y' conj(G[y'][y]) p[y'] (Hermitian);
    // a warp reads G[y'][y .. y+31] (consecutive) and broadcasts p[t][y']
    if constexpr (kSmallThreads % NY == 0) {
      // a thread's E elements share the row y = tid % NY (images tid / NY + k * kSmallThreads / NY):
      // one read of G[y'][y] serves all E, two y' per step (p as float4)
      constexpr int IPK = kSmallThreads / NY;
      const int y = tid % NY, t0 = tid / NY;
      float ar[E], ai[E];
#pragma unroll
      for (int k = 0; k < E; ++k) ar[k] = ai[k] = 0.f;
#pragma unroll 4
      for (int yp = 0; yp < NY; yp += 2) {
        const float2 g0 = Gs[yp * NY + y], g1 = Gs[(yp + 1) * NY + y];
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const float4 p = *reinterpret_cast<const float4*>(ps + (k * IPK + t0) * NY + yp);
          ar[k] = fmaf(g1.x, p.z, fmaf(g1.y, p.w, fmaf(g0.x, p.x, fmaf(g0.y, p.y, ar[k]))));
          ai[k] = fmaf(g1.x, p.w, fmaf(-g1.y, p.z, fmaf(g0.x, p.y, fmaf(-g0.y, p.x, ai[k]))));
        }
      }
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const int t = k * IPK + t0;
        const float2 pe = ps[t * NY + y];
        q[k] = make_float2(fmaf(lam, pe.x, ar[k]), fmaf(lam, pe.y, ai[k]));
        const float fp = pow2f(s_er[t]), fq = pow2f(s_eq[t]);
        v[k] = ff_dot2(make_float2(pe.x * fp, pe.y * fp), make_float2(q[k].x * fq, q[k].y * fq));
      }
    } else {
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const int e = k * kSmallThreads + tid, t = e / NY, y = e % NY;
        const float2* pt = ps + t * NY;
        float ar = 0.f, ai = 0.f;
#pragma unroll 8
        for (int yp = 0; yp < NY; ++yp) {
          const float2 g = Gs[yp * NY + y], p = pt[yp];
          ar = fmaf(g.x, p.x, fmaf(g.y, p.y, ar));   // Re(conj(g) p)
          ai = fmaf(g.x, p.y, fmaf(-g.y, p.x, ai));  // Im(conj(g) p)
        }
        const float2 pe = pt[y];
        q[k] = make_float2(fmaf(lam, pe.x, ar), fmaf(lam, pe.y, ai));
        const float fp = pow2f(s_er[t]), fq = pow2f(s_eq[t]);
        v[k] = ff_dot2(make_float2(pe.x * fp, pe.y * fp), make_float2(q[k].x * fq, q[k].y * fq));
      }
    }
    image_sums<NY, T>(v, red, s_unpq, s_tmp);
    if (!whole_image(s_tmp, part_pq)) break;
    if (tid < T) {
      float a = 0.f;
      if (s_live[tid]) {
        const double pq = s_tmp[tid];
        if (!(pq > 0.0) || !isfinite(pq)) {
          s_live[tid] = 0;  // breakdown: this system keeps its iterate
          s_rr[tid] = 0.0;
          status[b0 + tid] = 5;
        } else {
          a = (float)(s_rr[tid] / pq);
        }
      }
      s_alpha[tid] = a;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int e = k * kSmallThreads + tid, t = e / NY;
      if (s_live[t]) {
        const float a = s_alpha[t];
        const float2 p = ps[e];
        x[k] = make_float2(fmaf(a, p.x, x[k].x), fmaf(a, p.y, x[k].y));
        r[k] = make_float2(fmaf(-a, q[k].x, r[k].x), fmaf(-a, q[k].y, r[k].y));
      }
      const float f = pow2f(s_er[t]);
      const float2 rs = make_float2(r[k].x * f, r[k].y * f);
      v[k] = ff_dot2(rs, rs);
    }
    image_sums<NY, T>(v, red, s_unrr, s_tmp);
    if (tid < T && b0 + tid < nb) rr_out[(size_t)(b0 + tid) * nx + j] = s_tmp[tid];  // this column's ||r_j||^2
    __syncthreads();
    if (!whole_image(s_tmp, part_rr)) break;
    if (tid < T && s_live[tid]) {
      const double rrn = s_tmp[tid];
      s_beta[tid] = (float)(rrn / s_rr[tid]);
      s_rr[tid] = rrn;
      set_scales(tid, rrn);
      if (!isfinite(rrn)) status[b0 + tid] = 5;
      iters_out[(size_t)(b0 + tid) * nx + j] = it + 1;
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int e = k * kSmallThreads + tid, t = e / NY, y = e % NY, b = b0 + t;
    if (b < nb) X[(size_t)b * n + (int64_t)y * nx + j] = x[k];
  }
  if (!GLOBAL && tid < T && b0 + tid < nb) rr_out[(size_t)(b0 + tid) * nx + j] = s_rr[tid];
}

template <int NY, int T>
size_t small_smem() {
  return (size_t)NY * NY * 8 + (size_t)T * NY * 8 + (size_t)T * (NY / 32) * 8 + 3 * T * 8 + 2 * T * 4 + T * 4 + 8 +
         4 * T * 4 + 16;
}

template <int NY, int T>
bool launch_small(const float2* G, const float2* rhs, float2* X, int nx, int nb, int max_iter, double rtol2,
                  float lam, double* rr0, double* rr, int* iters, int* status, const SmallGlobal* glob,
                  cudaStream_t s) {
  const size_t sm = small_smem<NY, T>();
  if (!glob) {
    auto k = k_colcg_small<NY, T, false>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k<<<dim3(nx, (nb + T - 1) / T), kSmallThreads, sm, s>>>(G, rhs, X, nx, nb, max_iter, rtol2, lam, rr0, rr, iters,
                                                            status, nullptr, nullptr, nullptr, nullptr);
    return true;
  }
  // whole-image CG: a cooperative launch (every block resident for the grid
  // barriers); batches whose blocks do not all fit run as several launches
  auto k = k_colcg_small<NY, T, true>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kSmallThreads, sm) != cudaSuccess) return false;
  const int groups = (per * nsm) / nx;  // image groups of T per launch
  if (groups < 1) return false;
  for (int c0 = 0; c0 < nb; c0 += groups * T) {
    const int cn = nb - c0 < groups * T ? nb - c0 : groups * T;
    cudaMemsetAsync(glob->bar, 0, 2 * sizeof(unsigned), s);
    const float2* rhs_c = rhs + (size_t)c0 * NY * nx;
    float2* X_c = X + (size_t)c0 * NY * nx;
    double* rr0_c = rr0 + (size_t)c0 * nx;
    double* rr_c = rr + (size_t)c0 * nx;
    int* it_c = iters + (size_t)c0 * nx;
    int* st_c = status + c0;
    double* pq_c = glob->part_pq + (size_t)c0 * nx;
    double* pr_c = glob->part_rr + (size_t)c0 * nx;
    unsigned* bar = glob->bar;
    int* err = glob->err;
    int cnb = cn;
    void* args[] = {(void*)&G, (void*)&rhs_c, (void*)&X_c, (void*)&nx, (void*)&cnb, (void*)&max_iter,
                    (void*)&rtol2, (void*)&lam, (void*)&rr0_c, (void*)&rr_c, (void*)&it_c, (void*)&st_c,
                    (void*)&pq_c, (void*)&pr_c, (void*)&bar, (void*)&err};
    if (cudaLaunchCooperativeKernel((const void*)k, dim3(nx, (cn + T - 1) / T), dim3(kSmallThreads), args, sm, s) !=
        cudaSuccess)
      return false;
  }
  return true;
}

}  // namespace

bool colcg_small_supported(int ny) { return ny == 32 || ny == 64 || ny == 96; }

void launch_colcg_small_build(const float2* smaps, const uint8_t* mask_host, int nc, int ny, int nx, float2* G,
                              double2* pbuf, cudaStream_t s) {
  // P[d] = (1/ny) sum_k m_k exp(2 pi i k d / ny), FP64 on the host
  double2 P[128];
  const double pi2 = 6.283185307179586476925286766559;
  for (int d = 0; d < ny; ++d) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k < ny; ++k)
      if (mask_host[k]) {
        const double a = pi2 * (double)(((int64_t)k * d) % ny) / ny;
        re += cos(a);
        im += sin(a);
      }
    P[d] = make_double2(re / ny, im / ny);
  }
  cudaMemcpyAsync(pbuf, P, ny * sizeof(double2), cudaMemcpyHostToDevice, s);
  k_colcg_small_build<<<dim3((ny * ny + 255) / 256, nx), 256, 0, s>>>(smaps, pbuf, nc, ny, nx, G);
  cudaStreamSynchronize(s);  // P lives on the host stack until the copy has run
}

bool launch_colcg_small(const float2* G, const float2* rhs, float2* X, int ny, int nx, int nb, int max_iter,
                        double rtol2, float lam, double* rr0, double* rr, int* iters, int* status,
                        const SmallGlobal* glob, cudaStream_t s) {
  if (nb <= 0) return true;
  // images per block: 32 for ny = 32, 16 for ny = 64 (128 blocks for 64
  // columns and 32 images) and ny = 96 (shared memory)
  if (ny == 32) return launch_small<32, 32>(G, rhs, X, nx, nb, max_iter, rtol2, lam, rr0, rr, iters, status, glob, s);
  if (ny == 64) return launch_small<64, 16>(G, rhs, X, nx, nb, max_iter, rtol2, lam, rr0, rr, iters, status, glob, s);
  if (ny == 96) return launch_small<96, 16>(G, rhs, X, nx, nb, max_iter, rtol2, lam, rr0, rr, iters, status, glob, s);
  return false;
}

}  // namespace pico
