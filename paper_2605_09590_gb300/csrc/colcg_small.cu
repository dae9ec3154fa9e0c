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
// gmax (zeroed before the launch) receives the largest |component| of any G_j
// (non-negative floats order like their bit patterns).
__global__ void k_colcg_small_build(const float2* __restrict__ S, const double2* __restrict__ P, int nc, int ny,
                                    int nx, float2* __restrict__ G, unsigned* __restrict__ gmax) {
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
  const float2 g = make_float2((float)(p.x * re - p.y * im), (float)(p.x * im + p.y * re));
  G[((size_t)j * ny + y) * ny + yp] = g;
  const float m = fmaxf(fabsf(g.x), fabsf(g.y));
  if (isfinite(m)) atomicMax(gmax, __float_as_uint(m));
}

// Sum over the NY rows of every image of a per-element value held by the
// thread that owns element e = k * kSmallThreads + tid (image e / NY, row
// e % NY): a warp's 32 elements belong to one image; warp sums go to
// red[t][w], then thread t < T adds its NY / 32 slots in order into out[t].
template <int NY, int T>
__device__ __forceinline__ void image_sums(const ffloat (&v)[NY * T / kSmallThreads], ffloat* red, ffloat* out) {
  constexpr int E = NY * T / kSmallThreads;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const ffloat s = warp_sum_ff(v[k]);
    const int e = k * kSmallThreads + threadIdx.x;
    if (lane == 0) red[(e / NY) * (NY / 32) + (e % NY) / 32] = s;
  }
  __syncthreads();
  if (threadIdx.x < T) {
    ffloat s = red[threadIdx.x * (NY / 32)];
#pragma unroll
    for (int w = 1; w < NY / 32; ++w) s = ff_add(s, red[threadIdx.x * (NY / 32) + w]);
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// The same in FP64 (the one-off ||b_j||^2 before any scale is known).
template <int NY, int T>
__device__ __forceinline__ void image_sums_d(const double (&v)[NY * T / kSmallThreads], double* red, double* out) {
  constexpr int E = NY * T / kSmallThreads;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const double s = warp_sum_d(v[k]);
    const int e = k * kSmallThreads + threadIdx.x;
    if (lane == 0) red[(e / NY) * (NY / 32) + (e % NY) / 32] = s;
  }
  __syncthreads();
  if (threadIdx.x < T) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NY / 32; ++w) s += red[threadIdx.x * (NY / 32) + w];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Power-of-two scaling keeps the float-float products clear of FP32 underflow
// and overflow: values are multiplied by 2^e before the exact products and the
// sums by 2^-e afterwards (exact in the normal range).
__device__ __forceinline__ int clamp_exp(int e) { return e < -120 ? -120 : (e > 120 ? 120 : e); }
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + clamp_exp(e)) << 23); }
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }  // |e| <= 1000
// binary exponent e of a normal a > 0 (a = m 2^e, m in [0.5, 1))
__device__ __forceinline__ int exp_of(double a) { return (int)((__double_as_longlong(a) >> 52) & 0x7ff) - 1022; }
__device__ __forceinline__ int exp_of(float a) { return (int)((__float_as_uint(a) >> 23) & 0xff) - 126; }
// e with a * 2^e in [0.5, 1) (0 for zero or non-finite a)
__device__ __forceinline__ int inv_exp(float a) { return (a > 0.f && isfinite(a)) ? clamp_exp(-exp_of(a)) : 0; }
// e with ||r|| * 2^e near 1, from rr = ||r||^2 (every value here is a sum of
// squares of floats, far above the FP64 subnormals)
__device__ __forceinline__ int inv_exp_sqrt(double rr) {
  return (rr > 0.0 && isfinite(rr)) ? clamp_exp(-(exp_of(rr) >> 1)) : 0;
}
// value of a scaled float-float sum
__device__ __forceinline__ double ff_value(ffloat a, int un) { return ((double)a.hi + (double)a.lo) * pow2d(un); }
// a / b to about float precision (the first step of float-float division);
// b.hi > 0
__device__ __forceinline__ float ff_div(ffloat a, ffloat b) {
  const float q1 = a.hi / b.hi;
  const float rem = fmaf(-q1, b.hi, a.hi) + a.lo - q1 * b.lo;
  return q1 + rem / b.hi;
}

// Exchange words: (sequence << 32) | payload, written and read as single
// 64-bit strong (relaxed, GPU-scope) accesses, so a reader that sees the
// sequence it waits for sees the payload written with it.
__device__ __forceinline__ void st_word(unsigned long long* p, unsigned seq, unsigned payload) {
  const unsigned long long w = ((unsigned long long)seq << 32) | payload;
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}
__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
  unsigned long long w;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
  return w;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Block = (column j, images b0 .. b0 + T - 1).  rhs and x are natural-layout
// images [B][NY][nx]; rr0 / rr / iters receive the column's ||b_j||^2, final
// ||r_j||^2 and update count per image ([B][nx]).  gmax: the largest |G_j|
// component over every column (sets the scale of q).
// GLOBAL: CG on the whole image instead of per column.  The blocks of one
// image group exchange their column sums: each publishes its T sums in
// part[B][nx] as two tagged words per sum (the exchange's sequence number in
// the high half); each waits until the group's nx sums of an image carry the
// current sequence and adds them in column order, so every block of the group
// takes the same alpha and beta (Eq. 6 CG with the operator applied column by
// column).  An entry is overwritten two exchanges later, after its readers
// have published the exchange in between (whose values depend on what they
// read).  Groups are independent; a cooperative launch keeps all blocks
// resident, and every wait gives up after about two seconds (error 11).
template <int NY, int T, bool GLOBAL>
__global__ void __launch_bounds__(kSmallThreads, 2)
    k_colcg_small(const float2* __restrict__ G, const float* __restrict__ gmax, const float2* __restrict__ rhs,
                  float2* __restrict__ X, int nx, int nb, int max_iter, double rtol2, float lam,
                  double* __restrict__ rr0_out, double* __restrict__ rr_out, int* __restrict__ iters_out,
                  int* __restrict__ status, ulonglong2* __restrict__ part_pq, ulonglong2* __restrict__ part_rr,
                  int* __restrict__ err) {
  constexpr int E = NY * T / kSmallThreads;  // elements (image, row) per thread
  static_assert(NY % 32 == 0 && (NY * T) % kSmallThreads == 0, "tile shape");
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* Gs = reinterpret_cast<float2*>(smraw);             // [NY][NY]
  float2* ps = Gs + NY * NY;                                 // [T][NY] direction
  ffloat* red = reinterpret_cast<ffloat*>(ps + T * NY);      // [T][NY / 32] (FP64 in the first sum)
  double* s_rr0 = reinterpret_cast<double*>(red + T * (NY / 32));  // [T] ||b||^2
  double* s_rrd = s_rr0 + T;                                 // [T] ||r||^2
  double* s_rrcol = s_rrd + T;                               // [T] this column's ||r_j||^2
  ffloat* s_sum = reinterpret_cast<ffloat*>(s_rrcol + T);    // [T] latest (scaled) sum
  ffloat* s_rr = s_sum + T;                                  // [T] ||r||^2 scaled by 2^-s_rrun
  float* s_alpha = reinterpret_cast<float*>(s_rr + T);
  float* s_beta = s_alpha + T;
  int* s_live = reinterpret_cast<int*>(s_beta + T);
  int* s_rrun = s_live + T;
  int* s_er = s_rrun + T;  // scale exponent of r and p (from ||r||)
  int* s_eq = s_er + T;    // scale exponent of q = (G_j + lam) p
  int* s_iters = s_eq + T;
  int* s_any = s_iters + T;
  int* s_ok = s_any + 1;
  unsigned* s_xw = reinterpret_cast<unsigned*>(s_ok + 1);  // [2T] words being published

  const int j = blockIdx.x, b0 = blockIdx.y * T, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) *s_ok = 1;
  const int64_t n = (int64_t)NY * nx;
  unsigned seq = 0;
  // GLOBAL: publish this block's T column sums (two 32-bit halves each), wait
  // for the group's, and combine each image's nx sums in column order: warp w
  // takes images w, w + 8, ...; lane l columns l, l + 32, ... (loads of up to
  // four entries in flight, reissued until they carry the sequence), then a
  // fixed shuffle tree.  add(acc, hi, lo) folds one entry; done(t, acc) stores.
  auto exchange = [&](const unsigned* w_hi, const unsigned* w_lo, ulonglong2* part, auto zero, auto add,
                      auto done) -> bool {
    ++seq;
    if (tid < T && b0 + tid < nb) {
      ulonglong2* e = part + (size_t)(b0 + tid) * nx + j;
      st_word(&e->x, seq, w_hi[tid]);
      st_word(&e->y, seq, w_lo[tid]);
    }
    constexpr int IW = T / (kSmallThreads / 32);  // images per warp
    const int nj = (nx + 31) / 32, ne = IW * nj;  // entries per lane
    decltype(zero) accs[IW];
#pragma unroll
    for (int i = 0; i < IW; ++i) accs[i] = zero;
    bool ok = true;
    const uint64_t t0 = global_ns();
    for (int e0 = 0; e0 < ne; e0 += 4) {
      unsigned long long w0[4], w1[4];
      bool ready = false;
      while (!ready) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int e = e0 + m, i = e / nj, jj = lane + 32 * (e % nj), b = b0 + warp + 8 * i;
          if (e < ne && jj < nx && b < nb) {
            const ulonglong2* pe = part + (size_t)b * nx + jj;
            w0[m] = ld_word(&pe->x);
            w1[m] = ld_word(&pe->y);
          } else {
            w0[m] = w1[m] = (unsigned long long)seq << 32;
          }
        }
        ready = true;
#pragma unroll
        for (int m = 0; m < 4; ++m) ready = ready && (unsigned)(w0[m] >> 32) == seq && (unsigned)(w1[m] >> 32) == seq;
        if (!ready && global_ns() - t0 > 2000000000ull) {
          if (err) atomicCAS(err, 0, 11);
          ok = false;
          break;
        }
      }
      if (!ok) break;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int e = e0 + m, i = e / nj, jj = lane + 32 * (e % nj), b = b0 + warp + 8 * i;
        if (e < ne && jj < nx && b < nb) {
#pragma unroll
          for (int ii = 0; ii < IW; ++ii)
            if (ii == i) accs[ii] = add(accs[ii], (unsigned)w0[m], (unsigned)w1[m]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < IW; ++i) done(warp + 8 * i, accs[i]);
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0 && !ok) *s_ok = 0;
    __syncthreads();
    return *s_ok != 0;
  };
  auto whole_image = [&](ffloat* col, ulonglong2* part) -> bool {
    if (!GLOBAL) return true;
    const unsigned* hl = reinterpret_cast<const unsigned*>(col);  // col[t] = {hi, lo}: words 2t, 2t + 1
    unsigned* hi_w = reinterpret_cast<unsigned*>(s_xw);
    unsigned* lo_w = hi_w + T;
    if (tid < T) {  // read back by the same thread: no barrier needed
      hi_w[tid] = hl[2 * tid];
      lo_w[tid] = hl[2 * tid + 1];
    }
    const bool ok = exchange(
        hi_w, lo_w, part, ffloat{0.f, 0.f},
        [](ffloat a, unsigned h, unsigned l) { return ff_add(a, ffloat{__uint_as_float(h), __uint_as_float(l)}); },
        [&](int t, ffloat a) {
          a = warp_sum_ff(a);
          if (lane == 0 && b0 + t < nb) col[t] = a;
        });
    return ok;
  };
  for (int i = tid; i < NY * NY; i += kSmallThreads) Gs[i] = G[(size_t)j * NY * NY + i];
  const int eg = inv_exp(fmaxf(*gmax, lam));  // brings the largest entry of G_j + lam I to [0.5, 1)
  // this thread's elements: image t = e / NY, row y = e % NY (a warp's 32 share t)
  float2 x[E], r[E], q[E];
  ffloat v[E];
  {  // ||b_j||^2 in FP64 (no scale known yet), then over the image
    double vd[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int e = k * kSmallThreads + tid, t = e / NY, y = e % NY, b = b0 + t;
      r[k] = b < nb ? rhs[(size_t)b * n + (int64_t)y * nx + j] : make_float2(0.f, 0.f);
      x[k] = make_float2(0.f, 0.f);
      vd[k] = (double)r[k].x * r[k].x + (double)r[k].y * r[k].y;
    }
    double* redd = reinterpret_cast<double*>(red);
    image_sums_d<NY, T>(vd, redd, s_rr0);
    if (tid < T && b0 + tid < nb) {
      rr0_out[(size_t)(b0 + tid) * nx + j] = s_rr0[tid];
      s_rrcol[tid] = s_rr0[tid];
    }
    bool ok = true;
    if (GLOBAL) {
      if (tid < T) {  // the double's high and low 32 bits
        s_xw[tid] = (unsigned)__double2hiint(s_rr0[tid]);
        s_xw[T + tid] = (unsigned)__double2loint(s_rr0[tid]);
      }
      __syncthreads();
      ok = exchange(
          s_xw, s_xw + T, part_rr, 0.0,
          [](double a, unsigned h, unsigned l) { return a + __hiloint2double((int)h, (int)l); },
          [&](int t, double a) {
            a = warp_sum_d(a);
            if (lane == 0 && b0 + t < nb) s_rr0[t] = a;
          });
    }
    if (tid < T) {
      const double rr = s_rr0[tid];
      const int er = inv_exp_sqrt(rr), un = -2 * er;
      const double sc = rr * pow2d(2 * er);  // in [0.25, 1)
      const float hi = (float)sc;
      s_rr[tid] = ffloat{hi, (float)(sc - (double)hi)};
      s_rrun[tid] = un;
      s_rrd[tid] = rr;
      s_er[tid] = er;
      s_eq[tid] = clamp_exp(er + eg);
      s_beta[tid] = 0.f;
      s_iters[tid] = 0;
      if (b0 + tid < nb && !isfinite(rr)) status[b0 + tid] = 5;  // a non-finite right-hand side: x stays 0
    }
    if (tid == 0) *s_any = ok;
    __syncthreads();
    const bool go = *s_any != 0;
    __syncthreads();  // every thread has read the flag before the loop's first reset of it
    if (!go) max_iter = 0;
  }
  for (int it = 0; it < max_iter; ++it) {
    // which systems take this update (every block of a group decides alike)
    if (tid == 0) *s_any = 0;
    __syncthreads();
    if (tid < T) {
      const double rr = s_rrd[tid], rr0 = s_rr0[tid];
      const int live = b0 + tid < nb && isfinite(rr) && isfinite(rr0) && rr > rtol2 * rr0;
      s_live[tid] = live;
      if (live) *s_any = 1;
    }
    __syncthreads();
    if (!*s_any) break;
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
    image_sums<NY, T>(v, red, s_sum);
    if (!whole_image(s_sum, part_pq)) break;
    if (tid < T) {
      float a = 0.f;
      if (s_live[tid]) {
        const ffloat pq = s_sum[tid];  // p^H q scaled by 2^(er + eq)
        if (!(pq.hi > 0.f) || !isfinite(pq.hi)) {
          s_live[tid] = 0;  // breakdown: this system keeps its iterate
          s_rrd[tid] = 0.0;
          if (!GLOBAL) s_rrcol[tid] = 0.0;
          status[b0 + tid] = 5;
        } else {
          // rr / pq with rr scaled by 2^-rrun and pq by 2^(er + eq)
          a = ff_div(s_rr[tid], pq) * pow2f(s_rrun[tid] + s_er[tid] + s_eq[tid]);
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
    image_sums<NY, T>(v, red, s_sum);
    if (tid < T && s_live[tid]) s_rrcol[tid] = ff_value(s_sum[tid], -2 * s_er[tid]);  // this column's ||r_j||^2
    if (!whole_image(s_sum, part_rr)) break;
    if (tid < T && s_live[tid]) {
      const ffloat rrn = s_sum[tid];  // scaled by 2^(2 er)
      const int un = -2 * s_er[tid];
      const double rrd = ff_value(rrn, un);
      s_beta[tid] = ff_div(rrn, s_rr[tid]) * pow2f(un - s_rrun[tid]);
      s_rr[tid] = rrn;
      s_rrun[tid] = un;
      s_rrd[tid] = rrd;
      const int er = inv_exp_sqrt(rrd);
      s_er[tid] = er;
      s_eq[tid] = clamp_exp(er + eg);
      if (!isfinite(rrd)) status[b0 + tid] = 5;
      s_iters[tid] = it + 1;
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int e = k * kSmallThreads + tid, t = e / NY, y = e % NY, b = b0 + t;
    if (b < nb) X[(size_t)b * n + (int64_t)y * nx + j] = x[k];
  }
  if (tid < T && b0 + tid < nb) {
    rr_out[(size_t)(b0 + tid) * nx + j] = s_rrcol[tid];
    iters_out[(size_t)(b0 + tid) * nx + j] = s_iters[tid];
  }
}

template <int NY, int T>
size_t small_smem() {
  return (size_t)NY * NY * 8 + (size_t)T * NY * 8 + (size_t)T * (NY / 32) * 8 + 3 * T * 8 + 2 * T * 8 + 2 * T * 4 +
         5 * T * 4 + 8 + 2 * T * 4 + 16;
}

template <int NY, int T>
bool launch_small(const float2* G, const float* gmax, const float2* rhs, float2* X, int nx, int nb, int max_iter,
                  double rtol2, float lam, double* rr0, double* rr, int* iters, int* status, const SmallGlobal* glob,
                  cudaStream_t s) {
  const size_t sm = small_smem<NY, T>();
  if (!glob) {
    auto k = k_colcg_small<NY, T, false>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k<<<dim3(nx, (nb + T - 1) / T), kSmallThreads, sm, s>>>(G, gmax, rhs, X, nx, nb, max_iter, rtol2, lam, rr0, rr,
                                                            iters, status, nullptr, nullptr, nullptr);
    return true;
  }
  // whole-image CG: a cooperative launch (every block resident for the
  // exchanges); batches whose blocks do not all fit run as several launches
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
    const int ng = (cn + T - 1) / T;
    // sequence 0 everywhere: no entry of an earlier launch passes for this one's
    cudaMemsetAsync(glob->part_pq + (size_t)c0 * nx, 0, (size_t)cn * nx * sizeof(ulonglong2), s);
    cudaMemsetAsync(glob->part_rr + (size_t)c0 * nx, 0, (size_t)cn * nx * sizeof(ulonglong2), s);
    const float2* rhs_c = rhs + (size_t)c0 * NY * nx;
    float2* X_c = X + (size_t)c0 * NY * nx;
    double* rr0_c = rr0 + (size_t)c0 * nx;
    double* rr_c = rr + (size_t)c0 * nx;
    int* it_c = iters + (size_t)c0 * nx;
    int* st_c = status + c0;
    ulonglong2* pq_c = glob->part_pq + (size_t)c0 * nx;
    ulonglong2* pr_c = glob->part_rr + (size_t)c0 * nx;
    int* err = glob->err;
    int cnb = cn;
    void* args[] = {(void*)&G,     (void*)&gmax,  (void*)&rhs_c, (void*)&X_c,   (void*)&nx,    (void*)&cnb,
                    (void*)&max_iter, (void*)&rtol2, (void*)&lam,  (void*)&rr0_c, (void*)&rr_c,  (void*)&it_c,
                    (void*)&st_c,  (void*)&pq_c,  (void*)&pr_c,  (void*)&err};
    if (cudaLaunchCooperativeKernel((const void*)k, dim3(nx, ng), dim3(kSmallThreads), args, sm, s) != cudaSuccess)
      return false;
  }
  return true;
}

}  // namespace

bool colcg_small_supported(int ny) { return ny == 32 || ny == 64 || ny == 96; }

void launch_colcg_small_build(const float2* smaps, const uint8_t* mask_host, int nc, int ny, int nx, float2* G,
                              float* gmax, double2* pbuf, cudaStream_t s) {
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
  cudaMemsetAsync(gmax, 0, sizeof(float), s);
  k_colcg_small_build<<<dim3((ny * ny + 255) / 256, nx), 256, 0, s>>>(smaps, pbuf, nc, ny, nx, G,
                                                                     reinterpret_cast<unsigned*>(gmax));
  cudaStreamSynchronize(s);  // P lives on the host stack until the copy has run
}

bool launch_colcg_small(const float2* G, const float* gmax, const float2* rhs, float2* X, int ny, int nx, int nb,
                        int max_iter, double rtol2, float lam, double* rr0, double* rr, int* iters, int* status,
                        const SmallGlobal* glob, cudaStream_t s) {
  if (nb <= 0) return true;
  // images per block: 32 for ny = 32, 16 for ny = 64 (128 blocks for 64
  // columns and 32 images) and ny = 96 (shared memory)
  if (ny == 32) return launch_small<32, 32>(G, gmax, rhs, X, nx, nb, max_iter, rtol2, lam, rr0, rr, iters, status, glob,
                                    s);
  if (ny == 64) return launch_small<64, 16>(G, gmax, rhs, X, nx, nb, max_iter, rtol2, lam, rr0, rr, iters, status, glob,
                                    s);
  if (ny == 96) return launch_small<96, 16>(G, gmax, rhs, X, nx, nb, max_iter, rtol2, lam, rr0, rr, iters, status, glob,
                                    s);
  return false;
}

}  // namespace pico
