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

constexpr int kColTile = 16;  // columns per CTA of the PMR column kernel
constexpr int kRowTile = 16;  // rows per CTA of the row transforms

template <int N1, int N2>
struct ColShape {
  static constexpr int N = N1 * N2;
  // threads: one per (column, job), rounded up to whole warps
  static constexpr int NT = (kColTile * (N1 > N2 ? N1 : N2) + 31) / 32 * 32;
  // [N][kColTile] values, [N] twiddles, [N] sampled-line list
  static constexpr size_t smem = (size_t)N * kColTile * sizeof(float2) + (size_t)N * sizeof(float2) + N * sizeof(int);
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
// Normal operator q = (A^H A + lam) p on column tiles of kNormTile columns.
// CG = true fuses the CG direction update p = r + beta p (beta from the
// per-iteration r^H r partials) and emits the p^H q partial of this tile.
//
// The coil sensitivities of the tile are staged through shared memory with
// cp.async, one coil ahead of the FFTs (double buffer), so their L2 latency is
// hidden; the search direction and the accumulator stay in registers.  Small
// tiles (8 columns, 8 * max(N1, N2) threads) let three CTAs share an SM so
// that one CTA's barriers overlap another's arithmetic.
// ---------------------------------------------------------------------------
template <int N1, int N2>
struct NormShape {
  static constexpr int N = N1 * N2;
  static constexpr int NC = kNormTile;
  static constexpr int NT = (NC * (N1 > N2 ? N1 : N2) + 31) / 32 * 32;
  // Frequency jobs are ordered even k2 first, then odd k2 (see k2_of), so the
  // two groups of a half-warp differ by 2; a k2 stride of 4 (mod 16) float2
  // then puts them on different bank halves (conflict-free), and the four
  // groups of a warp share a parity -- for uniform R = 2 masks also a mask class.
  static constexpr int KST = N1 * NC + ((N1 * NC) % 16 == 0 ? 4 : 12);
  static constexpr size_t buf = (size_t)N2 * KST * sizeof(float2);
  static constexpr size_t stile = (size_t)N * NC * sizeof(float2);
  static constexpr size_t smem = buf + 2 * stile + (size_t)N * sizeof(float2) + (size_t)N * sizeof(float) + 64;
};

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src, bool valid) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int bytes = valid ? 8 : 0;  // 0: zero-fill without reading global memory
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(gmem_src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src, bool valid) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int bytes = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(gmem_src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int N1, int N2, bool CG>
__global__ void __launch_bounds__(NormShape<N1, N2>::NT, 3)
    k_col_normal(CartOp op, const float2* __restrict__ xin, float2* __restrict__ yout, float lam, CgArgs a,
                 int it) {
  using Sh = NormShape<N1, N2>;
  constexpr int N = N1 * N2;
  constexpr int NT = Sh::NT;
  constexpr int NC = Sh::NC;
  constexpr int KST = Sh::KST;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);                            // [N2][KST]
  float2* stile = reinterpret_cast<float2*>(smraw + Sh::buf);                // [2][N][NC]
  float2* tws = reinterpret_cast<float2*>(smraw + Sh::buf + 2 * Sh::stile);  // [N]
  float* ym = reinterpret_cast<float*>(tws + N);                             // [N]
  unsigned char* knz = reinterpret_cast<unsigned char*>(ym + N);             // [N2] frequency-group class
  __shared__ double red[(NT + 31) / 32];
  __shared__ float sh_beta;
  __shared__ int sh_done;

  const int t = threadIdx.x;
  const int col = t % NC, job = t / NC;
  const int b = blockIdx.y;
  const int nx = op.nx, ny = op.ny;
  const int col0 = blockIdx.x * NC;
  const int colg = col0 + col;
  const bool cval = colg < nx;

  // stage the first coil's sensitivities while the CG scalars are summed;
  // 16-byte copies (two columns) when rows are 16-byte aligned (nx even)
  const bool even = (nx & 1) == 0;
  auto stage = [&](int c, int slot) {
    const float2* __restrict__ S = op.smaps + (size_t)c * ny * nx;
    float2* dst = stile + (size_t)slot * N * NC;
    if (even) {
      for (int e = t; e < N * NC / 2; e += NT) {
        const int row = e / (NC / 2), cc = 2 * (e % (NC / 2));
        const bool v = col0 + cc < nx;
        cp_async16(dst + 2 * e, v ? (const void*)(S + (size_t)row * nx + col0 + cc) : (const void*)S, v);
      }
    } else {
      for (int e = t; e < N * NC; e += NT) {
        const int row = e / NC, cc = e % NC;
        const bool v = col0 + cc < nx;
        cp_async8(dst + e, v ? (const void*)(S + (size_t)row * nx + col0 + cc) : (const void*)S, v);
      }
    }
    cp_async_commit();
  };
  stage(0, 0);

  for (int i = t; i < N; i += NT) {
    tws[i] = op.tw[i];
    ym[i] = op.ymul[i];
  }
  // class of each frequency group k2 under the mask: 0 none of its N1
  // frequencies sampled (spectrum zero), 1 all sampled with one weight (the
  // DFT_N1 / inverse DFT_N1 pair is N1 x identity), 2 anything else
  if (t < N2) {
    const float w0 = op.ymul[t];
    bool any = false, uniform = true;
    for (int k1 = 0; k1 < N1; ++k1) {
      const float w = op.ymul[t + N2 * k1];
      any |= w != 0.f;
      uniform &= w == w0;
    }
    knz[t] = !any ? 0 : (uniform ? 1 : 2);
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
  if (CG && sh_done) {
    cp_async_wait_all();  // leave no copy in flight
    return;
  }

  const size_t img = (size_t)b * ny * nx;
  const bool rowjob = job < N1;
  const bool freqjob = job < N2;
  const int n1 = job;
  // frequency group of this frequency job: even groups first, then odd ones
  const int k2 = (N2 % 2 == 0) ? (job < N2 / 2 ? 2 * job : 2 * (job - N2 / 2) + 1) : job;

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
  const int fcls = freqjob ? knz[k2] : 0;
  const float fw = freqjob ? (float)N1 * ym[k2] : 0.f;

  // Two barriers per coil: (A) after the forward row-job pass, (B) after the
  // frequency pass.  Coil c+1's sensitivities are copied during the frequency
  // pass of coil c (its slot was last read in the inverse pass of coil c-1,
  // which every thread finished before barrier A of coil c) and waited for
  // before barrier B, so the inverse pass of coil c and the forward pass of
  // coil c+1 run back to back without a barrier between them.
  cp_async_wait_all();
  __syncthreads();  // coil 0 staged
  for (int c = 0; c < op.nc; ++c) {
    const float2* __restrict__ Ss = stile + (size_t)(c & 1) * N * NC;
    if (rowjob) {
      float2 z[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) z[n2] = cmul(Ss[(n1 + N1 * n2) * NC + col], p[n2]);
      DFT<N2, -1>::run(z);
#pragma unroll
      for (int k = 0; k < N2; ++k) buf[k * KST + n1 * NC + col] = k == 0 ? z[0] : cmul(z[k], tws[n1 * k]);
    }
    __syncthreads();  // (A)
    if (c + 1 < op.nc) stage(c + 1, (c + 1) & 1);
    if (fcls == 2) {
      float2 y[N1];
#pragma unroll
      for (int m = 0; m < N1; ++m) y[m] = buf[k2 * KST + m * NC + col];
      DFT<N1, -1>::run(y);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) y[k1] = cscale(y[k1], ym[k2 + N2 * k1]);
      DFT<N1, 1>::run(y);
#pragma unroll
      for (int m = 0; m < N1; ++m) buf[k2 * KST + m * NC + col] = m == 0 ? y[0] : cmul_cb(y[m], tws[m * k2]);
    } else if (fcls == 1) {
      // every frequency of the group sampled with weight ym: forward and inverse
      // DFT_N1 cancel to N1 x identity; only the conjugate twiddle remains
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        const float2 v = cscale(buf[k2 * KST + m * NC + col], fw);
        buf[k2 * KST + m * NC + col] = m == 0 ? v : cmul_cb(v, tws[m * k2]);
      }
    } else if (freqjob) {
      // no sampled frequency in this group: the masked spectrum is zero
#pragma unroll
      for (int m = 0; m < N1; ++m) buf[k2 * KST + m * NC + col] = make_float2(0.f, 0.f);
    }
    cp_async_wait_all();
    __syncthreads();  // (B): frequency pass done, coil c+1 staged
    if (rowjob) {
      float2 z[N2];
#pragma unroll
      for (int k = 0; k < N2; ++k) z[k] = buf[k * KST + n1 * NC + col];
      DFT<N2, 1>::run(z);
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) acc[n2] = cfma_c(acc[n2], Ss[(n1 + N1 * n2) * NC + col], z[n2]);
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
// The draws run first, over the block's sampled lines only (a list built
// per block), so that every lane of a warp draws: a draw loop over the
// frequency jobs' own lines idled the lanes whose line is not sampled
// (with R = 2 half of every warp).  The values wait in shared memory in
// line order, [ky][column], until the frequency jobs load them.
// ---------------------------------------------------------------------------
template <int N1, int N2>
__global__ void __launch_bounds__(ColShape<N1, N2>::NT, 1)
    k_col_pmr(CartOp op, float2* __restrict__ G, uint64_t seed, int64_t rep_begin, float sigma, float scale,
              const float2* __restrict__ data) {
  constexpr int N = N1 * N2;
  constexpr int NT = ColShape<N1, N2>::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* buf = reinterpret_cast<float2*>(smraw);
  float2* tws = buf + N * kColTile;
  int* lines = reinterpret_cast<int*>(tws + N);  // sampled ky, ascending
  __shared__ int nlines;

  const int t = threadIdx.x;
  const int col = t % kColTile, job = t / kColTile;
  const int bc = blockIdx.y;  // b * nc + c
  const int c = bc % op.nc, b = bc / op.nc;
  const int nx = op.nx, ny = op.ny;
  const int colg = blockIdx.x * kColTile + col;
  const bool cval = colg < nx;
  for (int i = t; i < N; i += NT) tws[i] = op.tw[i];
  if (t < 32) {  // warp 0 lists the sampled lines in order
    int base = 0;
    for (int k0 = 0; k0 < N; k0 += 32) {
      const bool m = k0 + t < N && op.mask[k0 + t];
      const unsigned bal = __ballot_sync(0xffffffffu, m);
      if (m) lines[base + __popc(bal & ((1u << t) - 1u))] = k0 + t;
      base += __popc(bal);
    }
    if (t == 0) nlines = base;
  }
  __syncthreads();
  const int nl = nlines;
  {
    const uint64_t key = splitmix64(seed, (uint64_t)(rep_begin + b));
    for (int i = t; i < nl * kColTile; i += NT) {
      const int ky = lines[i / kColTile], cc = i % kColTile, cg = blockIdx.x * kColTile + cc;
      float2 v = make_float2(0.f, 0.f);
      if (cg < nx) {
        const uint64_t e = ((uint64_t)c * ny + ky) * (uint64_t)nx + cg;
        v = data ? data[((size_t)b * op.nc * ny) * nx + e] : draw_cnoise(key, e, sigma);
      }
      buf[ky * kColTile + cc] = v;
    }
  }
  __syncthreads();
  const int n1 = job, k2 = job;
  float2 y[N1];
  if (job < N2) {
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const int ky = k2 + N2 * k1;
      y[k1] = op.mask[ky] ? buf[ky * kColTile + col] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();  // every line is loaded: the buffer takes the transposed layout
  if (job < N2) {
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
__global__ void __launch_bounds__(RowShape<M1, M2>::NT, (RowShape<M1, M2>::NT <= 320 ? 2 : 1))
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
  using Sh = NormShape<N1, N2>;
  const dim3 grid(cart_normal_tiles(op.nx), nb);
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
                      cudaStream_t s, const float2* data) {
  using Sh = ColShape<N1, N2>;
  const dim3 grid((op.nx + kColTile - 1) / kColTile, nb * op.nc);
  auto k = k_col_pmr<N1, N2>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
  const float scale = (float)(1.0 / sqrt((double)op.ny * (double)op.nx));
  k<<<grid, Sh::NT, Sh::smem, s>>>(op, G, seed, rep_begin, sigma, scale, data);
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
