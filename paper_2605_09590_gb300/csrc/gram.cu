// Dense per-column SENSE normal operator on the tensor cores (Cartesian
// phase-encode masks).
//
// With a mask on the phase-encode axis only, A^H A acts on every readout
// column j independently (the x-FFT cancels, Sec. 2.1.3 with M = M_y (x) I):
//   (A^H A p)[y, j] = sum_y' G_j[y, y'] p[y', j],
//   G_j[y, y'] = P[y - y'] sum_c conj(S_c[y, j]) S_c[y', j],
//   P[d] = (1/ny) sum_k m_k exp(2 pi i k d / ny)   (F_y^H M_y F_y, a circulant).
// G_j is Hermitian, ny x ny, and the same for every probe, so one normal
// operator over a batch of K images is nx dense complex products
// Q_j (K x ny) = P_j (K x ny) G_j^T -- a contraction with reuse K that runs
// on tcgen05 tensor cores.  FP32 accuracy comes from the 3-term TF32 split
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (G split once at set-up, the
// direction p split on the fly), accumulated in FP32 in tensor memory.
//
// CG vectors of a Gram-mode context live in a column-planar layout
// [image][x][re|im][y] (so that the contraction index y is contiguous); the
// kernels here convert to and from the natural [image][y][x] complex layout.
#include <cuda_fp16.h>

#include <vector>

#include "common.cuh"
#include "f16_split.cuh"
#include "kernels.cuh"
#include "tc_util.cuh"

namespace pico {

namespace {

using namespace tc;

constexpr int kGramRows = 128;   // images per CTA (MMA M)
constexpr int kGramThreads = 192;

// Contraction chunk per pipeline stage: KC = 16 values (64-byte rows, 64-byte
// swizzle) or KC = 8 (32-byte rows, 32-byte swizzle, twice the stages).
template <int KC>
struct GramTile {
  static constexpr uint32_t kATile = kGramRows * KC * 4;
  static constexpr uint32_t kRowBytes = KC * 4;
  // descriptor of a K-major tile: rows of KC*4 bytes, 8-row atoms
  static __device__ __forceinline__ uint64_t desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)((8u * kRowBytes) >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)(KC == 16 ? 4u : 6u) << 61;  // 64-byte or 32-byte swizzle
    return d;
  }
  // logical 16-byte chunk of a row from its position in shared memory: the
  // swizzle XORs byte-offset bits 4.. with bits 7..
  static __device__ __forceinline__ int chunk(int phys, int row) {
    return KC == 16 ? (phys ^ ((row >> 1) & 3)) : (phys ^ ((row >> 2) & 1));
  }
};

__device__ __forceinline__ void set_err(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------------------
// set-up: G_j split into TF32 head and remainder, stored stage-tiled
// ---------------------------------------------------------------------------
// Position of G_j[y, y'] (plane q: 0 re head, 1 im head, 2 re remainder, 3 im
// remainder) in the stage-tiled layout: block (j, y tile, chunk of kc values
// of y') holds the four planes of nt rows x kc values exactly as one pipeline
// stage holds them in shared memory, the 16-byte groups of a row swizzled
// (64-byte swizzle for kc = 16, 32-byte for kc = 8), so that one bulk copy
// fills the B operand of a stage.
__device__ __forceinline__ size_t gt_offset(int j, int y, int yp, int q, int ny, int nt, int kc) {
  const int t = y / nt, r = y - t * nt, c = yp / kc, e = yp - c * kc;
  const int grp = e >> 2, phys = kc == 16 ? (grp ^ ((r >> 1) & 3)) : (grp ^ ((r >> 2) & 1));
  return ((((size_t)j * (ny / nt) + t) * (ny / kc) + c) * 4 + q) * (size_t)nt * kc + (size_t)r * kc + 4 * phys +
         (e & 3);
}

// The FP16 form of the same tiling: stages of 16 values of y' (32-byte rows,
// 32-byte swizzle: the two 16-byte groups of a row swap on rows 4..7 of every
// 8-row atom), halves instead of floats.
__device__ __forceinline__ size_t gt_offset_h(int j, int y, int yp, int q, int ny, int nt) {
  const int t = y / nt, r = y - t * nt, c = yp >> 4, e = yp & 15;
  const int phys = (e >> 3) ^ ((r >> 2) & 1);
  return ((((size_t)j * (ny / nt) + t) * (ny / 16) + c) * 4 + q) * (size_t)nt * 16 + (size_t)r * 16 + 8 * phys +
         (e & 7);
}

__global__ void k_gram_build(const float2* __restrict__ S, const double2* __restrict__ P, int nc, int ny, int nx,
                             int nt, int kc, float* __restrict__ G) {
  const int j = blockIdx.y;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ny * ny) return;
  const int y = (int)(t / ny), yp = (int)(t % ny);
  const int64_t n = (int64_t)ny * nx;
  double re = 0.0, im = 0.0;
  for (int c = 0; c < nc; ++c) {
    const float2 a = S[c * n + (int64_t)y * nx + j], b = S[c * n + (int64_t)yp * nx + j];
    // conj(a) b
    re += (double)a.x * b.x + (double)a.y * b.y;
    im += (double)a.x * b.y - (double)a.y * b.x;
  }
  int d = y - yp;
  if (d < 0) d += ny;
  const double2 p = P[d];
  const double gr = p.x * re - p.y * im, gi = p.x * im + p.y * re;
  float hr, lr, hi_, li;
  split_tf32((float)gr, hr, lr);
  split_tf32((float)gi, hi_, li);
  G[gt_offset(j, y, yp, 0, ny, nt, kc)] = hr;
  G[gt_offset(j, y, yp, 1, ny, nt, kc)] = hi_;
  G[gt_offset(j, y, yp, 2, ny, nt, kc)] = (float)(gr - (double)hr);
  G[gt_offset(j, y, yp, 3, ny, nt, kc)] = (float)(gi - (double)hi_);
}

// The same G_j with the sensitivities of column j staged in shared memory
// (block = column j x 32 output rows; all y' per block).
// F16: G_j scaled by the power of two gscale[j] (pow2_scale of the bound
// |G_j[y, y']| <= P[0] max_y sum_c |S_c[y, j]|^2, Cauchy-Schwarz with
// |P[d]| <= P[0]) and split into an FP16 head and FP16 remainder.
template <bool F16>
__global__ void __launch_bounds__(256) k_gram_build_smem(const float2* __restrict__ S, const double2* __restrict__ P,
                                                         int nc, int ny, int nx, int nt, int kc,
                                                         void* __restrict__ Gv, float* __restrict__ gscale) {
  extern __shared__ float2 sc[];  // [nc][ny] sensitivities of column j
  __shared__ float red[8];
  const int j = blockIdx.x, y_lo = blockIdx.y * 32;
  const int64_t n = (int64_t)ny * nx;
  for (int i = threadIdx.x; i < nc * ny; i += blockDim.x) {
    const int c = i / ny, y = i % ny;
    sc[i] = S[c * n + (int64_t)y * nx + j];
  }
  __syncthreads();
  float gs = 1.f;
  if (F16) {
    float m = 0.f;
    for (int y = threadIdx.x; y < ny; y += blockDim.x) {
      float e = 0.f;
      for (int c = 0; c < nc; ++c) e = fmaf(sc[c * ny + y].x, sc[c * ny + y].x, fmaf(sc[c * ny + y].y, sc[c * ny + y].y, e));
      m = fmaxf(m, e);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    // 1.01: room for the FP32 rounding of the sums below
    gs = pow2_scale(1.01 * (double)m * fabs(P[0].x));
    if (blockIdx.y == 0 && threadIdx.x == 0) gscale[j] = gs;
  }
  float* G = static_cast<float*>(Gv);
  __half* Gh = static_cast<__half*>(Gv);
  for (int t = threadIdx.x; t < 32 * ny; t += blockDim.x) {
    const int y = y_lo + t / ny, yp = t % ny;
    if (y >= ny) break;
    // FP32 with compensated (Kahan) summation over the coils: FP64 arithmetic
    // is a small fraction of the FP32 rate on this part
    float re = 0.f, rc = 0.f, im = 0.f, ic = 0.f;
    for (int c = 0; c < nc; ++c) {
      const float2 a = sc[c * ny + y], b = sc[c * ny + yp];
      const float tr = fmaf(a.x, b.x, a.y * b.y) - rc;
      const float sr = re + tr;
      rc = (sr - re) - tr;
      re = sr;
      const float ti = fmaf(a.x, b.y, -a.y * b.x) - ic;
      const float si = im + ti;
      ic = (si - im) - ti;
      im = si;
    }
    int d = y - yp;
    if (d < 0) d += ny;
    const double2 p = P[d];
    const float px = (float)p.x, py = (float)p.y;
    const float gr = fmaf(px, re, -py * im), gi = fmaf(px, im, py * re);
    if (F16) {
      const float sr = gr * gs, si = gi * gs;
      const __half hr = __float2half_rn(sr), hi_ = __float2half_rn(si);
      Gh[gt_offset_h(j, y, yp, 0, ny, nt)] = hr;
      Gh[gt_offset_h(j, y, yp, 1, ny, nt)] = hi_;
      Gh[gt_offset_h(j, y, yp, 2, ny, nt)] = __float2half_rn(sr - __half2float(hr));
      Gh[gt_offset_h(j, y, yp, 3, ny, nt)] = __float2half_rn(si - __half2float(hi_));
    } else {
      float hr, lr, hi_, li;
      split_tf32(gr, hr, lr);
      split_tf32(gi, hi_, li);
      G[gt_offset(j, y, yp, 0, ny, nt, kc)] = hr;
      G[gt_offset(j, y, yp, 1, ny, nt, kc)] = hi_;
      G[gt_offset(j, y, yp, 2, ny, nt, kc)] = lr;
      G[gt_offset(j, y, yp, 3, ny, nt, kc)] = li;
    }
  }
}

// per-image CG scalars of iteration it: beta = rr(it) / rr(it-1) (0 at it = 0),
// done flag, and the bound pn on the new direction's entries (|p| <= ||p|| <=
// ||r|| + beta ||p_prev||) with its power-of-two FP16 scale
__global__ void k_gram_scalars(CgArgs a, int it, float* beta, int* done, double* pn, float* pscale) {
  const int b = blockIdx.x;
  const double* base = a.rr_part + (size_t)b * (a.itmax + 1) * a.PB;
  const double rr = warp_sum_parts(base + (size_t)it * a.PB, a.PB);
  const double rr0 = warp_sum_parts(base, a.PB);
  const double rrp = it > 0 ? warp_sum_parts(base + (size_t)(it - 1) * a.PB, a.PB) : 1.0;
  if (threadIdx.x == 0) {
    done[b] = !(rr > a.rtol2 * rr0);
    const float bt = it > 0 ? (float)(rr / rrp) : 0.f;
    beta[b] = bt;
    if (pn) {
      const double p = sqrt(fmax(rr, 0.0)) + (it > 0 ? (double)bt * pn[b] : 0.0);
      pn[b] = p;
      pscale[b] = pow2_scale(p);
    }
  }
}

// FP16 operand scale of an operator application: from max |x| over the image
__global__ void __launch_bounds__(256) k_gram_apply_scale(const float* __restrict__ x, int64_t n2, float* pscale) {
  __shared__ float red[8];
  const float* xb = x + (size_t)blockIdx.x * n2;
  float m = 0.f;
  for (int64_t i = threadIdx.x; i < n2; i += 256) m = fmaxf(m, fabsf(xb[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = red[0];
    for (int w = 1; w < 8; ++w) t = fmaxf(t, red[w]);
    pscale[blockIdx.x] = pow2_scale((double)t);
  }
}

// ---------------------------------------------------------------------------
// layout conversion: natural [b][y][x] complex <-> column-planar [b][x][re|im][y]
// ---------------------------------------------------------------------------
__global__ void k_to_cp(const float2* __restrict__ in, float* __restrict__ out, int ny, int nx) {
  __shared__ float2 tile[32][33];
  const int b = blockIdx.z, x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  const int64_t n = (int64_t)ny * nx;
  const float2* src = in + (size_t)b * n;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int y = y0 + r, x = x0 + threadIdx.x;
    if (y < ny && x < nx) tile[r][threadIdx.x] = src[(int64_t)y * nx + x];
  }
  __syncthreads();
  float* dst = out + (size_t)b * 2 * n;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int x = x0 + r, y = y0 + threadIdx.x;
    if (y < ny && x < nx) {
      const float2 v = tile[threadIdx.x][r];
      dst[(int64_t)x * 2 * ny + y] = v.x;
      dst[(int64_t)x * 2 * ny + ny + y] = v.y;
    }
  }
}

__global__ void k_from_cp(const float* __restrict__ in, float2* __restrict__ out, int ny, int nx) {
  __shared__ float2 tile[32][33];
  const int b = blockIdx.z, x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  const int64_t n = (int64_t)ny * nx;
  const float* src = in + (size_t)b * 2 * n;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int x = x0 + r, y = y0 + threadIdx.x;
    if (y < ny && x < nx)
      tile[threadIdx.x][r] = make_float2(src[(int64_t)x * 2 * ny + y], src[(int64_t)x * 2 * ny + ny + y]);
  }
  __syncthreads();
  float2* dst = out + (size_t)b * n;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int y = y0 + r, x = x0 + threadIdx.x;
    if (y < ny && x < nx) dst[(int64_t)y * nx + x] = tile[r][threadIdx.x];
  }
}

// ---------------------------------------------------------------------------
// per-column CG: the epilogue of one CG update (column-CG mode)
// ---------------------------------------------------------------------------
// With CG run separately on every readout column j (A^H A is block diagonal
// over columns), the update of column j needs only sums over that column's
// ny rows: p^H q for alpha, then ||r||^2 for beta.  The nyt CTAs that hold the
// row tiles of one (image tile, column) form a thread-block cluster and add
// their partial sums through distributed shared memory (each CTA sums the nyt
// partials in rank order, so all of them get the same bits), then every CTA
// updates x and r on its own rows:
//   phase A  q = D + lam p (D in tensor memory, p tiles by TMA) -> p^H q partial
//   exchange alpha = rr / p^H q
//   phase B  x += alpha p, r -= alpha q on (p, x, r) tiles in shared memory,
//            stored back by TMA; ||r_new||^2 partial
//   exchange beta = ||r_new||^2 / rr; the rank-0 CTA writes the column's
//            rr, beta, done and iteration count for the next launch
//   a last cluster barrier keeps every CTA alive until its peers have read
//   its exchange slots.
// Tiles are 128 images x 32 rows of one plane (128-byte swizzle), two planes
// (re, im) per vector; phase B keeps up to two (p, x, r) groups in flight in
// the idle pipeline buffers, phase A up to two p tiles after the first group.
__device__ __forceinline__ double* xch_of(float* beta_s) {
  return reinterpret_cast<double*>(beta_s + 2 * kGramRows);  // after beta and the FP16 row scales
}

template <int KC>
__device__ __forceinline__ void colcg_epilogue(uint8_t* sm, int S, uint32_t stage_bytes, uint64_t* pbar, double* xch,
                                               uint32_t tbase, int NT, int quarter, int row, int k, int j,
                                               int ytile, int n0, int m0, bool accok, float fsc, const GramArgs& g,
                                               const ColCgArgs& cc, const CUtensorMap& mPe, const CUtensorMap& mXe,
                                               const CUtensorMap& mRe) {
  constexpr uint32_t kPlane = kGramRows * 128;   // one plane of a 32-row tile: 16 KB
  constexpr uint32_t kTile = 2 * kPlane;         // re and im planes
  const int ng = NT / 32;
  const size_t area = (size_t)S * stage_bytes;
  const int nbB = area >= 6 * (size_t)kTile ? 2 : 1;
  const uint32_t aoff = 3 * kTile;
  const int nbA = (int)min((size_t)2, (area - aoff) / kTile);
  auto bbuf = [&](int gi) { return sm + (size_t)(gi % nbB) * 3 * kTile; };
  auto abuf = [&](int gi) { return sm + aoff + (size_t)(gi % nbA) * kTile; };
  const bool leader = threadIdx.x == 64;
  auto loadA = [&](int gi) {
    uint64_t* b = &pbar[gi % nbA];
    mbar_expect_tx(b, kTile);
    tma_load_4d(abuf(gi), &mPe, b, n0 + 32 * gi, 0, j, m0);
    tma_load_4d(abuf(gi) + kPlane, &mPe, b, n0 + 32 * gi, 1, j, m0);
  };
  auto loadB = [&](int gi) {
    uint64_t* b = &pbar[2 + gi % nbB];
    uint8_t* d = bbuf(gi);
    mbar_expect_tx(b, 3 * kTile);
    tma_load_4d(d, &mPe, b, n0 + 32 * gi, 0, j, m0);
    tma_load_4d(d + kPlane, &mPe, b, n0 + 32 * gi, 1, j, m0);
    tma_load_4d(d + kTile, &mXe, b, n0 + 32 * gi, 0, j, m0);
    tma_load_4d(d + kTile + kPlane, &mXe, b, n0 + 32 * gi, 1, j, m0);
    tma_load_4d(d + 2 * kTile, &mRe, b, n0 + 32 * gi, 0, j, m0);
    tma_load_4d(d + 2 * kTile + kPlane, &mRe, b, n0 + 32 * gi, 1, j, m0);
  };
  const bool inb = k < g.nb;
  const size_t cidx = (size_t)(inb ? k : 0) * g.nx + j;
  const bool live = accok && inb && !cc.done[cidx];
  const double rr = live ? cc.rr[cidx] : 0.0;
  const int sw = row & 7;  // 16-byte group swizzle of this row
  const float lam = g.lam;

  // ---- phase A: p^H q over this CTA's rows ----
  if (leader && accok) {
    for (int gi = 0; gi < nbA && gi < ng; ++gi) loadA(gi);
    loadB(0);
  }
  double pq = 0.0;
  for (int gi = 0; gi < ng; ++gi) {
    const bool pok = accok && mbar_wait(&pbar[gi % nbA], (gi / nbA) & 1);
    if (accok && !pok) set_err(g.err, 6);
    const float4* pre = reinterpret_cast<const float4*>(abuf(gi) + (size_t)row * 128);
    const float4* pim = reinterpret_cast<const float4*>(abuf(gi) + kPlane + (size_t)row * 128);
    const uint32_t ta = tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(32 * gi);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float dr[16], di[16];
      tmem_ld16x2(ta + 16 * h, ta + (uint32_t)NT + 16 * h, dr, di);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        dr[u] *= fsc;
        di[u] *= fsc;
      }
      if (live && pok) {
        float acc = 0.f;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int ph = (4 * h + v) ^ sw;
          const float4 pr = pre[ph], pi = pim[ph];
          acc = fmaf(pr.x, fmaf(lam, pr.x, dr[4 * v + 0]), acc);
          acc = fmaf(pr.y, fmaf(lam, pr.y, dr[4 * v + 1]), acc);
          acc = fmaf(pr.z, fmaf(lam, pr.z, dr[4 * v + 2]), acc);
          acc = fmaf(pr.w, fmaf(lam, pr.w, dr[4 * v + 3]), acc);
          acc = fmaf(pi.x, fmaf(lam, pi.x, di[4 * v + 0]), acc);
          acc = fmaf(pi.y, fmaf(lam, pi.y, di[4 * v + 1]), acc);
          acc = fmaf(pi.z, fmaf(lam, pi.z, di[4 * v + 2]), acc);
          acc = fmaf(pi.w, fmaf(lam, pi.w, di[4 * v + 3]), acc);
        }
        pq += (double)acc;
      }
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");  // every row of this p tile has been read
    if (leader && accok && gi + nbA < ng) loadA(gi + nbA);
  }
  // ---- exchange 1: p^H q over the whole column ----
  const int nyt = g.nyt;
  double pq_tot = pq;
  if (nyt > 1) {
    xch[row] = pq;
    cluster_sync_all();
    pq_tot = 0.0;
    for (int rk = 0; rk < nyt; ++rk) pq_tot += rk == ytile ? xch[row] : ld_dsmem_f64(&xch[row], (uint32_t)rk);
  }
  bool upd = live, broke = false;
  float alpha = 0.f;
  if (live) {
    if (!(pq_tot > 0.0) || !isfinite(pq_tot)) {
      upd = false;
      broke = true;
    } else {
      alpha = (float)(rr / pq_tot);
    }
  }
  // ---- phase B: x += alpha p, r -= alpha q; ||r_new||^2 ----
  if (leader && accok && nbB > 1 && ng > 1) loadB(1);  // the phase-A buffers are free now
  double rrn = 0.0;
  for (int gi = 0; gi < ng; ++gi) {
    const bool bok = accok && mbar_wait(&pbar[2 + gi % nbB], (gi / nbB) & 1);
    if (accok && !bok) set_err(g.err, 7);
    uint8_t* d = bbuf(gi);
    const float4* pre = reinterpret_cast<const float4*>(d + (size_t)row * 128);
    const float4* pim = reinterpret_cast<const float4*>(d + kPlane + (size_t)row * 128);
    float4* xre = reinterpret_cast<float4*>(d + kTile + (size_t)row * 128);
    float4* xim = reinterpret_cast<float4*>(d + kTile + kPlane + (size_t)row * 128);
    float4* rre = reinterpret_cast<float4*>(d + 2 * kTile + (size_t)row * 128);
    float4* rim = reinterpret_cast<float4*>(d + 2 * kTile + kPlane + (size_t)row * 128);
    const uint32_t ta = tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(32 * gi);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float dr[16], di[16];
      tmem_ld16x2(ta + 16 * h, ta + (uint32_t)NT + 16 * h, dr, di);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        dr[u] *= fsc;
        di[u] *= fsc;
      }
      if (upd && bok) {
        float acc = 0.f;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int ph = (4 * h + v) ^ sw;
          const float pa[4] = {pre[ph].x, pre[ph].y, pre[ph].z, pre[ph].w};
          const float pb[4] = {pim[ph].x, pim[ph].y, pim[ph].z, pim[ph].w};
          float xa[4] = {xre[ph].x, xre[ph].y, xre[ph].z, xre[ph].w};
          float xb[4] = {xim[ph].x, xim[ph].y, xim[ph].z, xim[ph].w};
          float ra[4] = {rre[ph].x, rre[ph].y, rre[ph].z, rre[ph].w};
          float rb[4] = {rim[ph].x, rim[ph].y, rim[ph].z, rim[ph].w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            xa[e] = fmaf(alpha, pa[e], xa[e]);
            xb[e] = fmaf(alpha, pb[e], xb[e]);
            ra[e] = fmaf(-alpha, fmaf(lam, pa[e], dr[4 * v + e]), ra[e]);
            rb[e] = fmaf(-alpha, fmaf(lam, pb[e], di[4 * v + e]), rb[e]);
            acc = fmaf(ra[e], ra[e], fmaf(rb[e], rb[e], acc));
          }
          xre[ph] = make_float4(xa[0], xa[1], xa[2], xa[3]);
          xim[ph] = make_float4(xb[0], xb[1], xb[2], xb[3]);
          rre[ph] = make_float4(ra[0], ra[1], ra[2], ra[3]);
          rim[ph] = make_float4(rb[0], rb[1], rb[2], rb[3]);
        }
        rrn += (double)acc;
      }
    }
    // every row of this group is written before one thread stores the x and r tiles
    fence_proxy_async_smem();
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (leader && bok) {
      tma_store_4d(&mXe, d + kTile, n0 + 32 * gi, 0, j, m0);
      tma_store_4d(&mXe, d + kTile + kPlane, n0 + 32 * gi, 1, j, m0);
      tma_store_4d(&mRe, d + 2 * kTile, n0 + 32 * gi, 0, j, m0);
      tma_store_4d(&mRe, d + 2 * kTile + kPlane, n0 + 32 * gi, 1, j, m0);
      bulk_commit();
      if (gi + nbB < ng) {
        bulk_wait_read();
        loadB(gi + nbB);
      }
    }
  }
  if (leader) bulk_wait_all();
  // ---- exchange 2: ||r_new||^2 over the whole column; the next step ----
  double rr_tot = rrn;
  if (nyt > 1) {
    xch[kGramRows + row] = rrn;
    cluster_sync_all();
    rr_tot = 0.0;
    for (int rk = 0; rk < nyt; ++rk)
      rr_tot += rk == ytile ? xch[kGramRows + row] : ld_dsmem_f64(&xch[kGramRows + row], (uint32_t)rk);
  }
  if (ytile == 0 && live) {
    if (upd && isfinite(rr_tot)) {
      cc.rr[cidx] = rr_tot;
      cc.iters[cidx] += 1;
      const bool stop = !(rr_tot > cc.rtol2 * cc.rr0[cidx]);
      const float bt = stop ? 0.f : (float)(rr_tot / rr);
      cc.beta[cidx] = bt;
      if (stop) cc.done[cidx] = 1;
      if (cc.pn) {  // bound on the next direction r + beta p: sqrt(rr_new) + beta pn
        const double p = sqrt(rr_tot) + (double)bt * cc.pn[cidx];
        cc.pn[cidx] = p;
        cc.pscale[cidx] = pow2_scale(p);
      }
    } else {
      broke = true;
    }
    if (broke) {
      cc.done[cidx] = 1;
      cc.beta[cidx] = 0.f;
      cc.status[k] = 5;
    }
  }
  // no CTA leaves while a peer may still read its exchange slots
  if (nyt > 1) cluster_sync_all();
}

// ---------------------------------------------------------------------------
// the tensor-core normal operator
// ---------------------------------------------------------------------------
// CTA (y tile, image tile, column j).  Warp 0: TMA producer.  Warp 1: TMEM
// owner and MMA issuer.  Warps 2-5: split the direction into TF32 head and
// remainder in shared memory during the main loop, then run the epilogue
// (tensor memory -> q = G p + lam p, the new direction p, the p^H q partial).
// Pipeline per contraction chunk (16 values of y'): stage s holds
//   A: [r_re | r_im | pold_re | pold_im] 128 x 16 fp32 each, rewritten in place
//      as [p_re hi | p_im hi | p_re lo | p_im lo]
//   B: [G_re hi | G_im hi | G_re lo | G_im lo] NT x 16 fp32 each
// and D_re (columns 0..NT-1), D_im (NT..2NT-1) accumulate in tensor memory:
//   D_re += p_re G_re^T - p_im G_im^T,  D_im += p_re G_im^T + p_im G_re^T.
// With AT (tiles with 2 NT + 4 KC S <= 512 tensor-memory columns) the split
// direction goes to tensor memory instead, [p_re hi | p_im hi | p_re lo |
// p_im lo] KC columns each per stage from column 2 NT, one image per lane,
// and the MMAs read A from there: shared memory then carries only the TMA
// tiles and the B operand reads, which keeps the tensor pipe, not the
// shared-memory bandwidth, the limit of the main loop.
template <int KC, bool AT, bool COL, bool F16>
__global__ void __launch_bounds__(kGramThreads, 1)
    k_gram_normal(const __grid_constant__ CUtensorMap mIn, const __grid_constant__ CUtensorMap mPold,
                  const __grid_constant__ CUtensorMap mPe, const __grid_constant__ CUtensorMap mQe,
                  const __grid_constant__ CUtensorMap mRe, GramArgs g, ColCgArgs cc) {
  static_assert(!F16 || (KC == 16 && !AT), "the FP16 split runs with 16-value stages in shared memory");
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  const int NT = g.nt, S = g.stages;
  using T = GramTile<KC>;
  using H = GramTile<8>;  // FP16 operands: 32-byte rows, 32-byte swizzle (byte-identical to 8 FP32 values)
  constexpr uint32_t kATile = T::kATile;
  constexpr uint32_t kASplit = F16 ? kGramRows * 32 : 0;  // one FP16 plane of the split direction
  const uint32_t btile = F16 ? (uint32_t)NT * 32 : (uint32_t)NT * KC * 4;
  const uint32_t stage_bytes = 4 * kATile + 4 * kASplit + 4 * btile;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + (size_t)S * stage_bytes);
  uint64_t* full = bars;
  uint64_t* conv = bars + S;
  uint64_t* empty = bars + 2 * S;
  uint64_t* accf = bars + 3 * S;
  uint64_t* pbar = bars + 3 * S + 1;   // epilogue staging of p: up to 8 buffers, one phase per use
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 3 * S + 9);
  float* beta_s = reinterpret_cast<float*>(tslot + 4);
  float* ps_s = beta_s + kGramRows;  // FP16: power-of-two scale of each image's direction

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ytile = blockIdx.x % g.nyt, itile = blockIdx.x / g.nyt, j = blockIdx.y;
  const int n0 = ytile * NT, m0 = itile * kGramRows;
  const int nkc = g.ny / KC;
  const bool use_pold = g.cg && g.it > 0;

  auto slotA = [&](int s, int q) { return sm + (size_t)s * stage_bytes + (size_t)q * kATile; };
  auto slotAS = [&](int s, int q) { return sm + (size_t)s * stage_bytes + 4 * kATile + (size_t)q * kASplit; };
  auto slotB = [&](int s, int q) {
    return sm + (size_t)s * stage_bytes + 4 * kATile + 4 * kASplit + (size_t)q * btile;
  };
  // one stage: the A inputs by TMA (r, and p_old after the first iteration),
  // the stage-tiled B block of G_j by one bulk copy
  const uint32_t stage_tx = (use_pold ? 4u : 2u) * kATile + 4u * btile;
  const uint8_t* gsrc = static_cast<const uint8_t*>(g.G) + ((size_t)j * g.nyt + ytile) * nkc * 4 * btile;
  auto issue = [&](int kc) {
    const int s = kc % S, y0 = kc * KC;
    mbar_expect_tx(&full[s], stage_tx);
    tma_load_4d(slotA(s, 0), &mIn, &full[s], y0, 0, j, m0);
    tma_load_4d(slotA(s, 1), &mIn, &full[s], y0, 1, j, m0);
    if (use_pold) {
      tma_load_4d(slotA(s, 2), &mPold, &full[s], y0, 0, j, m0);
      tma_load_4d(slotA(s, 3), &mPold, &full[s], y0, 1, j, m0);
    }
    bulk_load(slotB(s, 0), gsrc + (size_t)kc * 4 * btile, 4u * btile, &full[s]);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 128);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    if (g.tma_epi) {
      for (int b = 0; b < 8; ++b) mbar_init(&pbar[b], 1);
    } else {
      mbar_init(&pbar[0], 128);
      mbar_init(&pbar[1], 128);
    }
    fence_mbar_init();
    // the first S stages need no free-slot wait: start them before the
    // tensor-memory allocation and the block-wide barrier
    tma_prefetch_desc(&mIn);
    if (use_pold) tma_prefetch_desc(&mPold);
    for (int kc = 0; kc < S && kc < nkc; ++kc) issue(kc);
  }
  if (warp >= 2) {
    const int r = threadIdx.x - 64;
    const int k = m0 + r;
    if constexpr (COL)
      beta_s[r] = (use_pold && k < g.nb) ? cc.beta[(size_t)k * g.nx + j] : 0.f;
    else
      beta_s[r] = (use_pold && k < g.nb) ? g.beta[k] : 0.f;
    if constexpr (F16) {
      if constexpr (COL)
        ps_s[r] = k < g.nb ? cc.pscale[(size_t)k * g.nx + j] : 1.f;
      else
        ps_s[r] = k < g.nb ? g.pscale[k] : 1.f;
    }
  }
  if (warp == 1) tmem_alloc(tslot, g.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      for (int kc = S; kc < nkc; ++kc) {
        if (!mbar_wait(&empty[kc % S], ((kc / S) - 1) & 1)) {
          set_err(g.err, 1);
          break;
        }
        issue(kc);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id = idesc_tf32(kGramRows, NT, false), idn = idesc_tf32(kGramRows, NT, true);
      const uint32_t dre = tbase, dim = tbase + (uint32_t)NT;
      for (int kc = 0; kc < nkc; ++kc) {
        const int s = kc % S;
        if (!mbar_wait(&conv[s], (kc / S) & 1)) {
          set_err(g.err, 2);
          break;
        }
        tc_fence_after();
        if constexpr (AT) {
          const uint32_t a0 = tbase + 2u * NT + (uint32_t)(s * 4 * KC);
          const uint32_t bhr = smem_u32(slotB(s, 0)), bhi = smem_u32(slotB(s, 1));
          const uint32_t blr = smem_u32(slotB(s, 2)), bli = smem_u32(slotB(s, 3));
#pragma unroll
          for (int kk = 0; kk < KC / 8; ++kk) {
            const uint32_t o = 32u * kk, c = 8u * kk;
            const uint32_t acc0 = (kc == 0 && kk == 0) ? 0u : 1u;
            const uint32_t Ahr = a0 + c, Ahi = a0 + KC + c, Alr = a0 + 2 * KC + c, Ali = a0 + 3 * KC + c;
            const uint64_t Bhr = T::desc(bhr + o), Bhi = T::desc(bhi + o);
            const uint64_t Blr = T::desc(blr + o), Bli = T::desc(bli + o);
            mma_tf32_ts(dre, Ahr, Bhr, id, acc0);
            mma_tf32_ts(dre, Ahr, Blr, id, 1);
            mma_tf32_ts(dre, Alr, Bhr, id, 1);
            mma_tf32_ts(dre, Ahi, Bhi, idn, 1);
            mma_tf32_ts(dre, Ahi, Bli, idn, 1);
            mma_tf32_ts(dre, Ali, Bhi, idn, 1);
            mma_tf32_ts(dim, Ahr, Bhi, id, acc0);
            mma_tf32_ts(dim, Ahr, Bli, id, 1);
            mma_tf32_ts(dim, Alr, Bhi, id, 1);
            mma_tf32_ts(dim, Ahi, Bhr, id, 1);
            mma_tf32_ts(dim, Ahi, Blr, id, 1);
            mma_tf32_ts(dim, Ali, Bhr, id, 1);
          }
          mma_commit(&empty[s]);
          continue;
        }
        if constexpr (F16) {
          // one K = 16 step per stage: 3 split products x 4 real products
          const uint32_t hd = idesc_f16(kGramRows, NT, false), hdn = idesc_f16(kGramRows, NT, true);
          const uint32_t acc0 = kc == 0 ? 0u : 1u;
          const uint64_t Ahr = H::desc(smem_u32(slotAS(s, 0))), Ahi = H::desc(smem_u32(slotAS(s, 1)));
          const uint64_t Alr = H::desc(smem_u32(slotAS(s, 2))), Ali = H::desc(smem_u32(slotAS(s, 3)));
          const uint64_t Bhr = H::desc(smem_u32(slotB(s, 0))), Bhi = H::desc(smem_u32(slotB(s, 1)));
          const uint64_t Blr = H::desc(smem_u32(slotB(s, 2))), Bli = H::desc(smem_u32(slotB(s, 3)));
          mma_f16(dre, Ahr, Bhr, hd, acc0);
          mma_f16(dre, Ahr, Blr, hd, 1);
          mma_f16(dre, Alr, Bhr, hd, 1);
          mma_f16(dre, Ahi, Bhi, hdn, 1);
          mma_f16(dre, Ahi, Bli, hdn, 1);
          mma_f16(dre, Ali, Bhi, hdn, 1);
          mma_f16(dim, Ahr, Bhi, hd, acc0);
          mma_f16(dim, Ahr, Bli, hd, 1);
          mma_f16(dim, Alr, Bhi, hd, 1);
          mma_f16(dim, Ahi, Bhr, hd, 1);
          mma_f16(dim, Ahi, Blr, hd, 1);
          mma_f16(dim, Ali, Bhr, hd, 1);
          mma_commit(&empty[s]);
          continue;
        }
        const uint32_t ahr = smem_u32(slotA(s, 0)), ahi = smem_u32(slotA(s, 1));
        const uint32_t alr = smem_u32(slotA(s, 2)), ali = smem_u32(slotA(s, 3));
        const uint32_t bhr = smem_u32(slotB(s, 0)), bhi = smem_u32(slotB(s, 1));
        const uint32_t blr = smem_u32(slotB(s, 2)), bli = smem_u32(slotB(s, 3));
#pragma unroll
        for (int kk = 0; kk < KC / 8; ++kk) {
          const uint32_t o = 32u * kk;
          const uint32_t acc0 = (kc == 0 && kk == 0) ? 0u : 1u;
          const uint64_t Ahr = T::desc(ahr + o), Ahi = T::desc(ahi + o);
          const uint64_t Alr = T::desc(alr + o), Ali = T::desc(ali + o);
          const uint64_t Bhr = T::desc(bhr + o), Bhi = T::desc(bhi + o);
          const uint64_t Blr = T::desc(blr + o), Bli = T::desc(bli + o);
          // D_re += p_re G_re^T - p_im G_im^T
          mma_tf32(dre, Ahr, Bhr, id, acc0);
          mma_tf32(dre, Ahr, Blr, id, 1);
          mma_tf32(dre, Alr, Bhr, id, 1);
          mma_tf32(dre, Ahi, Bhi, idn, 1);
          mma_tf32(dre, Ahi, Bli, idn, 1);
          mma_tf32(dre, Ali, Bhi, idn, 1);
          // D_im += p_re G_im^T + p_im G_re^T
          mma_tf32(dim, Ahr, Bhi, id, acc0);
          mma_tf32(dim, Ahr, Bli, id, 1);
          mma_tf32(dim, Alr, Bhi, id, 1);
          mma_tf32(dim, Ahi, Bhr, id, 1);
          mma_tf32(dim, Ahi, Blr, id, 1);
          mma_tf32(dim, Ali, Bhr, id, 1);
        }
        mma_commit(&empty[s]);
      }
      mma_commit(accf);
    }
  }
  if (COL && warp < 2) {
    // the epilogue's three cluster-wide exchanges: every thread of the cluster takes part
    if (g.nyt > 1)
      for (int e = 0; e < 3; ++e) cluster_sync_all();
  } else if (warp < 2) {
  } else {
    // ---- split p = r + beta p_old into TF32 head / remainder, in place ----
    // The chunks inside this CTA's output rows [n0, n0 + NT) also store p to
    // the new direction buffer (un-swizzling the 16-byte chunk index).
    const int e = threadIdx.x - 64;  // 0..127
    const int kc_lo = n0 / KC, kc_hi = (n0 + NT) / KC;
    const size_t img2 = (size_t)2 * g.ny * g.nx;
    bool ok = true;
    if constexpr (AT) {
      // one image per thread: row = tensor-memory lane of this warp's quarter
      const int rowi = 32 * (warp & 3) + lane, kimg = m0 + rowi;
      const float b = beta_s[rowi];
      const uint32_t tl = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + 2u * NT;
      float* pdst = (g.pnew && kimg < g.nb) ? g.pnew + (size_t)kimg * img2 + (size_t)j * 2 * g.ny : nullptr;
      for (int kc = 0; kc < nkc; ++kc) {
        const int s = kc % S;
        if (ok && !mbar_wait(&full[s], (kc / S) & 1)) {
          set_err(g.err, 3);
          ok = false;
        }
        ok = __all_sync(0xffffffffu, ok);  // the tensor-memory stores are warp-collective
        tc_fence_after();
        if (ok) {
          const float4* r_re = reinterpret_cast<const float4*>(slotA(s, 0)) + rowi * (KC / 4);
          const float4* r_im = reinterpret_cast<const float4*>(slotA(s, 1)) + rowi * (KC / 4);
          const float4* o_re = reinterpret_cast<const float4*>(slotA(s, 2)) + rowi * (KC / 4);
          const float4* o_im = reinterpret_cast<const float4*>(slotA(s, 3)) + rowi * (KC / 4);
          float vr[KC], vi[KC];
#pragma unroll
          for (int c = 0; c < KC / 4; ++c) {
            const int ph = T::chunk(c, rowi);  // the swizzle is an involution
            float4 a = r_re[ph], d = r_im[ph];
            if (use_pold) {
              const float4 w = o_re[ph], u = o_im[ph];
              a.x = fmaf(b, w.x, a.x); a.y = fmaf(b, w.y, a.y); a.z = fmaf(b, w.z, a.z); a.w = fmaf(b, w.w, a.w);
              d.x = fmaf(b, u.x, d.x); d.y = fmaf(b, u.y, d.y); d.z = fmaf(b, u.z, d.z); d.w = fmaf(b, u.w, d.w);
            }
            vr[4 * c] = a.x; vr[4 * c + 1] = a.y; vr[4 * c + 2] = a.z; vr[4 * c + 3] = a.w;
            vi[4 * c] = d.x; vi[4 * c + 1] = d.y; vi[4 * c + 2] = d.z; vi[4 * c + 3] = d.w;
            if (pdst && kc >= kc_lo && kc < kc_hi) {
              reinterpret_cast<float4*>(pdst + kc * KC)[c] = a;
              reinterpret_cast<float4*>(pdst + g.ny + kc * KC)[c] = d;
            }
          }
          float hr[KC], lr[KC], hi_[KC], li[KC];
#pragma unroll
          for (int i = 0; i < KC; ++i) {
            split_tf32(vr[i], hr[i], lr[i]);
            split_tf32(vi[i], hi_[i], li[i]);
          }
          const uint32_t ta = tl + (uint32_t)(s * 4 * KC);
          if constexpr (KC == 16) {
            tmem_st16(ta, hr);
            tmem_st16(ta + KC, hi_);
            tmem_st16(ta + 2 * KC, lr);
            tmem_st16(ta + 3 * KC, li);
          } else {
            tmem_st8(ta, hr);
            tmem_st8(ta + KC, hi_);
            tmem_st8(ta + 2 * KC, lr);
            tmem_st8(ta + 3 * KC, li);
          }
          tmem_wait_st();
        }
        tc_fence_before();
        mbar_arrive(&conv[s]);
      }
    } else
    for (int kc = 0; kc < nkc; ++kc) {
      const int s = kc % S;
      if (ok && !mbar_wait(&full[s], (kc / S) & 1)) {
        set_err(g.err, 3);
        ok = false;
      }
      if (ok) {
        float4* r_re = reinterpret_cast<float4*>(slotA(s, 0));
        float4* r_im = reinterpret_cast<float4*>(slotA(s, 1));
        float4* p_re = reinterpret_cast<float4*>(slotA(s, 2));
        float4* p_im = reinterpret_cast<float4*>(slotA(s, 3));
#pragma unroll
        for (int i = 0; i < KC / 4; ++i) {
          const int q = e + 128 * i;  // float4 index in the 128 x KC tile; row = q / (KC/4)
          const float b = beta_s[q / (KC / 4)];
          float4 vr = r_re[q], vi = r_im[q];
          if (use_pold) {
            const float4 wr = p_re[q], wi = p_im[q];
            vr.x = fmaf(b, wr.x, vr.x); vr.y = fmaf(b, wr.y, vr.y);
            vr.z = fmaf(b, wr.z, vr.z); vr.w = fmaf(b, wr.w, vr.w);
            vi.x = fmaf(b, wi.x, vi.x); vi.y = fmaf(b, wi.y, vi.y);
            vi.z = fmaf(b, wi.z, vi.z); vi.w = fmaf(b, wi.w, vi.w);
          }
          if (g.pnew && kc >= kc_lo && kc < kc_hi) {
            const int rowi = q / (KC / 4), kimg = m0 + rowi;
            if (kimg < g.nb) {
              const int chunk = T::chunk(q % (KC / 4), rowi);
              const size_t o = (size_t)kimg * img2 + (size_t)j * 2 * g.ny + (size_t)kc * KC + 4 * chunk;
              *reinterpret_cast<float4*>(g.pnew + o) = vr;
              *reinterpret_cast<float4*>(g.pnew + o + g.ny) = vi;
            }
          }
          if constexpr (F16) {
            // scaled by the image's power of two, split into FP16 head and remainder,
            // written to the stage's split planes (32-byte rows, 32-byte swizzle)
            const int rowi = q / (KC / 4), lc = T::chunk(q % (KC / 4), rowi);
            const float sc = ps_s[rowi];
            uint2 hre, him, lre, lim;
            split_f16x4(vr.x * sc, vr.y * sc, vr.z * sc, vr.w * sc, hre, lre);
            split_f16x4(vi.x * sc, vi.y * sc, vi.z * sc, vi.w * sc, him, lim);
            const size_t off = (size_t)rowi * 32 + (size_t)(((lc >> 1) ^ ((rowi >> 2) & 1)) * 16) + (lc & 1) * 8;
            *reinterpret_cast<uint2*>(slotAS(s, 0) + off) = hre;
            *reinterpret_cast<uint2*>(slotAS(s, 1) + off) = him;
            *reinterpret_cast<uint2*>(slotAS(s, 2) + off) = lre;
            *reinterpret_cast<uint2*>(slotAS(s, 3) + off) = lim;
          } else {
            float4 hr, lr, hi4, li;
            split_tf32(vr.x, hr.x, lr.x); split_tf32(vr.y, hr.y, lr.y);
            split_tf32(vr.z, hr.z, lr.z); split_tf32(vr.w, hr.w, lr.w);
            split_tf32(vi.x, hi4.x, li.x); split_tf32(vi.y, hi4.y, li.y);
            split_tf32(vi.z, hi4.z, li.z); split_tf32(vi.w, hi4.w, li.w);
            r_re[q] = hr;
            r_im[q] = hi4;
            p_re[q] = lr;
            p_im[q] = li;
          }
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(&conv[s]);
    }

    // ---- epilogue ----
    // p of this CTA's rows (stored above by the split warps, or the input x in
    // apply mode) is staged into the now idle pipeline buffers by bulk copies,
    // [row][re|im][W] with a 16-byte pad per row (conflict-free row reads), in
    // passes of W output rows over two buffers: the next pass's p arrives, and
    // the previous pass's q leaves, while a pass computes.  Each thread
    // overwrites its row with q and stores it back with two contiguous bulk
    // copies (one image per thread, so direct stores would touch 32 cache
    // lines per warp instruction).  Rows are private to their thread, so a
    // buffer is reloaded as soon as its own thread's stores have read it.
    fence_proxy_async_global();
    __threadfence_block();
    asm volatile("bar.sync 1, 128;" ::: "memory");
    const int quarter = warp & 3;          // TMEM lanes 32*quarter .. +31
    const int row = 32 * quarter + lane;
    const int k = m0 + row;
    const bool accok = mbar_wait(accf, 0);
    if (!accok) set_err(g.err, 4);
    tc_fence_after();
    // FP16 operands were scaled by powers of two (G_j by gscale[j], the image's
    // direction by ps_s[row]): undo both on the accumulator
    const float fsc = F16 ? 1.f / (g.gscale[j] * ps_s[row]) : 1.f;
    if constexpr (COL) {
      colcg_epilogue<KC>(sm, S, stage_bytes, pbar, xch_of(beta_s), tbase, NT, quarter, row, k, j, ytile, n0, m0,
                         accok, fsc, g, cc, mPe, mQe, mRe);
    } else {
    const bool inb = k < g.nb;
    const bool valid = accok && inb && !(g.cg && g.done[k]);
    const size_t col = (size_t)(inb ? k : 0) * img2 + (size_t)j * 2 * g.ny;
    const float* psrc = g.cg ? g.pnew : g.in;
    if (g.tma_epi) {
      // Passes of 32 output rows: p re / im of the 128 images arrive as two
      // 128-byte-swizzled tensor tiles (rows = images), q overwrites them in
      // place and leaves by two tensor stores; as many passes as fit are in
      // flight at once.  The maps cover exactly this launch's nb images, so
      // rows past the batch are neither read nor written.
      constexpr uint32_t kPlane = kGramRows * 128;
      const int ng = NT / 32;
      const int nbuf = min(min(ng, 8), (int)((size_t)S * stage_bytes / (2 * kPlane)));
      const bool leader = threadIdx.x == 64;
      auto ebuf = [&](int gi) { return sm + (size_t)(gi % nbuf) * 2 * kPlane; };
      auto eload = [&](int gi) {
        uint64_t* b = &pbar[gi % nbuf];
        mbar_expect_tx(b, 2 * kPlane);
        tma_load_4d(ebuf(gi), &mPe, b, n0 + 32 * gi, 0, j, m0);
        tma_load_4d(ebuf(gi) + kPlane, &mPe, b, n0 + 32 * gi, 1, j, m0);
      };
      if (leader && accok)
        for (int gi = 0; gi < nbuf; ++gi) eload(gi);
      double pq = 0.0;
      const int sw = row & 7;  // 16-byte group swizzle of this row
      for (int gi = 0; gi < ng; ++gi) {
        const bool pok = accok && mbar_wait(&pbar[gi % nbuf], (gi / nbuf) & 1);
        if (accok && !pok) set_err(g.err, 5);
        float4* pre = reinterpret_cast<float4*>(ebuf(gi) + (size_t)row * 128);
        float4* pim = reinterpret_cast<float4*>(ebuf(gi) + kPlane + (size_t)row * 128);
        const uint32_t ta = tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(32 * gi);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float dr[16], di[16];
          tmem_ld16x2(ta + 16 * h, ta + (uint32_t)NT + 16 * h, dr, di);
          if (F16) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              dr[u] *= fsc;
              di[u] *= fsc;
            }
          }
          if (valid && pok) {
            float acc = 0.f;  // p^H q over these 16 rows in FP32, then summed in FP64
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const int ph = (4 * h + v) ^ sw;
              const float4 pr = pre[ph], pi = pim[ph];
              float4 qr, qi;
              qr.x = fmaf(g.lam, pr.x, dr[4 * v + 0]); qr.y = fmaf(g.lam, pr.y, dr[4 * v + 1]);
              qr.z = fmaf(g.lam, pr.z, dr[4 * v + 2]); qr.w = fmaf(g.lam, pr.w, dr[4 * v + 3]);
              qi.x = fmaf(g.lam, pi.x, di[4 * v + 0]); qi.y = fmaf(g.lam, pi.y, di[4 * v + 1]);
              qi.z = fmaf(g.lam, pi.z, di[4 * v + 2]); qi.w = fmaf(g.lam, pi.w, di[4 * v + 3]);
              pre[ph] = qr;
              pim[ph] = qi;
              acc = fmaf(pr.x, qr.x, acc); acc = fmaf(pr.y, qr.y, acc);
              acc = fmaf(pr.z, qr.z, acc); acc = fmaf(pr.w, qr.w, acc);
              acc = fmaf(pi.x, qi.x, acc); acc = fmaf(pi.y, qi.y, acc);
              acc = fmaf(pi.z, qi.z, acc); acc = fmaf(pi.w, qi.w, acc);
            }
            pq += (double)acc;
          }
        }
        // every row of this pass is written before one thread stores the tiles
        // (rows of converged images still hold p: the CG update skips them)
        fence_proxy_async_smem();
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (leader && pok) {
          tma_store_4d(&mQe, ebuf(gi), n0 + 32 * gi, 0, j, m0);
          tma_store_4d(&mQe, ebuf(gi) + kPlane, n0 + 32 * gi, 1, j, m0);
          bulk_commit();
          if (gi + nbuf < ng) {
            bulk_wait_read();
            eload(gi + nbuf);
          }
        }
      }
      if (leader) bulk_wait_read();
      if (valid && g.pq) g.pq[((size_t)k * g.itmax + g.it) * g.PA + (size_t)j * g.nyt + ytile] = pq;
    } else {
    int W2 = NT;  // widest pass for which two buffers fit
    while (W2 > 16 && 2 * (size_t)kGramRows * (8u * W2 + 16u) > (size_t)S * stage_bytes) W2 -= 16;
    const int np = (NT + W2 - 1) / W2;
    const int W = ((NT + np - 1) / np + 15) / 16 * 16;
    const uint32_t pitch = 8u * W + 16u;
    auto rowbuf = [&](int i) { return reinterpret_cast<float*>(sm + ((size_t)(i & 1) * kGramRows + row) * pitch); };
    auto stage_p = [&](int i) {
      // every thread arrives once per use, announcing its own bytes before
      // issuing them
      const int w0 = i * W, wn = min(W, NT - w0);
      if (accok && inb) {
        float* pr = rowbuf(i);
        mbar_expect_tx(&pbar[i & 1], 8u * wn);
        bulk_load(pr, psrc + col + n0 + w0, 4u * wn, &pbar[i & 1]);
        bulk_load(pr + W, psrc + col + g.ny + n0 + w0, 4u * wn, &pbar[i & 1]);
      } else {
        mbar_arrive(&pbar[i & 1]);
      }
    };
    stage_p(0);
    if (np > 1) stage_p(1);
    double pq = 0.0;
    for (int i = 0; i < np; ++i) {
      const int w0 = i * W, wn = min(W, NT - w0);
      const bool pok = mbar_wait(&pbar[i & 1], (i >> 1) & 1);
      if (!pok) set_err(g.err, 5);
      float* prow = rowbuf(i);
      for (int c = 0; c < wn / 16; ++c) {
        float dr[16], di[16];
        const uint32_t ta = tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(w0 + 16 * c);
        tmem_ld16x2(ta, ta + (uint32_t)NT, dr, di);
        if (F16) {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            dr[u] *= fsc;
            di[u] *= fsc;
          }
        }
        if (valid && pok) {
          float4* pr4 = reinterpret_cast<float4*>(prow + 16 * c);
          float4* pi4 = reinterpret_cast<float4*>(prow + W + 16 * c);
          float acc = 0.f;  // p^H q over these 16 rows in FP32, then summed in FP64
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const float4 pr = pr4[v], pi = pi4[v];
            float4 qr, qi;
            qr.x = fmaf(g.lam, pr.x, dr[4 * v + 0]); qr.y = fmaf(g.lam, pr.y, dr[4 * v + 1]);
            qr.z = fmaf(g.lam, pr.z, dr[4 * v + 2]); qr.w = fmaf(g.lam, pr.w, dr[4 * v + 3]);
            qi.x = fmaf(g.lam, pi.x, di[4 * v + 0]); qi.y = fmaf(g.lam, pi.y, di[4 * v + 1]);
            qi.z = fmaf(g.lam, pi.z, di[4 * v + 2]); qi.w = fmaf(g.lam, pi.w, di[4 * v + 3]);
            pr4[v] = qr;
            pi4[v] = qi;
            acc = fmaf(pr.x, qr.x, acc); acc = fmaf(pr.y, qr.y, acc);
            acc = fmaf(pr.z, qr.z, acc); acc = fmaf(pr.w, qr.w, acc);
            acc = fmaf(pi.x, qi.x, acc); acc = fmaf(pi.y, qi.y, acc);
            acc = fmaf(pi.z, qi.z, acc); acc = fmaf(pi.w, qi.w, acc);
          }
          pq += (double)acc;
        }
      }
      if (valid && pok) {
        fence_proxy_async_smem();
        bulk_store(g.q + col + n0 + w0, prow, 4u * wn);
        bulk_store(g.q + col + g.ny + n0 + w0, prow + W, 4u * wn);
        bulk_commit();
      }
      if (i + 2 < np) {
        bulk_wait_read();  // this thread's row of buffer i & 1 has been stored
        stage_p(i + 2);
      }
    }
    bulk_wait_read();  // shared memory is read by the stores before the block exits

    if (valid && g.pq) g.pq[((size_t)k * g.itmax + g.it) * g.PA + (size_t)j * g.nyt + ytile] = pq;
    }
    }  // !COL
  }

  // teardown: every TMA issued has been consumed by the split warps (or they
  // timed out); the accumulator barrier orders the MMAs before the free
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tbase, g.tmem_cols);
  }
}

// x = 0 and the per-column CG scalars of nb right-hand sides (column-planar r)
__global__ void __launch_bounds__(64) k_colcg_init(ColCgArgs cc, int ny, int nx) {
  __shared__ double part[2];
  const int j = blockIdx.x, b = blockIdx.y;
  const size_t cidx = (size_t)b * nx + j;
  const float* rc = cc.r + cidx * 2 * ny;
  float* xc = cc.x + cidx * 2 * ny;
  double acc = 0.0;
  for (int i = threadIdx.x; i < 2 * ny; i += 64) {
    const double v = (double)rc[i];
    acc = fma(v, v, acc);
    xc[i] = 0.f;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double rr = part[0] + part[1];
    const_cast<double*>(cc.rr0)[cidx] = rr;
    cc.rr[cidx] = rr;
    cc.beta[cidx] = 0.f;
    cc.iters[cidx] = 0;
    if (cc.pn) {
      cc.pn[cidx] = sqrt(rr);  // p_0 = r_0
      cc.pscale[cidx] = pow2_scale(sqrt(rr));
    }
    const bool bad = !isfinite(rr);
    cc.done[cidx] = bad || !(rr > 0.0);
    if (bad) cc.status[b] = 5;  // a non-finite right-hand side: breakdown, x stays 0
  }
}

// *flag = 1 if a column is still iterating (the flag is zeroed before)
__global__ void k_colcg_any_live(ColCgArgs cc, int n, int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !cc.done[i]) atomicExch(flag, 1);
}

// per image: most updates of any column; ||r|| / ||b|| over the whole image
__global__ void k_colcg_report(ColCgArgs cc, int nx, int* iters, double* relres) {
  const int b = blockIdx.x;
  double r2 = 0.0, b2 = 0.0;
  int it = 0;
  for (int j = threadIdx.x; j < nx; j += 32) {
    const size_t c = (size_t)b * nx + j;
    r2 += cc.rr[c];
    b2 += cc.rr0[c];
    it = max(it, cc.iters[c]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    b2 += __shfl_xor_sync(0xffffffffu, b2, o);
    it = max(it, __shfl_xor_sync(0xffffffffu, it, o));
  }
  if (threadIdx.x == 0) {
    iters[b] = it;
    relres[b] = !isfinite(b2) ? (double)NAN : b2 > 0.0 ? sqrt(r2 / b2) : 0.0;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

}  // namespace

bool gram_supported(int ny, int nx) {
  if (ny < 32 || ny % 16 != 0 || ny > 1024 || nx < 1) return false;
  return gram_tile(ny) > 0;
}

int gram_tile(int ny) {
  if (ny % 16) return 0;
  if (ny <= 256) return ny;
  for (int t = 256; t >= 16; t -= 16)
    if (ny % t == 0) return t;
  return 0;
}

size_t gram_bytes(int ny, int nx) { return (size_t)2 * nx * 2 * ny * ny * sizeof(float); }

int gram_pa(int ny, int nx) { return nx * (ny / gram_tile(ny)); }

bool gram_encode_x(CUtensorMap* m, float* base, int ny, int nx, int B, int kc) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[4] = {(cuuint64_t)ny, 2, (cuuint64_t)nx, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)ny * 4, (cuuint64_t)2 * ny * 4, (cuuint64_t)2 * ny * nx * 4};
  cuuint32_t box[4] = {(cuuint32_t)kc, 1, 1, kGramRows}, es[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             kc == 16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_plane_map(CUtensorMap* m, const void* base, int rows, int L, int64_t planes, int cols, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15) || (L * 8) % 16 || (cols * 8) % 16 || cols > 256 ||
      box_rows > 256 || box_rows < 1)
    return false;
  cuuint64_t dims[3] = {(cuuint64_t)L, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)L * 8, (cuuint64_t)rows * L * 8};
  cuuint32_t box[3] = {(cuuint32_t)cols, (cuuint32_t)box_rows, 1}, es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool gram_encode_e(CUtensorMap* m, float* base, int ny, int nx, int B) {
  EncodeTiledFn enc = encode_fn();
  if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  cuuint64_t dims[4] = {(cuuint64_t)ny, 2, (cuuint64_t)nx, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)ny * 4, (cuuint64_t)2 * ny * 4, (cuuint64_t)2 * ny * nx * 4};
  cuuint32_t box[4] = {32, 1, 1, kGramRows}, es[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void launch_gram_build(const float2* smaps, const uint8_t* mask_host, int nc, const GramOp& op, double2* pbuf,
                       cudaStream_t s) {
  const int ny = op.ny, nx = op.nx;
  // P[d] = (1/ny) sum_k m_k exp(2 pi i k d / ny), in FP64 on the host
  std::vector<double2> P(ny), tw(ny);
  const double pi2 = 6.283185307179586476925286766559;
  for (int e = 0; e < ny; ++e) tw[e] = make_double2(std::cos(pi2 * e / ny), std::sin(pi2 * e / ny));
  for (int d = 0; d < ny; ++d) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k < ny; ++k)
      if (mask_host[k]) {
        const double2 w = tw[(int)(((int64_t)k * d) % ny)];
        re += w.x;
        im += w.y;
      }
    P[d] = make_double2(re / ny, im / ny);
  }
  cudaMemcpyAsync(pbuf, P.data(), ny * sizeof(double2), cudaMemcpyHostToDevice, s);
  const size_t sbytes = (size_t)nc * ny * sizeof(float2);
  if (op.f16) {
    // the FP16 form needs the column's sensitivities in shared memory (its scale bound)
    cudaFuncSetAttribute(k_gram_build_smem<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sbytes);
    k_gram_build_smem<true><<<dim3(nx, (ny + 31) / 32), 256, sbytes, s>>>(smaps, pbuf, nc, ny, nx, op.nt, 16,
                                                                           op.G, op.gscale);
  } else if (sbytes <= 200 * 1024) {
    cudaFuncSetAttribute(k_gram_build_smem<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sbytes);
    k_gram_build_smem<false><<<dim3(nx, (ny + 31) / 32), 256, sbytes, s>>>(smaps, pbuf, nc, ny, nx, op.nt,
                                                                            op.kc, op.G, op.gscale);
  } else {
    const int64_t tot = (int64_t)ny * ny;
    k_gram_build<<<dim3((unsigned)((tot + 255) / 256), nx), 256, 0, s>>>(smaps, pbuf, nc, ny, nx, op.nt, op.kc,
                                                                          static_cast<float*>(op.G));
  }
  cudaStreamSynchronize(s);  // P lives on the host stack until the copy has run
}

void launch_gram_scalars(const CgArgs& a, int nb, int it, float* beta, int* done, double* pn, float* pscale,
                         cudaStream_t s) {
  k_gram_scalars<<<nb, 32, 0, s>>>(a, it, beta, done, pn, pscale);
}

void launch_gram_apply_scale(const float* x, int ny, int nx, int nb, float* pscale, cudaStream_t s) {
  if (nb > 0) k_gram_apply_scale<<<nb, 256, 0, s>>>(x, (int64_t)2 * ny * nx, pscale);
}

size_t gram_smem(int ny, int kc, bool f16, int* stages) {
  const int nt = gram_tile(ny);
  const size_t stage = f16 ? 4 * (size_t)kGramRows * 16 * 4 + 4 * (size_t)kGramRows * 32 + 4 * (size_t)nt * 32
                           : 4 * (size_t)kGramRows * kc * 4 + 4 * (size_t)nt * kc * 4;
  int S = (int)((220 * 1024 - 2560) / stage);
  if (S > 8) S = 8;
  if (S < 2) S = 2;
  *stages = S;
  // barriers, TMEM slot, per-row beta and FP16 scale, per-column CG exchange slots (two FP64 sums per row)
  return 1024 + (size_t)S * stage + (3 * (size_t)S + 9) * 8 + 16 + 2 * kGramRows * 4 + 2 * kGramRows * 8 + 64;
}

void launch_gram_normal(const GramOp& op, const CUtensorMap& mIn, const CUtensorMap& mPold, GramArgs g,
                        cudaStream_t s) {
  const bool f16 = op.f16 && op.kc == 16 && !op.a_tmem;
  int S = 0;
  const size_t smem = gram_smem(op.ny, op.kc, f16, &S);
  // the split direction goes to tensor memory when it fits beside the accumulators
  const bool at = !f16 && op.a_tmem && 2 * op.nt + 4 * op.kc * S <= 512;
  void (*kern)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap,
               GramArgs, ColCgArgs) =
      f16 ? k_gram_normal<16, false, false, true>
          : op.kc == 16 ? (at ? k_gram_normal<16, true, false, false> : k_gram_normal<16, false, false, false>)
                        : (at ? k_gram_normal<8, true, false, false> : k_gram_normal<8, false, false, false>);
  // the shared-memory opt-in is per device and kernel; cache it per (thread, device)
  constexpr int kMaxDev = 16;
  static thread_local size_t configured[kMaxDev][5] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const int ki = f16 ? 4 : (op.kc == 16 ? 0 : 2) + (at ? 1 : 0);
  if (dev < 0 || dev >= kMaxDev || configured[dev][ki] < smem) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (dev >= 0 && dev < kMaxDev) configured[dev][ki] = smem;
  }
  g.ny = op.ny;
  g.nx = op.nx;
  g.nt = op.nt;
  g.nyt = op.ny / op.nt;
  g.stages = S;
  g.G = op.G;
  g.gscale = op.gscale;
  g.tmem_cols = 32;
  const int need = at ? 2 * op.nt + 4 * op.kc * S : 2 * op.nt;
  while (g.tmem_cols < need) g.tmem_cols *= 2;
  const unsigned itiles = (unsigned)((g.nb + kGramRows - 1) / kGramRows);
  const dim3 grid((unsigned)g.nyt * itiles, op.nx);
  // epilogue maps over exactly the nb images of this launch (128-byte swizzle,
  // 32-value boxes of 128 images)
  CUtensorMap mPe{}, mQe{};
  const float* psrc = g.cg ? g.pnew : g.in;
  g.tma_epi = op.nt % 32 == 0 && g.nb > 0 && gram_encode_e(&mPe, const_cast<float*>(psrc), op.ny, op.nx, g.nb) &&
              gram_encode_e(&mQe, g.q, op.ny, op.nx, g.nb);
  kern<<<grid, kGramThreads, smem, s>>>(mIn, mPold, mPe, mQe, mQe, g, ColCgArgs{});
}

bool gram_colcg_supported(int ny, int nx) {
  if (!gram_supported(ny, nx)) return false;
  const int nt = gram_tile(ny);
  return nt % 32 == 0 && ny / nt <= 4;
}

bool launch_gram_colcg(const GramOp& op, const CUtensorMap& mIn, const CUtensorMap& mPold, GramArgs g,
                       const ColCgArgs& cc, cudaStream_t s) {
  const bool f16 = op.f16 && op.kc == 16;
  int S = 0;
  const size_t smem = gram_smem(op.ny, op.kc, f16, &S);
  void (*kern)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap,
               GramArgs, ColCgArgs) = f16 ? k_gram_normal<16, false, true, true>
                                          : op.kc == 16 ? k_gram_normal<16, false, true, false>
                                                        : k_gram_normal<8, false, true, false>;
  constexpr int kMaxDev = 16;
  static thread_local size_t configured[kMaxDev][3] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const int ki = f16 ? 2 : op.kc == 16 ? 0 : 1;
  if (dev < 0 || dev >= kMaxDev || configured[dev][ki] < smem) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (dev >= 0 && dev < kMaxDev) configured[dev][ki] = smem;
  }
  g.ny = op.ny;
  g.nx = op.nx;
  g.nt = op.nt;
  g.nyt = op.ny / op.nt;
  g.stages = S;
  g.G = op.G;
  g.gscale = op.gscale;
  g.cg = 1;
  g.tma_epi = 1;
  g.tmem_cols = 32;
  while (g.tmem_cols < 2 * op.nt) g.tmem_cols *= 2;
  if (g.nb <= 0) return true;
  // tile maps over exactly the nb images of this launch: p (written by the
  // main loop's split warps), x and r (read and written by the epilogue)
  CUtensorMap mPe{}, mXe{}, mRe{};
  if (!gram_encode_e(&mPe, g.pnew, op.ny, op.nx, g.nb) || !gram_encode_e(&mXe, cc.x, op.ny, op.nx, g.nb) ||
      !gram_encode_e(&mRe, cc.r, op.ny, op.nx, g.nb))
    return false;  // nothing launched
  const unsigned itiles = (unsigned)((g.nb + kGramRows - 1) / kGramRows);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)g.nyt * itiles, op.nx);
  cfg.blockDim = dim3(kGramThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)g.nyt;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, mIn, mPold, mPe, mXe, mRe, g, cc) == cudaSuccess;
}

void launch_colcg_init(const ColCgArgs& cg, int ny, int nx, int nb, cudaStream_t s) {
  if (nb > 0) k_colcg_init<<<dim3(nx, nb), 64, 0, s>>>(cg, ny, nx);
}
void launch_colcg_any_live(const ColCgArgs& cg, int nx, int nb, int* flag, cudaStream_t s) {
  const int n = nx * nb;
  cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (n > 0) k_colcg_any_live<<<(n + 255) / 256, 256, 0, s>>>(cg, n, flag);
}
void launch_colcg_report(const ColCgArgs& cg, int nx, int nb, int* iters, double* relres, cudaStream_t s) {
  if (nb > 0) k_colcg_report<<<nb, 32, 0, s>>>(cg, nx, iters, relres);
}

void launch_to_cp(const float2* in, float* out, int ny, int nx, int nb, cudaStream_t s) {
  k_to_cp<<<dim3((nx + 31) / 32, (ny + 31) / 32, nb), dim3(32, 8), 0, s>>>(in, out, ny, nx);
}
void launch_from_cp(const float* in, float2* out, int ny, int nx, int nb, cudaStream_t s) {
  k_from_cp<<<dim3((nx + 31) / 32, (ny + 31) / 32, nb), dim3(32, 8), 0, s>>>(in, out, ny, nx);
}

}  // namespace pico
