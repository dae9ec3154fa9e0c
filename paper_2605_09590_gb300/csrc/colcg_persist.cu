// Per-column CG with the whole solve in one launch, for Cartesian phase-encode
// images with a tensor-core Gram operator (ny = CS * NT rows, CS <= 8).
//
// With a phase-encode mask A^H A is block diagonal over the readout columns
// (Sec. 2.1.3 with M = M_y (x) I), so CG on Eq. 6 splits into independent
// column systems (G_j + lam I) x_j = b_j, each converging on its own (the
// stopping rule ||r_j|| <= rtol ||b_j|| per column).  A cluster of CS CTAs
// owns one column j and a tile of 128 images for every iteration of the
// solve; CTA `rank` holds rows [rank NT, rank NT + NT) of x, r and p:
//   x, p (FP32) and the accumulator D in tensor memory (one image per lane),
//   r (FP32) in shared memory,
// so the CG vectors never leave the chip between iterations.  Per iteration:
//   main loop   D = sum_k p[k] G_j[rows, k] on tcgen05 (kind::f16, FP16 head
//               + remainder of p and G after power-of-two scaling, 12 MMAs of
//               M 128 x N NT x K 16 per 16-row chunk).  The A operand (the
//               split direction of all ny rows) comes from a global buffer in
//               which every CTA of the cluster leaves its own rows' chunks
//               (L2-resident), the B operand from the stage-tiled G_j;
//   phase A     q = D / (gscale ps) + lam p, the p^H q partial of the CTA's rows;
//   exchange 1  p^H q over the column (distributed shared memory, rank order);
//   phase B     x += alpha p, r -= alpha q, the ||r||^2 partial;
//   exchange 2  ||r||^2 over the column, beta, the stopping rule;
//   phase C     p = r + beta p, its FP16 split written for the next main loop.
// Every CTA of a cluster adds the partials in rank order, so all of them take
// the same alpha, beta and stopping decisions (and leave the loop together).
// Inner products: FP32 partial sums of 16 rows (as in the one-update kernel),
// float-float across chunks and CTAs; values scaled by the direction's
// power-of-two FP16 scale, so no FP32 underflow.  Every mbarrier wait is
// bounded (about 2 s, then an error code); an error ends the solve on every
// CTA of the cluster at the same iteration (flags exchanged after the last
// cluster barrier of each iteration).
#include <cuda_fp16.h>

#include "common.cuh"
#include "f16_split.cuh"
#include "kernels.cuh"
#include "tc_util.cuh"

namespace pico {

namespace {

using namespace tc;

constexpr int kPM = 128;                    // images per cluster (MMA M, one per tensor-memory lane)
constexpr int kPThreads = 320;              // warp 0 loads, warp 1 MMA, warps 2-9 epilogue (two halves)
constexpr uint32_t kPlaneA = kPM * 32;      // one FP16 plane of a 16-row chunk: 4 KB
constexpr uint32_t kChunkA = 4 * kPlaneA;   // [re head | im head | re rem | im rem]: 16 KB

struct PersistArgs {
  const void* G;         // FP16 stage-tiled G_j for row blocks of NT
  const float* gscale;   // [nx] power-of-two scale of G_j
  const float* R;        // right-hand sides, column-planar [B][nx][2][ny]
  float* X;              // solutions, same layout
  uint8_t* psplit;       // [nx][tiles][ny / 16] chunks of kChunkA bytes
  double* rr0;           // [B][nx] ||b_j||^2
  double* rr;            // [B][nx] final ||r_j||^2
  int* iters;            // [B][nx] updates taken
  int* status;           // [B] 5 on breakdown
  int* err;              // first failure code of a bounded wait
  int ny, nx, nb, tiles, max_iter, stages;
  double rtol2;
  float lam;
};

// descriptor of a K-major FP16 tile with 32-byte rows (16 values), 8-row
// atoms, 32-byte swizzle
__device__ __forceinline__ uint64_t desc32(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)((8u * 32u) >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)6u << 61;
  return d;
}

__device__ __forceinline__ void set_err(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// float-float value at the same shared-memory offset in the CTA of cluster rank `rank`
__device__ __forceinline__ ffloat ld_dsmem_ff(const ffloat* local, uint32_t rank) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(local)), "r"(rank));
  float h, l;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(h), "=f"(l) : "r"(ra) : "memory");
  return ffloat{h, l};
}
__device__ __forceinline__ int ld_dsmem_i32(const int* local, uint32_t rank) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(local)), "r"(rank));
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
  return v;
}

// float-float sum at a power-of-two scale 2^e, as a double
__device__ __forceinline__ double ff_unscale(ffloat a, int e) {
  return ldexp((double)a.hi + (double)a.lo, -e);
}
__device__ __forceinline__ int exp2_of(float pow2) { return (int)((__float_as_uint(pow2) >> 23) & 0xff) - 127; }
// a / b to about float precision (b.hi > 0)
__device__ __forceinline__ float ff_div(ffloat a, ffloat b) {
  const float q1 = a.hi / b.hi;
  const float rem = fmaf(-q1, b.hi, a.hi) + a.lo - q1 * b.lo;
  return q1 + rem / b.hi;
}
__device__ __forceinline__ ffloat ff_scale(ffloat a, float pow2) { return ffloat{a.hi * pow2, a.lo * pow2}; }

// the FP16 split of 8 values (one plane pair) of image row i into logical
// 16-byte group g of a chunk: 32-byte rows, the two groups swapped on rows
// 4..7 of every 8-row atom (32-byte swizzle)
__device__ __forceinline__ void store_split8(uint8_t* chunk, int plane_hi, int plane_lo, int i, int g, const float* v,
                                             float sc) {
  uint2 h0, l0, h1, l1;
  split_f16x4(v[0] * sc, v[1] * sc, v[2] * sc, v[3] * sc, h0, l0);
  split_f16x4(v[4] * sc, v[5] * sc, v[6] * sc, v[7] * sc, h1, l1);
  const size_t off = (size_t)i * 32 + (size_t)((g ^ ((i >> 2) & 1)) * 16);
  *reinterpret_cast<uint4*>(chunk + (size_t)plane_hi * kPlaneA + off) = make_uint4(h0.x, h0.y, h1.x, h1.y);
  *reinterpret_cast<uint4*>(chunk + (size_t)plane_lo * kPlaneA + off) = make_uint4(l0.x, l0.y, l1.x, l1.y);
}

template <int NT>
__global__ void __launch_bounds__(kPThreads, 1) k_colcg_persist(PersistArgs a) {
  static_assert(NT % 16 == 0 && 6 * NT <= 512, "row block");
  constexpr int NO = NT / 8;                 // 8-row octets of this CTA; epilogue half h takes o = h, h + 2, ...
  constexpr int NCH = NT / 16;               // 16-row chunks of this CTA (its own main-loop stages)
  constexpr uint32_t kB = NT * 128;          // B block: 4 FP16 planes of NT x 16
  constexpr uint32_t kStage = kChunkA + kB;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  const int S = a.stages;
  float* r_re = reinterpret_cast<float*>(sm + (size_t)S * kStage);  // [NT][128]
  float* r_im = r_re + NT * kPM;
  ffloat* xpq = reinterpret_cast<ffloat*>(r_im + NT * kPM);  // [2 halves][128] exchange slots
  ffloat* xrr = xpq + 2 * kPM;
  int* xab = reinterpret_cast<int*>(xrr + 2 * kPM);  // [0] sticky error flag, [1..2] any-live by iteration parity
  uint64_t* full = reinterpret_cast<uint64_t*>(xab + 4);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accf + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const int CS = a.ny / NT;
  const int tile = blockIdx.x / CS, j = blockIdx.y;
  const int n0 = (int)rank * NT, m0 = tile * kPM;
  const int nkc = a.ny / 16, kc0 = n0 / 16;
  const uint8_t* gsrc = static_cast<const uint8_t*>(a.G) + ((size_t)j * CS + rank) * nkc * kB;
  uint8_t* pcol = a.psplit + ((size_t)j * a.tiles + tile) * nkc * kChunkA;  // this (column, tile)'s chunks

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    fence_mbar_init();
    xab[0] = 0;
    xab[1] = 0;
    xab[2] = 0;
  }
  if (warp == 1) tmem_alloc(tslot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  // epilogue thread state: image i of the tile (tensor-memory lane i), rows of
  // the octets of half h
  const bool epi = warp >= 2;
  const int h = (warp - 2) >> 2;
  const int quarter = warp & 3, i = 32 * quarter + lane, img = m0 + i;
  const bool valid = epi && img < a.nb;
  const uint32_t tl = tbase + ((uint32_t)(32 * quarter) << 16);
  const uint32_t tD = tl, tX = tl + 2 * NT, tP = tl + 4 * NT;  // re at +0, im at +NT
  const float gsi = epi ? 1.f / a.gscale[j] : 1.f;
  const float lam = a.lam;
  double rr0 = 0.0, rrd = 0.0;
  ffloat rrs{0.f, 0.f};  // ||r||^2 scaled by ps^2
  double pn = 0.0;  // bound on the direction's entries, sqrt(rr) + beta pn (FP64: rr falls far below FP32's range)
  float ps = 1.f;
  bool live = false, broke = false;
  int iters = 0;
  // sum of the 2 CS partials of image i in (rank, half) order: the same bits on every CTA and half
  auto gather = [&](const ffloat* slots) {
    ffloat t{0.f, 0.f};
    for (int rk = 0; rk < CS; ++rk) {
      t = ff_add(t, ld_dsmem_ff(&slots[i], (uint32_t)rk));
      t = ff_add(t, ld_dsmem_ff(&slots[kPM + i], (uint32_t)rk));
    }
    return t;
  };

  // Main-loop stage t of update `it` takes chunk (kc0 + t) mod ny/16: this
  // CTA's own chunks come first, so that they can be loaded and multiplied
  // while the cluster barrier that publishes the peers' chunks completes.
  int issued = 0;     // stages issued by the producer (all updates)
  int committed = 0;  // accumulator commits by the MMA thread
  auto produce = [&](int it, int t0, int t1) -> bool {  // producer thread: stages t0 .. t1 - 1
    for (int t = t0; t < t1; ++t) {
      const int gidx = it * nkc + t, s = gidx % S, kc = (kc0 + t) % nkc;
      if (gidx >= S && !mbar_wait(&empty[s], ((gidx / S) - 1) & 1)) {
        set_err(a.err, 21);
        return false;
      }
      uint8_t* st = sm + (size_t)s * kStage;
      mbar_expect_tx(&full[s], kStage);
      bulk_load(st, pcol + (size_t)kc * kChunkA, kChunkA, &full[s]);
      bulk_load(st + kChunkA, gsrc + (size_t)kc * kB, kB, &full[s]);
      issued = gidx + 1;
    }
    return true;
  };
  auto consume = [&](int it, int t0, int t1) -> bool {  // MMA thread: stages t0 .. t1 - 1
    const uint32_t hd = idesc_f16(kPM, NT, false), hdn = idesc_f16(kPM, NT, true);
    const uint32_t dre = tbase, dim = tbase + NT;
    for (int t = t0; t < t1; ++t) {
      const int gidx = it * nkc + t, s = gidx % S;
      if (!mbar_wait(&full[s], (gidx / S) & 1)) {
        set_err(a.err, 22);
        return false;
      }
      tc_fence_after();
      const uint32_t sa = smem_u32(sm + (size_t)s * kStage), sbb = sa + kChunkA;
      const uint32_t acc0 = t == 0 ? 0u : 1u;
      const uint64_t Ahr = desc32(sa), Ahi = desc32(sa + kPlaneA);
      const uint64_t Alr = desc32(sa + 2 * kPlaneA), Ali = desc32(sa + 3 * kPlaneA);
      const uint64_t Bhr = desc32(sbb), Bhi = desc32(sbb + NT * 32);
      const uint64_t Blr = desc32(sbb + 2 * NT * 32), Bli = desc32(sbb + 3 * NT * 32);
      // D_re += p_re G_re^T - p_im G_im^T ; D_im += p_re G_im^T + p_im G_re^T
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
    }
    return true;
  };
  // after this CTA's split of update `it` is complete (block barrier), between
  // the arrive and the wait of the cluster barrier: the own stages of `it`.
  // A failure here is published before the next exchange, so that every CTA
  // of the cluster reads the same error flags after the same barrier.
  bool late_err = false;
  auto early = [&](int it) {
    if (it >= a.max_iter) return;
    if (warp == 0 && lane == 0) late_err = !produce(it, 0, NCH);
    else if (warp == 1 && lane == 0) late_err = !consume(it, 0, NCH);
  };

  // ---- start: r = b, x = 0, p = r; ||b_j||^2; the split of p for the first main loop ----
  if (epi) {
    const float* bre = a.R + ((size_t)(valid ? img : 0) * a.nx + j) * 2 * a.ny + n0;
    const float* bim = bre + a.ny;
    float mx = 0.f;
    const float zero[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int o = h; o < NO; o += 2) {
      float vr[8], vi[8];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float4 w = valid ? reinterpret_cast<const float4*>(bre + 8 * o)[u] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 z = valid ? reinterpret_cast<const float4*>(bim + 8 * o)[u] : make_float4(0.f, 0.f, 0.f, 0.f);
        vr[4 * u] = w.x; vr[4 * u + 1] = w.y; vr[4 * u + 2] = w.z; vr[4 * u + 3] = w.w;
        vi[4 * u] = z.x; vi[4 * u + 1] = z.y; vi[4 * u + 2] = z.z; vi[4 * u + 3] = z.w;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        r_re[(8 * o + u) * kPM + i] = vr[u];
        r_im[(8 * o + u) * kPM + i] = vi[u];
        mx = fmaxf(mx, fmaxf(fabsf(vr[u]), fabsf(vi[u])));
      }
      tmem_st8(tP + 8 * o, vr);
      tmem_st8(tP + NT + 8 * o, vi);
      tmem_st8(tX + 8 * o, zero);
      tmem_st8(tX + NT + 8 * o, zero);
    }
    tmem_wait_st();
    // this half's ||b||^2 over its rows, scaled by its largest entry (float-float)
    const float sb = pow2_scale_f(mx);
    ffloat acc{0.f, 0.f};
    for (int o = h; o < NO; o += 2) {
      float f = 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float br = r_re[(8 * o + u) * kPM + i] * sb, bi = r_im[(8 * o + u) * kPM + i] * sb;
        f = fmaf(br, br, fmaf(bi, bi, f));
      }
      acc = ff_add(acc, ffloat{f, 0.f});
    }
    reinterpret_cast<double*>(xrr)[h * kPM + i] = ff_unscale(acc, 2 * exp2_of(sb));
  }
  cluster_sync_all();
  if (epi) {
    for (int rk = 0; rk < CS; ++rk)
      for (int hh = 0; hh < 2; ++hh) {
        uint32_t ra;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                     : "=r"(ra)
                     : "r"(smem_u32(reinterpret_cast<double*>(xrr) + hh * kPM + i)), "r"((uint32_t)rk));
        double v;
        asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
        rr0 += v;
      }
    rrd = rr0;
    const bool bad = !isfinite(rr0);
    live = valid && !bad && rr0 > 0.0;
    if (valid && bad) broke = true;
    pn = sqrt(rr0);
    ps = pow2_scale(pn);
    {
      const double v = rr0 * (double)ps * (double)ps;
      const float hi = (float)v;
      rrs = ffloat{hi, (float)(v - (double)hi)};
    }
    // the split of p = b for this half's octets
    for (int o = h; o < NO; o += 2) {
      float vr[8], vi[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        vr[u] = r_re[(8 * o + u) * kPM + i];
        vi[u] = r_im[(8 * o + u) * kPM + i];
      }
      uint8_t* ch = pcol + (size_t)(kc0 + (o >> 1)) * kChunkA;
      store_split8(ch, 0, 2, i, o & 1, vr, ps);
      store_split8(ch, 1, 3, i, o & 1, vi, ps);
    }
    fence_proxy_async_global();  // generic writes of the split, read by the bulk copies
    if (live) xab[1] = 1;  // any live system in this tile (benign race: every writer stores 1)
  }
  tc_fence_before();
  __syncthreads();           // this CTA's split of the first direction is complete
  cluster_arrive_release();  // ... and published to the peers
  early(0);
  cluster_wait_acquire();
  tc_fence_after();
  bool any_live = xab[1] != 0;
  bool abort = false;
  if (threadIdx.x == 0) xab[2] = 0;

  for (int it = 0; it < a.max_iter && any_live && !abort; ++it) {
    // ---- main loop: the peers' chunks (the own ones are in flight since the last barrier) ----
    if (warp == 0 && lane == 0) {
      if (late_err) xab[0] = 1;
      fence_proxy_async_global();
      if (!produce(it, NCH, nkc)) xab[0] = 1;
    } else if (warp == 1 && lane == 0) {
      if (late_err) xab[0] = 1;
      if (!consume(it, NCH, nkc)) xab[0] = 1;
      mma_commit(accf);
      ++committed;
    }
    // ---- phase A: q = D / (gscale ps) + lam p; p^H q (scaled by ps^2) ----
    const float fsc = gsi / ps;
    if (epi) {
      // one thread waits for the accumulator; the other epilogue warps sleep in a
      // named barrier instead of polling, which would take issue slots from the
      // MMA warp on the same scheduler
      if (threadIdx.x == 64 && !mbar_wait(accf, it & 1)) {
        set_err(a.err, 23);
        xab[0] = 1;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(kPThreads - 64) : "memory");
      tc_fence_after();
      ffloat pq{0.f, 0.f};
#pragma unroll 1
      for (int o = h; o < NO; o += 2) {
        float dr[8], di[8], pr[8], pi[8];
        tmem_ld8x4(tD + 8 * o, tD + NT + 8 * o, tP + 8 * o, tP + NT + 8 * o, dr, di, pr, pi);
        float f = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float qr = fmaf(lam, pr[u], dr[u] * fsc), qi = fmaf(lam, pi[u], di[u] * fsc);
          f = fmaf(pr[u] * ps, qr * ps, fmaf(pi[u] * ps, qi * ps, f));
        }
        pq = ff_add(pq, ffloat{f, 0.f});
      }
      xpq[h * kPM + i] = pq;
    }
    tc_fence_before();
    cluster_sync_all();  // exchange 1
    tc_fence_after();
    float alpha = 0.f;
    bool upd = false;
    if (epi) {
      const ffloat pqt = gather(xpq);
      if (live) {
        if (!(pqt.hi > 0.f) || !isfinite(pqt.hi)) {
          live = false;
          broke = true;
        } else {
          alpha = ff_div(rrs, pqt);
          upd = true;
        }
      }
      // ---- phase B: x += alpha p, r -= alpha q; ||r||^2 (scaled by ps^2) ----
      // tensor-memory loads and stores are warp-collective: every lane takes
      // part whenever one lane of its warp updates (the others store back
      // what they loaded)
      ffloat rn{0.f, 0.f};
      if (__any_sync(0xffffffffu, upd)) {
#pragma unroll 1
        for (int o = h; o < NO; o += 2) {
          float f = 0.f;
          float dr[8], di[8], pr[8], pi[8], xr[8], xi[8];
          tmem_ld8x6(tD + 8 * o, tD + NT + 8 * o, tP + 8 * o, tP + NT + 8 * o, tX + 8 * o, tX + NT + 8 * o, dr, di,
                     pr, pi, xr, xi);
          if (upd) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const float qr = fmaf(lam, pr[u], dr[u] * fsc), qi = fmaf(lam, pi[u], di[u] * fsc);
              xr[u] = fmaf(alpha, pr[u], xr[u]);
              xi[u] = fmaf(alpha, pi[u], xi[u]);
              float* rre = &r_re[(8 * o + u) * kPM + i];
              float* rim = &r_im[(8 * o + u) * kPM + i];
              const float nr = fmaf(-alpha, qr, *rre), ni = fmaf(-alpha, qi, *rim);
              *rre = nr;
              *rim = ni;
              f = fmaf(nr * ps, nr * ps, fmaf(ni * ps, ni * ps, f));
            }
          }
          tmem_st8(tX + 8 * o, xr);
          tmem_st8(tX + NT + 8 * o, xi);
          rn = ff_add(rn, ffloat{f, 0.f});
        }
        tmem_wait_st();
      }
      xrr[h * kPM + i] = rn;
    }
    tc_fence_before();
    cluster_sync_all();  // exchange 2
    tc_fence_after();
    if (epi) {
      const ffloat rnt = gather(xrr);
      float beta = 0.f;
      bool cont = false;
      if (upd) {
        const double rn_d = ff_unscale(rnt, 2 * exp2_of(ps));
        if (!isfinite(rn_d)) {
          live = false;
          broke = true;
        } else {
          ++iters;
          rrd = rn_d;
          const bool stop = !(rn_d > a.rtol2 * rr0);
          if (stop) {
            live = false;
          } else {
            beta = ff_div(rnt, rrs);
            cont = true;
          }
          rrs = rnt;
        }
      }
      // ---- phase C: p = r + beta p and its split (scale from sqrt(rr) + beta pn) ----
      if (cont) {
        pn = sqrt(rrd) + (double)beta * pn;
        const float psn = pow2_scale(pn);
        rrs = ff_scale(rrs, (psn / ps) * (psn / ps));  // exact: powers of two
        ps = psn;
      }
      if (__any_sync(0xffffffffu, cont)) {  // warp-collective, as in phase B
#pragma unroll 1
        for (int o = h; o < NO; o += 2) {
          float pr[8], pi[8];
          tmem_ld8x2(tP + 8 * o, tP + NT + 8 * o, pr, pi);
          if (cont) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              pr[u] = fmaf(beta, pr[u], r_re[(8 * o + u) * kPM + i]);
              pi[u] = fmaf(beta, pi[u], r_im[(8 * o + u) * kPM + i]);
            }
          }
          tmem_st8(tP + 8 * o, pr);
          tmem_st8(tP + NT + 8 * o, pi);
          if (cont) {
            uint8_t* ch = pcol + (size_t)(kc0 + (o >> 1)) * kChunkA;
            store_split8(ch, 0, 2, i, o & 1, pr, ps);
            store_split8(ch, 1, 3, i, o & 1, pi, ps);
          }
        }
        tmem_wait_st();
        fence_proxy_async_global();
        if (cont) xab[1 + ((it + 1) & 1)] = 1;
      }
    }
    tc_fence_before();
    __syncthreads();           // this CTA's split is complete and the accumulator read for the last time
    cluster_arrive_release();  // the split is published; flags are final
    early(it + 1);             // the own stages of the next update (discarded if the solve ends here)
    cluster_wait_acquire();
    tc_fence_after();
    any_live = xab[1 + ((it + 1) & 1)] != 0;
    bool ab = false;
    for (int rk = 0; rk < CS; ++rk) ab = ab || ld_dsmem_i32(&xab[0], (uint32_t)rk) != 0;
    abort = ab;
    // the other parity's flag is next written in iteration it + 1, after exchange 2
    if (threadIdx.x == 0) xab[1 + (it & 1)] = 0;
  }

  // ---- results: x to global, the column's scalars (rank 0, half 0) ----
  if (epi) {  // every epilogue lane loads (warp-collective); valid lanes store
    float* xre = a.X + ((size_t)(valid ? img : 0) * a.nx + j) * 2 * a.ny + n0;
    float* xim = xre + a.ny;
    for (int o = h; o < NO; o += 2) {
      float xr[8], xi[8];
      tmem_ld8x2(tX + 8 * o, tX + NT + 8 * o, xr, xi);
      if (valid) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          reinterpret_cast<float4*>(xre + 8 * o)[u] = make_float4(xr[4 * u], xr[4 * u + 1], xr[4 * u + 2], xr[4 * u + 3]);
          reinterpret_cast<float4*>(xim + 8 * o)[u] = make_float4(xi[4 * u], xi[4 * u + 1], xi[4 * u + 2], xi[4 * u + 3]);
        }
      }
    }
  }
  if (valid && rank == 0 && h == 0) {
    const size_t cidx = (size_t)img * a.nx + j;
    a.rr0[cidx] = rr0;
    a.rr[cidx] = rrd;
    a.iters[cidx] = iters;
    if (broke) a.status[img] = 5;
  }
  // teardown: no bulk copy or MMA of this CTA in flight, no peer still reading
  // this CTA's shared memory, then the tensor memory is freed
  if (warp == 0 && lane == 0) {
    for (int g = issued - S < 0 ? 0 : issued - S; g < issued; ++g)
      if (!mbar_wait(&full[g % S], (g / S) & 1)) set_err(a.err, 24);
  }
  if (warp == 1 && lane == 0) {  // also covers MMAs of an update that did not run (its own stages)
    mma_commit(accf);
    ++committed;
    if (!mbar_wait(accf, (committed - 1) & 1)) set_err(a.err, 25);
  }
  tc_fence_before();
  cluster_sync_all();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

template <int NT>
size_t persist_smem(int* stages) {
  const size_t stage = kChunkA + (size_t)NT * 128;
  const size_t fixed = 1024 + (size_t)2 * NT * kPM * 4 + 4 * kPM * 8 + 16 + 64;
  int S = (int)((225 * 1024 - fixed) / (stage + 16));
  if (S > 6) S = 6;
  *stages = S;
  return fixed + (size_t)S * (stage + 16);
}

template <int NT>
bool launch_nt(const PersistArgs& a0, cudaStream_t s) {
  PersistArgs a = a0;
  int S = 0;
  const size_t smem = persist_smem<NT>(&S);
  if (S < 2) return false;
  a.stages = S;
  auto kern = k_colcg_persist<NT>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return false;
  const int CS = a.ny / NT;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(CS * a.tiles), (unsigned)a.nx);
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a) == cudaSuccess;
}

}  // namespace

int colcg_persist_rows(int ny) {
  if (ny % 16 != 0) return 0;
  for (int nt : {80, 64, 48, 32})
    if (ny % nt == 0 && ny / nt >= 2 && ny / nt <= 8) return nt;
  return 0;
}

size_t colcg_persist_split_bytes(int ny, int nx, int B) {
  return (size_t)nx * ((B + kPM - 1) / kPM) * (ny / 16) * kChunkA;
}

bool launch_colcg_persist(const void* G, const float* gscale, const float* R, float* X, uint8_t* psplit, double* rr0,
                          double* rr, int* iters, int* status, int* err, int ny, int nx, int nb, int max_iter,
                          double rtol2, float lam, cudaStream_t s) {
  if (nb <= 0) return true;
  const int nt = colcg_persist_rows(ny);
  PersistArgs a{G, gscale, R, X, psplit, rr0, rr, iters, status, err, ny, nx, nb, (nb + kPM - 1) / kPM,
                max_iter, 0, rtol2, lam};
  switch (nt) {
    case 80: return launch_nt<80>(a, s);
    case 64: return launch_nt<64>(a, s);
    case 48: return launch_nt<48>(a, s);
    case 32: return launch_nt<32>(a, s);
    default: return false;
  }
}

}  // namespace pico
