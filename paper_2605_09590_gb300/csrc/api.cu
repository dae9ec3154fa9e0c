// C-ABI layer of libpico: context management, operator set-up and the
// stream-ordered drivers of the PICO / PMR / CG hot path.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <map>
#include <set>
#include <tuple>
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "pico.h"
#include "common.cuh"
#include "kernels.cuh"

using cd = std::complex<double>;

struct pico_ctx {
  int kind = 0, ny = 0, nx = 0, nc = 0;
  int64_t n = 0;
  cudaStream_t stream = nullptr;
  double lam_rel = 0, lam_phys = 0, lambda_max = 0, margin = 1.01;
  int power_iters = 0, max_batch = 64, itmax = 128;
  // device operator
  float2* smaps = nullptr;
  float* ymul = nullptr;
  float2* tw = nullptr;
  float2* twx = nullptr;
  uint8_t* mask = nullptr;
  // workspace
  float2 *X = nullptr, *R = nullptr, *P = nullptr, *Q = nullptr;
  double *rr_part = nullptr, *pq_part = nullptr;
  int* status = nullptr;
  int* d_iters = nullptr;
  int* cg_done = nullptr;     // [B] per-system stop flag of the current iteration (Toeplitz passes)
  int* d_flag = nullptr;      // device flag of the early-stop check
  int* h_flag = nullptr;      // pinned host copy
  float* cg_alpha = nullptr;  // [B] per-system step of the current CG iteration
  int* cg_state = nullptr;    // [B] 0 update, 1 converged, 2 breakdown
  float* cg_alpha2 = nullptr;  // [B] the same for odd iterations (tensor-core path: x advanced per pair)
  int* cg_state2 = nullptr;
  bool pair_x = true;          // PICO_CG_PAIR_X=0: x advanced every iteration on the tensor-core path
  double* d_relres = nullptr;
  double* d_norm = nullptr;
  double* d_adapt = nullptr;
  float2* G = nullptr;  // PMR buffer, allocated on first use: Cartesian hybrid [B][nc][ny][nx],
                        // spiral gridded noise [B][nc][2n][2n]
  pico::CartOp cop{};
  // spiral operator
  pico::SpiralOp sop{};
  float* That = nullptr;
  float* deapod = nullptr;
  float2* tw2 = nullptr;
  float2* u = nullptr;
  float2* cphase = nullptr;
  int* tile_ptr = nullptr;
  int* tile_idx = nullptr;
  float* traj = nullptr;
  float* grid_w = nullptr;  // [nsamp][2][taps] gridding weights of each sample's window
  int2* grid_o = nullptr;   // [nsamp] first grid index of each window
  int64_t nsamp = 0;
  float2* Gt = nullptr;  // Toeplitz / 2-D intermediates [B][nc][n][L]
  bool mask2d = false;   // Cartesian with a 2-D sampling mask (normal operator by the 2-D passes, L = n)
  int toep_rl = 16;      // image rows per block of the Toeplitz / 2-D row passes
  // nonlinear CS state (pico_cs_*)
  bool cs_ready = false;
  int cs_iters = 0, cs_levels = 0;
  double cs_lc = 0, cs_tau = 0;
  std::vector<float> cs_c;     // momentum coefficients c_k
  float2* cs_traj = nullptr;   // [iters][n] wavelet coefficients W y_k of the reconstruction
  int cs_traj_cap = 0;         // iterations cs_traj has room for
  float2* cs_buf = nullptr;    // [6][B][n] work images
  float2* cs_ahb = nullptr;    // A^H b of the reconstruction's data [n]
  float2* cs_x0 = nullptr;     // the reconstruction f(b) [n]
  double cs_lam = 0;           // lambda_l1 of the reconstruction
  int64_t cs_generation = 0;   // pico_cs_recon calls so far (the linearisation point's version)
  pico::Wavelet wav{};
  // dense per-column normal operator on the tensor cores (Cartesian phase-encode
  // masks): CG vectors in the column-planar layout, two direction buffers
  bool gram = false;     // G built: batches of at least kGramMinBatch images use it
  bool gram_on = false;  // the batch in flight uses it (CG vectors column-planar)
  int pa_fft = 0, pa_gram = 0, gram_min_batch = 64;
  int probe_batch = 0;          // probes per CG batch of the map entry points (0: max_batch)
  std::vector<uint8_t> gmask;   // host copy of the phase-encode mask (rebuilding G)
  pico::GramOp gop{};
  CUtensorMap mR{}, mX{}, mP0{}, mP1{};
  float* P2 = nullptr;
  float* g_beta = nullptr;
  int* g_done = nullptr;
  bool gram_f16 = true;         // FP16 operands when the stage shape allows (PICO_GRAM_TF32=1: TF32)
  double* g_pn = nullptr;       // [B] FP16 form: bound on each direction's entries
  float* g_pscale = nullptr;    // [B] and its power-of-two operand scale
  int* g_err = nullptr;
  double2* g_pbuf = nullptr;
  pico::CgArgs cg{};
  // CG run per readout column (pico_set_solver): per (image, column) scalars
  int solver = PICO_SOLVER_GLOBAL;
  double *col_rr0 = nullptr, *col_rr = nullptr;
  float* col_beta = nullptr;
  int *col_done = nullptr, *col_iters = nullptr;
  double* col_pn = nullptr;     // FP16 form: bound on each column direction's entries [B][nx]
  float* col_pscale = nullptr;
  // larger phase-encode images: the whole per-column solve in one launch
  // (a cluster owns a column and 128 images; G_j tiled for its row blocks)
  bool persist_off = false;     // PICO_COLCG_PERSIST=0, TF32 operands, or the buffers do not fit
  void* per_G = nullptr;
  float* per_gscale = nullptr;
  uint8_t* per_split = nullptr;  // the split directions the cluster's CTAs share
  float2* col_G = nullptr;  // small images: G_j of every column, [nx][ny][ny] (whole solve on chip)
  float* col_gmax = nullptr;  // largest |component| of any G_j
  bool col_small = false;
  bool onchip = false;       // small phase-encode images: every CG solve runs on chip (either solver)
  pico::SmallGlobal sglob{};  // whole-image CG on chip: exchanged column partials
  std::string host_fail;  // a launch that could not be issued (reported by the entry point)
  size_t device_bytes = 0, budget = 0;
  bool async_alloc = false;  // stream-ordered cudaMallocAsync / cudaFreeAsync (serving contexts)
  std::vector<void*> allocs;
  std::string err;
  // launch accounting and optional per-class event timing
  int64_t launches = 0;
  bool profiling = false;
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> event_pool;
  double prof_ms[4] = {0, 0, 0, 0};
  int64_t prof_n[4] = {0, 0, 0, 0};
  // CUDA graphs of the CG iteration loop, keyed by (nb, max_iter, rtol, lam)
  cudaStream_t cap = nullptr;
  bool use_graphs = true;
  std::map<std::tuple<int, int, int, double, float>, std::pair<cudaGraphExec_t, int64_t>> graphs;
  std::set<std::tuple<int, int, int, double, float>> seen;
};

namespace {

pico_status fail(pico_ctx* c, pico_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

pico_status cuda_check(pico_ctx* c, const char* where) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, PICO_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  if (c && !c->host_fail.empty()) {
    const std::string m = std::string(where) + ": " + c->host_fail;
    c->host_fail.clear();
    return fail(c, PICO_E_CUDA, m);
  }
  return PICO_OK;
}

template <typename T>
pico_status dalloc(pico_ctx* c, T** p, size_t count) {
  const size_t bytes = count * sizeof(T);
  if (c->budget && c->device_bytes + bytes > c->budget)
    return fail(c, PICO_E_OOM, "device footprint exceeds hbm_budget");
  void* q = nullptr;
  const cudaError_t e = c->async_alloc ? cudaMallocAsync(&q, bytes, c->stream) : cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, PICO_E_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  c->allocs.push_back(q);
  c->device_bytes += bytes;
  *p = static_cast<T*>(q);
  return PICO_OK;
}

// Cholesky of a Hermitian positive-definite matrix (lower), FP64.
bool cholesky(std::vector<cd>& a, int n) {
  for (int j = 0; j < n; ++j) {
    double d = a[j * n + j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(a[j * n + k]);
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    a[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      cd s = a[i * n + j];
      for (int k = 0; k < j; ++k) s -= a[i * n + k] * std::conj(a[j * n + k]);
      a[i * n + j] = s / d;
    }
    for (int i = 0; i < j; ++i) a[i * n + j] = 0.0;
  }
  return true;
}

// inverse of a lower-triangular matrix by forward substitution
std::vector<cd> tril_inverse(const std::vector<cd>& L, int n) {
  std::vector<cd> inv(n * n, 0.0);
  for (int col = 0; col < n; ++col) {
    for (int i = 0; i < n; ++i) {
      cd s = (i == col) ? cd(1.0) : cd(0.0);
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * inv[k * n + col];
      inv[i * n + col] = s / L[i * n + i];
    }
  }
  return inv;
}

std::vector<float2> twiddles(int N) {
  std::vector<float2> t(N);
  for (int e = 0; e < N; ++e) {
    const double a = -2.0 * M_PI * (double)e / (double)N;
    t[e] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  return t;
}

constexpr uint64_t kPowerSeed = 0x50574D;  // start vector of the power method

cudaEvent_t take_event(pico_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Bracket one kernel launch: count it and, when profiling, time it with events.
struct Launch {
  pico_ctx* c;
  int cls;
  cudaEvent_t a = nullptr;
  Launch(pico_ctx* c_, int cls_, int kernels = 1) : c(c_), cls(cls_) {
    c->launches += kernels;
    count_ = kernels;
    if (c->profiling) {
      a = take_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  int count_ = 0;
  // correct the kernel count when fewer kernels than announced were launched
  void count(int delta) { c->launches += delta; count_ += delta; }
  ~Launch() {
    if (a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, c->stream);
      c->recs.push_back({cls, a, b});
    }
  }
};

void prof_collect(pico_ctx* c) {
  if (c->recs.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& r : c->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.cls] += ms;
      c->prof_n[r.cls] += 1;
    }
    c->event_pool.push_back(r.a);
    c->event_pool.push_back(r.b);
  }
  c->recs.clear();
}

float* cpf(float2* p) { return reinterpret_cast<float*>(p); }

// Pick the normal operator for a batch of nb images (sets the layout of the
// CG vectors and the number of p^H q partials per iteration).  Below
// gram_min_batch images (64 unless PICO_GRAM_MIN_BATCH says otherwise) the
// column-FFT kernel is as fast as the Gram operator, whose cost is dominated
// by streaming G once per launch.
void select_path(pico_ctx* c, int nb) {
  c->gram_on = c->gram && (nb >= c->gram_min_batch || c->solver == PICO_SOLVER_COLUMNS);
  c->cg.PA = c->gram_on ? c->pa_gram : c->pa_fft;
}
bool column_mode(const pico_ctx* c) { return c->solver == PICO_SOLVER_COLUMNS && c->gram_on; }
bool column_small(const pico_ctx* c) { return c->solver == PICO_SOLVER_COLUMNS && c->col_small; }
pico::ColCgArgs col_args(pico_ctx* c) {
  return pico::ColCgArgs{reinterpret_cast<float*>(c->X), reinterpret_cast<float*>(c->R), c->col_rr0, c->col_rr,
                         c->col_beta, c->col_done, c->col_iters, c->status, c->cg.rtol2, c->col_pn,
                         c->col_pscale};
}
// Gram mode: the direction written by CG iteration `it` (two buffers alternate,
// because the operator reads the previous direction while writing the new one)
float* gram_pbuf(pico_ctx* c, int it) { return (it & 1) ? c->P2 : cpf(c->P); }
const CUtensorMap& gram_pmap(pico_ctx* c, int it) { return (it & 1) ? c->mP1 : c->mP0; }
pico::CgArgs gram_cg(pico_ctx* c, int it) {
  pico::CgArgs a = c->cg;
  a.P = reinterpret_cast<float2*>(gram_pbuf(c, it));
  return a;
}

// (A^H A + lam) x for nb images (class 0).  Gram mode: x is one of the
// context's column-planar buffers X or R.
void op_apply(pico_ctx* c, const float2* x, float2* y, int nb, float lam) {
  if (c->gram_on) {
    const CUtensorMap& m = x == c->X ? c->mX : c->mR;
    pico::GramArgs g{};
    g.in = reinterpret_cast<const float*>(x);
    g.q = cpf(y);
    g.nb = nb;
    g.lam = lam;
    g.itmax = c->itmax;
    g.err = c->g_err;
    g.pscale = c->g_pscale;
    Launch L(c, 0, c->gop.f16 ? 2 : 1);
    if (c->gop.f16) pico::launch_gram_apply_scale(g.in, c->ny, c->nx, nb, c->g_pscale, c->stream);
    pico::launch_gram_normal(c->gop, m, m, g, c->stream);
    return;
  }
  if (c->kind == PICO_CARTESIAN && !c->mask2d) {
    Launch L(c, 0);
    pico::launch_cart_apply(c->cop, x, y, nb, lam, c->stream);
  } else {
    Launch L(c, 0, 3);
    pico::launch_toep_apply(c->sop, x, y, c->Gt, nb, lam, c->stream);
  }
}

// CG iteration `it`, operator half (class 0)
void op_cg_normal(pico_ctx* c, int nb, int it, float lam) {
  if (c->gram_on) {
    {
      Launch L(c, 1);
      pico::launch_gram_scalars(c->cg, nb, it, c->g_beta, c->g_done, c->gop.f16 ? c->g_pn : nullptr, c->g_pscale,
                                c->stream);
    }
    pico::GramArgs g{};
    g.in = cpf(c->R);
    g.pold = gram_pbuf(c, it + 1);
    g.pnew = gram_pbuf(c, it);
    g.q = cpf(c->Q);
    g.beta = c->g_beta;
    g.done = c->g_done;
    g.pscale = c->g_pscale;
    g.pq = c->cg.pq_part;
    g.itmax = c->itmax;
    g.PA = c->cg.PA;
    g.it = it;
    g.nb = nb;
    g.cg = 1;
    g.lam = lam;
    g.err = c->g_err;
    Launch L(c, 0);
    pico::launch_gram_normal(c->gop, c->mR, gram_pmap(c, it + 1), g, c->stream);
    return;
  }
  if (c->kind == PICO_CARTESIAN && !c->mask2d) {
    Launch L(c, 0);
    pico::launch_cart_cg_normal(c->cop, c->cg, nb, it, lam, c->stream);
  } else {
    Launch L(c, 0, 3);
    pico::launch_toep_cg_normal(c->sop, c->cg, c->Gt, nb, it, lam, c->stream);
  }
}

// The CG iterations of one batch: 2 * max_iter kernels (normal operator + update).
// Replayed from a CUDA graph (captured on a private stream the second time a
// (nb, max_iter, rtol, lam) combination is used) unless profiling is on.
// the paired x update of the tensor-core path (x advanced once per two
// iterations; the per-system step of iteration it in the set of its parity)
bool pair_path(const pico_ctx* c) { return c->gram_on && c->pair_x && c->n % 2 == 0 && !column_mode(c); }
float* pair_alpha(pico_ctx* c, int it) { return (it & 1) ? c->cg_alpha2 : c->cg_alpha; }
int* pair_state(pico_ctx* c, int it) { return (it & 1) ? c->cg_state2 : c->cg_state; }
// after iterations [0, last]: a solve that ended on an even iteration still
// owes x its last step
void pair_flush(pico_ctx* c, int nb, int last) {
  if (!pair_path(c) || last < 0 || (last & 1)) return;
  Launch L(c, 1);
  pico::launch_cg_flush_pair(gram_cg(c, last), nb, pair_alpha(c, last), pair_state(c, last),
                             reinterpret_cast<const float2*>(gram_pbuf(c, last)), c->stream);
}

// CG iterations [it0, it1) of one batch: 2-3 kernels per iteration (normal
// operator, step, update), replayed from a CUDA graph (captured on a private
// stream the second time a (nb, it0, it1, rtol, lam) combination is used)
// unless profiling is on.
void cg_range(pico_ctx* c, int nb, int it0, int it1, double rtol, float lam) {
  auto direct = [&]() {
    if (column_mode(c)) {
      // one fused launch per update: operator, step, x and r updates, next beta
      for (int it = it0; it < it1; ++it) {
        pico::GramArgs g{};
        g.in = cpf(c->R);
        g.pold = gram_pbuf(c, it + 1);
        g.pnew = gram_pbuf(c, it);
        g.itmax = c->itmax;
        g.it = it;
        g.nb = nb;
        g.cg = 1;
        g.lam = lam;
        g.err = c->g_err;
        Launch L(c, 0);
        if (!pico::launch_gram_colcg(c->gop, c->mR, gram_pmap(c, it + 1), g, col_args(c), c->stream))
          c->host_fail = "per-column CG launch failed (tile map encoding or cluster launch)";
      }
      return;
    }
    for (int it = it0; it < it1; ++it) {
      op_cg_normal(c, nb, it, lam);
      {
        Launch L(c, 1, 2);
        const pico::CgArgs a = c->gram_on ? gram_cg(c, it) : c->cg;
        if (pair_path(c)) {
          // the Gram path keeps p of it - 1 (the other direction buffer) through it:
          // x advances once per pair of iterations
          if (pico::launch_cg_step_pair(a, nb, it, pair_alpha(c, it), pair_state(c, it), pair_alpha(c, it + 1),
                                        pair_state(c, it + 1),
                                        reinterpret_cast<const float2*>(gram_pbuf(c, it + 1)), c->stream))
            continue;
        }
        if (!pico::launch_cg_step(a, nb, it, c->cg_alpha, c->cg_state, c->stream)) {
          L.count(-1);
          pico::launch_cg_update(a, nb, it, c->stream);
        }
      }
    }
  };
  if (c->profiling || !c->use_graphs || it1 <= it0) return direct();
  const auto key = std::make_tuple(nb, it0, it1, rtol, lam);
  auto itg = c->graphs.find(key);
  if (itg == c->graphs.end()) {
    if (c->seen.insert(key).second) return direct();  // first use: plain launches (sets kernel attributes)
    cudaStream_t user = c->stream;
    c->stream = c->cap;
    const int64_t before = c->launches;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool ok = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      direct();
      ok = cudaStreamEndCapture(c->cap, &g) == cudaSuccess && g;
    }
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    c->stream = user;
    const int64_t kernels = c->launches - before;
    c->launches = before;
    if (!ok) {
      cudaGetLastError();
      c->use_graphs = false;
      return direct();
    }
    itg = c->graphs.emplace(key, std::make_pair(ex, kernels)).first;
  }
  cudaGraphLaunch(itg->second.first, c->stream);
  c->launches += itg->second.second;
}

// With a residual tolerance the iterations run in chunks of kStopChunk; after
// each chunk one small kernel reports whether every system of the batch has
// met the stopping rule (or broken down), and the host stops there -- the
// remaining iterations would only skip converged systems.  Fixed-count
// solves (rtol = 0) run as one range without host synchronisation.
constexpr int kStopChunk = 4;
void cg_iterations(pico_ctx* c, int nb, int max_iter, double rtol, float lam) {
  c->cg.rtol2 = rtol * rtol;
  if (!(rtol > 0.0) || !c->h_flag) {
    cg_range(c, nb, 0, max_iter, rtol, lam);
    return pair_flush(c, nb, max_iter - 1);
  }
  int last = -1;  // last iteration run
  for (int it0 = 0; it0 < max_iter; it0 += kStopChunk) {
    const int it1 = std::min(max_iter, it0 + kStopChunk);
    cg_range(c, nb, it0, it1, rtol, lam);
    last = it1 - 1;
    if (it1 == max_iter) break;
    if (column_mode(c)) {
      { Launch L(c, 1); pico::launch_colcg_any_live(col_args(c), c->nx, nb, c->d_flag, c->stream); }
      cudaMemcpyAsync(c->h_flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return;
      if (!*c->h_flag) break;
      continue;
    }
    { Launch L(c, 1); pico::launch_cg_all_done(c->cg, nb, it1, c->d_flag, c->stream); }
    cudaMemcpyAsync(c->h_flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return;
    if (*c->h_flag) break;
  }
  pair_flush(c, nb, last);
}

// Per-column CG with the whole solve in one launch (FP16 operands, ny a
// multiple of a supported row block): G_j in the cluster's row tiling and the
// shared split-direction buffer, built on first use.  false: the per-update
// kernels run instead.
bool persist_setup(pico_ctx* c) {
  if (c->per_G) return true;
  if (c->persist_off || !c->gram || !c->gram_f16 || (size_t)c->nc * c->ny * 8 > 200 * 1024) return false;
  const int nt = pico::colcg_persist_rows(c->ny);
  if (!nt) return (c->persist_off = true, false);
  const size_t gbytes = (size_t)8 * c->nx * c->ny * c->ny;  // four FP16 planes
  const size_t sbytes = pico::colcg_persist_split_bytes(c->ny, c->nx, c->max_batch);
  if (c->budget && c->device_bytes + gbytes + sbytes + 4 * (size_t)c->nx > c->budget) return (c->persist_off = true, false);
  const std::string keep = c->err;
  if (dalloc(c, reinterpret_cast<uint8_t**>(&c->per_G), gbytes) != PICO_OK ||
      dalloc(c, &c->per_gscale, (size_t)c->nx) != PICO_OK || dalloc(c, &c->per_split, sbytes) != PICO_OK) {
    c->err = keep;  // not an error of the call: the per-update kernels take over
    c->per_G = nullptr;
    return (c->persist_off = true, false);
  }
  pico::GramOp op{};
  op.ny = c->ny;
  op.nx = c->nx;
  op.nt = nt;
  op.kc = 16;
  op.a_tmem = 0;
  op.f16 = 1;
  op.G = c->per_G;
  op.gscale = c->per_gscale;
  pico::launch_gram_build(c->smaps, c->gmask.data(), c->nc, op, c->g_pbuf, c->stream);
  return true;
}
bool persist_path(pico_ctx* c) { return column_mode(c) && persist_setup(c); }
void run_cg_persist(pico_ctx* c, int nb, int max_iter, double rtol, float lam) {
  Launch L(c, 0);
  if (!pico::launch_colcg_persist(c->per_G, c->per_gscale, cpf(c->R), reinterpret_cast<float*>(c->X), c->per_split,
                                  c->col_rr0, c->col_rr, c->col_iters, c->status, c->g_err, c->ny, c->nx, nb,
                                  max_iter, rtol * rtol, lam, c->stream))
    c->host_fail = "per-column CG launch failed (cluster launch of the whole solve)";
}

// the whole CG solve of small images on chip (per column, or the whole image
// with sum exchanges between the blocks of an image group): rhs in R, x to X
// (natural layout)
void run_cg_small(pico_ctx* c, int nb, int max_iter, double rtol, float lam) {
  Launch L(c, 0);
  const pico::SmallGlobal* glob = c->solver == PICO_SOLVER_COLUMNS ? nullptr : &c->sglob;
  if (!pico::launch_colcg_small(c->col_G, c->col_gmax, c->R, c->X, c->ny, c->nx, nb, max_iter, rtol * rtol, lam,
                                c->col_rr0, c->col_rr, c->col_iters, c->status, glob, c->stream))
    c->host_fail = "on-chip CG launch failed (cooperative launch of the whole-image solve)";
}
bool small_path(const pico_ctx* c) { return c->onchip || column_small(c); }

pico_status run_cg(pico_ctx* c, int nb, int max_iter, double rtol, float lam) {
  c->cg.rtol2 = rtol * rtol;
  if (small_path(c)) {
    run_cg_small(c, nb, max_iter, rtol, lam);
    return cuda_check(c, "cg");
  }
  if (persist_path(c)) {
    run_cg_persist(c, nb, max_iter, rtol, lam);
    return cuda_check(c, "cg");
  }
  if (column_mode(c)) {
    Launch L(c, 1);
    pico::launch_colcg_init(col_args(c), c->ny, c->nx, nb, c->stream);
  } else {
    Launch L(c, 1);
    pico::launch_cg_init_rhs(c->cg, nb, c->stream);
  }
  cg_iterations(c, nb, max_iter, rtol, lam);
  return cuda_check(c, "cg");
}

// CG start from probes: x = 0, r = v (the probes of indices begin ..)
void init_from_probe(pico_ctx* c, int nb, uint64_t seed, int64_t begin, int kind) {
  if (c->gram_on) {
    // probes drawn in the natural layout into Q, then rearranged into R
    pico::CgArgs a = c->cg;
    a.R = c->Q;
    { Launch L(c, 1); pico::launch_cg_init_probe(a, nb, seed, begin, kind, c->stream); }
    { Launch L(c, 1); pico::launch_to_cp(c->Q, cpf(c->R), c->ny, c->nx, nb, c->stream); }
  } else {
    Launch L(c, 1);
    pico::launch_cg_init_probe(c->cg, nb, seed, begin, kind, c->stream);
  }
}

pico_status run_cg_from_probe(pico_ctx* c, int nb, int max_iter, double rtol, float lam, uint64_t seed,
                              int64_t begin, int kind) {
  c->cg.rtol2 = rtol * rtol;
  init_from_probe(c, nb, seed, begin, kind);
  if (small_path(c)) {
    run_cg_small(c, nb, max_iter, rtol, lam);
    return cuda_check(c, "cg");
  }
  if (persist_path(c)) {
    run_cg_persist(c, nb, max_iter, rtol, lam);
    return cuda_check(c, "cg");
  }
  if (column_mode(c)) {
    Launch L(c, 1);
    pico::launch_colcg_init(col_args(c), c->ny, c->nx, nb, c->stream);
  }
  cg_iterations(c, nb, max_iter, rtol, lam);
  return cuda_check(c, "cg");
}

// captured CG graphs depend on the operator choice, which their key omits
void clear_graphs(pico_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.first);
  c->graphs.clear();
  c->seen.clear();
}

// probes / replicas per CG batch of the map entry points
int probe_chunk(const pico_ctx* c) {
  return c->probe_batch > 0 ? std::min(c->probe_batch, c->max_batch) : c->max_batch;
}

// k-space / grid work buffer shared by PMR, the forward and the adjoint operator:
// Cartesian [B][nc][ny][nx], spiral [B][nc][2n][2n]; allocated on first use
pico_status ensure_kbuf(pico_ctx* c) {
  if (c->G) return PICO_OK;
  const size_t per = c->kind == PICO_CARTESIAN ? (size_t)c->n : (size_t)4 * c->n;
  return dalloc(c, &c->G, (size_t)c->max_batch * c->nc * per);
}

// 2-D mask adjoint of k-space planes already in c->G (masked, scaled): inverse
// column and row FFTs in place, then the conj(S) coil combine into out [nb][n]
void adjoint2d_from_kbuf(pico_ctx* c, float2* out, int nb) {
  const int n1 = c->ny;
  { Launch L(c, 2); pico::launch_fft_cols(n1, c->G, c->tw2, c->nx, nb * c->nc, c->n, 1, c->stream); }
  { Launch L(c, 2); pico::launch_fft_rows(c->nx, c->G, c->tw2, c->ny, nb * c->nc, c->n, 1, c->stream); }
  { Launch L(c, 2); pico::launch_coil_combine(c->G, c->smaps, c->nc, out, c->n, nb, c->stream); }
}

pico_status check_iter(pico_ctx* c, int max_iter, double rtol) {
  if (max_iter < 0 || max_iter > c->itmax) return fail(c, PICO_E_INVALID, "max_iter outside [0, max_iter_cap]");
  if (!(rtol >= 0.0)) return fail(c, PICO_E_INVALID, "rtol must be >= 0");
  return PICO_OK;
}


// 2-D Cartesian mask: the normal operator runs the unpadded 2-D passes with the
// real multiplier mask(ky, kx) / n^2 (orthonormal DFT pair), L = n.
pico_status cart2d_setup(pico_ctx* c, const pico_operator_desc* d, int img, int P1, int P2) {
  const int64_t n = c->n;
  pico_status st = PICO_OK;
  if ((st = dalloc(c, &c->That, (size_t)n)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->tw2, (size_t)img)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->mask, (size_t)n)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->Gt, std::max((size_t)c->max_batch * c->nc * n, (size_t)n))) != PICO_OK) return st;
  std::vector<float> T(n);
  for (int64_t i = 0; i < n; ++i) T[i] = d->mask[i] ? (float)(1.0 / (double)n) : 0.f;
  const std::vector<float2> tw = twiddles(img);
  cudaMemcpyAsync(c->That, T.data(), T.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(c->tw2, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(c->mask, d->mask, (size_t)n, cudaMemcpyHostToDevice, c->stream);
  c->sop = pico::SpiralOp{};
  c->sop.n = img;
  c->sop.L = img;
  c->sop.nc = c->nc;
  c->sop.P1 = P1;
  c->sop.P2 = P2;
  c->sop.smaps = c->smaps;
  c->sop.tw2 = c->tw2;
  c->sop.That = c->That;
  c->sop.err = c->g_err;
  c->sop.row_lines = c->toep_rl;
  c->twx = c->tw2;
  c->tw = c->tw2;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "2-D mask set-up");
  return PICO_OK;
}

// I0(x) by its power series sum_k (x^2/4)^k / (k!)^2 (FP64; x < 30 here)
double bessel_i0(double x) {
  const double q = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 200; ++k) {
    term *= q / ((double)k * (double)k);
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}

// Spiral operator set-up: trajectory, gridding bins, deapodisation, twiddles,
// and the Toeplitz kernel T^ = DFT_2N(h) / ((2N)^2 N^2) computed on the device.
pico_status spiral_setup(pico_ctx* c, const pico_operator_desc* d, int img, int L, int P1, int P2, int kbw) {
  const int64_t M = c->nsamp;
  const int nc = c->nc;
  pico_status st = PICO_OK;
  if ((st = dalloc(c, &c->traj, (size_t)2 * M)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->u, (size_t)M)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->cphase, (size_t)M)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->That, (size_t)L * L)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->deapod, (size_t)img)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->tw2, (size_t)L)) != PICO_OK) return st;
  // Toeplitz intermediates; also holds the (2N)^2 kernel during set-up
  if ((st = dalloc(c, &c->Gt, std::max((size_t)c->max_batch * nc * img * L, (size_t)L * L))) != PICO_OK) return st;

  // sample positions on the 2N grid (u = 2k), image-centre phase e^{i pi (kx + ky)}
  const double hw = 0.5 * kbw;
  const int tiles_x = L / 16, ntiles = tiles_x * tiles_x;
  std::vector<float2> u(M), ph(M);
  std::vector<int> cnt(ntiles + 1, 0);
  std::vector<std::vector<int>> touch(M);
  for (int64_t m = 0; m < M; ++m) {
    const double kx = d->traj[2 * m], ky = d->traj[2 * m + 1];
    if (!std::isfinite(kx) || !std::isfinite(ky)) return fail(c, PICO_E_INVALID, "non-finite trajectory sample");
    u[m] = make_float2((float)(2.0 * kx), (float)(2.0 * ky));
    const double a = M_PI * (kx + ky);
    ph[m] = make_float2((float)std::cos(a), (float)std::sin(a));
    // grid tiles within the kernel half-width (conservative by 1e-3 grid units)
    const double ux = 2.0 * kx, uy = 2.0 * ky;
    int tx[4], ty[4], ntx = 0, nty = 0;
    for (int g = (int)std::floor(ux - hw - 1e-3); g <= (int)std::ceil(ux + hw + 1e-3); ++g) {
      const int t = (((g % L) + L) % L) / 16;
      bool seen = false;
      for (int i = 0; i < ntx; ++i) seen |= tx[i] == t;
      if (!seen && ntx < 4) tx[ntx++] = t;
    }
    for (int g = (int)std::floor(uy - hw - 1e-3); g <= (int)std::ceil(uy + hw + 1e-3); ++g) {
      const int t = (((g % L) + L) % L) / 16;
      bool seen = false;
      for (int i = 0; i < nty; ++i) seen |= ty[i] == t;
      if (!seen && nty < 4) ty[nty++] = t;
    }
    for (int i = 0; i < nty; ++i)
      for (int j = 0; j < ntx; ++j) {
        touch[m].push_back(ty[i] * tiles_x + tx[j]);
        cnt[ty[i] * tiles_x + tx[j] + 1]++;
      }
  }
  for (int t = 0; t < ntiles; ++t) cnt[t + 1] += cnt[t];
  std::vector<int> idx(cnt[ntiles]);
  std::vector<int> fillp(cnt.begin(), cnt.end() - 1);
  for (int64_t m = 0; m < M; ++m)
    for (int t : touch[m]) idx[fillp[t]++] = (int)m;  // increasing sample order inside each tile
  if ((st = dalloc(c, &c->tile_ptr, (size_t)ntiles + 1)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->tile_idx, std::max<size_t>(1, idx.size()))) != PICO_OK) return st;

  // Kaiser-Bessel kernel phi(t) = I0(beta sqrt(1 - (2t/W)^2)) / I0(beta) and its
  // Fourier transform phi^(nu) = W sinh(z)/z / I0(beta), z = sqrt(beta^2 - (pi W nu)^2)
  const double os = 2.0;
  const double beta = M_PI * std::sqrt((kbw / os) * (kbw / os) * (os - 0.5) * (os - 0.5) - 0.8);
  const double i0b = bessel_i0(beta);
  std::vector<float> dap(img);
  for (int x = 0; x < img; ++x) {
    const double nu = (double)(x - img / 2) / (double)L;
    const double z2 = beta * beta - (M_PI * kbw * nu) * (M_PI * kbw * nu);
    double ft;
    if (z2 > 0) {
      const double z = std::sqrt(z2);
      ft = kbw * std::sinh(z) / z;
    } else {
      const double z = std::sqrt(-z2);
      ft = z > 0 ? kbw * std::sin(z) / z : (double)kbw;
    }
    dap[x] = (float)(1.0 / ((ft / i0b) * std::sqrt((double)img)));
  }
  const std::vector<float2> tw = twiddles(L);
  cudaMemcpyAsync(c->traj, d->traj, (size_t)2 * M * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(c->u, u.data(), (size_t)M * sizeof(float2), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(c->cphase, ph.data(), (size_t)M * sizeof(float2), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(c->tile_ptr, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream);
  if (!idx.empty())
    cudaMemcpyAsync(c->tile_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(c->deapod, dap.data(), dap.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(c->tw2, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream);

  c->sop = pico::SpiralOp{img,      L,         nc,         P1,          P2,           c->smaps,
                          c->tw2,   c->That,   c->deapod,  M,           c->u,         c->cphase,
                          c->tile_ptr, c->tile_idx, (float)beta, (float)hw, (float)(1.0 / i0b), c->g_err,
                          c->toep_rl};
  // the Kaiser-Bessel window of every sample, once (the gridding of each PMR
  // replica batch and pico_adjoint look the weights up)
  if ((st = dalloc(c, &c->grid_w, std::max<size_t>(1, pico::grid_table_floats(M)))) != PICO_OK) return st;
  if ((st = dalloc(c, &c->grid_o, std::max<size_t>(1, (size_t)M))) != PICO_OK) return st;
  c->sop.gw = c->grid_w;
  c->sop.go = c->grid_o;
  { Launch Lg(c, 3); pico::launch_grid_table(c->sop, c->grid_w, c->grid_o, c->stream); }
  // Toeplitz kernel: h on the 2N grid (in the Toeplitz buffer), 2-D DFT, real part, scale
  float2* cbuf = c->Gt;  // max_batch * nc * N * 2N >= (2N)^2 complex values
  { Launch Lh(c, 3); pico::launch_toep_h(c->traj, M, img, cbuf, c->stream); }
  { Launch Lf(c, 3, 2); pico::launch_toep_fft2(c->sop, cbuf, c->stream); }
  const double scale = 1.0 / ((double)img * img * (double)L * L);
  { Launch Lz(c, 3); pico::launch_toep_finalize(cbuf, L, (float)scale, c->That, c->stream); }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "spiral set-up");
  return cuda_check(c, "spiral set-up");
}


// ---------------------------------------------------------------------------
// nonlinear CS: L1-wavelet FISTA and its Jacobian (Sec. 2.2.5)
// ---------------------------------------------------------------------------
// Daubechies' orthonormal scaling filter with 4 vanishing moments (8 taps), as
// tabulated by Daubechies (Comm. Pure Appl. Math. 41, 1988, Table 1).
constexpr double kDb4[8] = {0.2303778133088964,  0.7148465705529154, 0.6308807679298587, -0.0279837694168599,
                            -0.1870348117190931, 0.0308413818355607, 0.0328830116668852, -0.0105974017850690};

pico_status cs_buffers(pico_ctx* c) {
  if (c->cs_buf) return PICO_OK;
  pico_status st = dalloc(c, &c->cs_buf, (size_t)6 * c->max_batch * c->n);
  if (st == PICO_OK) st = dalloc(c, &c->cs_ahb, (size_t)c->n);
  if (st == PICO_OK) st = dalloc(c, &c->cs_x0, (size_t)c->n);
  for (int m = 0; m < 8; ++m) {
    c->wav.h[m] = (float)kDb4[m];
    c->wav.g[m] = (float)((m % 2 ? -1.0 : 1.0) * kDb4[7 - m]);
  }
  c->wav.L = 8;
  return st;
}
float2* cs_e(pico_ctx* c, int k) { return c->cs_buf + (size_t)k * c->max_batch * c->n; }

void cs_W(pico_ctx* c, const float2* x, float2* coef, float2* tmp, int nb, int levels) {
  Launch L(c, 3, pico::dwt_kernels(levels));
  pico::launch_dwt(x, coef, tmp, c->ny, levels, nb, c->wav, c->stream);
}
void cs_WH(pico_ctx* c, const float2* coef, float2* x, float2* tmp, int nb, int levels) {
  Launch L(c, 3, pico::idwt_kernels(levels, coef == x));
  pico::launch_idwt(coef, x, tmp, c->ny, levels, nb, c->wav, c->stream);
}

// FISTA iterations on nb data terms A^H b_i (rhs, stride rhs_stride; 0 = one broadcast term).
// Result x in E0 (E1..E3 work).  With `keep`, nb == 1 and W y_k is stored as the
// linearisation point of the Jacobian.
void cs_fista(pico_ctx* c, const float2* rhs, int64_t rhs_stride, int nb, bool keep) {
  float2 *x = cs_e(c, 0), *z = cs_e(c, 1), *t2 = cs_e(c, 2), *t3 = cs_e(c, 3);
  const int64_t n = c->n;
  const float inv_lc = (float)(1.0 / c->cs_lc), tau = (float)c->cs_tau;
  cudaMemsetAsync(x, 0, (size_t)nb * n * sizeof(float2), c->stream);
  cudaMemsetAsync(z, 0, (size_t)nb * n * sizeof(float2), c->stream);
  for (int k = 0; k < c->cs_iters; ++k) {
    op_apply(c, z, t2, nb, 0.f);
    { Launch L(c, 3); pico::launch_cs_gradstep(z, t2, rhs, rhs_stride, inv_lc, t3, n, nb, c->stream); }
    cs_W(c, t3, t3, t2, nb, c->cs_levels);
    { Launch L(c, 3); pico::launch_cs_soft(t3, keep ? c->cs_traj + (size_t)k * n : nullptr, t3, tau, n, nb,
                                           c->stream); }
    cs_WH(c, t3, t3, t2, nb, c->cs_levels);
    { Launch L(c, 3); pico::launch_cs_momentum(t3, x, z, c->cs_c[k], n, nb, c->stream); }
  }
}

// dx (E0) = J applied to the image-domain tangent A^H db given in `ahdb` [nb][n]
void cs_jvp_core(pico_ctx* c, const float2* ahdb, int nb) {
  float2 *dx = cs_e(c, 0), *dz = cs_e(c, 1), *t2 = cs_e(c, 2), *t3 = cs_e(c, 3);
  const int64_t n = c->n;
  const float inv_lc = (float)(1.0 / c->cs_lc), tau = (float)c->cs_tau;
  cudaMemsetAsync(dx, 0, (size_t)nb * n * sizeof(float2), c->stream);
  cudaMemsetAsync(dz, 0, (size_t)nb * n * sizeof(float2), c->stream);
  for (int k = 0; k < c->cs_iters; ++k) {
    op_apply(c, dz, t2, nb, 0.f);
    { Launch L(c, 3); pico::launch_cs_gradstep(dz, t2, ahdb, n, inv_lc, t3, n, nb, c->stream); }
    cs_W(c, t3, t3, t2, nb, c->cs_levels);
    { Launch L(c, 3); pico::launch_cs_soft_tan(c->cs_traj + (size_t)k * n, t3, tau, n, nb, c->stream); }
    cs_WH(c, t3, t3, t2, nb, c->cs_levels);
    { Launch L(c, 3); pico::launch_cs_momentum(t3, dx, dz, c->cs_c[k], n, nb, c->stream); }
  }
}

// E0 = (sum_k ybar_k) / Lc for the output cotangent `xbar` [nb][n] (reverse sweep)
void cs_vjp_core(pico_ctx* c, const float2* xbar, int nb) {
  float2 *ys = cs_e(c, 0), *zb = cs_e(c, 1), *t2 = cs_e(c, 2), *t3 = cs_e(c, 3), *xbn = cs_e(c, 5);
  const int64_t n = c->n;
  const float inv_lc = (float)(1.0 / c->cs_lc), tau = (float)c->cs_tau;
  cudaMemsetAsync(ys, 0, (size_t)nb * n * sizeof(float2), c->stream);
  cudaMemsetAsync(zb, 0, (size_t)nb * n * sizeof(float2), c->stream);
  cudaMemcpyAsync(xbn, xbar, (size_t)nb * n * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream);
  for (int k = c->cs_iters - 1; k >= 0; --k) {
    { Launch L(c, 3); pico::launch_vjp_a(xbn, zb, t3, c->cs_c[k], n, nb, c->stream); }
    cs_W(c, t3, t3, t2, nb, c->cs_levels);
    { Launch L(c, 3); pico::launch_cs_soft_tan(c->cs_traj + (size_t)k * n, t3, tau, n, nb, c->stream); }
    cs_WH(c, t3, t3, t2, nb, c->cs_levels);
    op_apply(c, t3, t2, nb, 0.f);
    { Launch L(c, 3); pico::launch_vjp_b(t3, t2, inv_lc, zb, ys, n, nb, c->stream); }
  }
  { Launch L(c, 3); pico::launch_scale(ys, inv_lc, n, nb, c->stream); }
}

// out[b] = A^H n_b for the whitened k-space noise of replicas rep_begin.. (PMR, Sec. 1); needs ensure_kbuf
void noise_adjoint(pico_ctx* c, float2* out, int nb, uint64_t seed, int64_t rep_begin, double sigma) {
  if (c->mask2d) {
    { Launch L(c, 2); pico::launch_noise_kspace2d(c->G, c->mask, c->nc, c->n, nb, seed, rep_begin,
                                                  (float)(sigma / std::sqrt((double)c->n)), c->stream); }
    adjoint2d_from_kbuf(c, out, nb);
  } else if (c->kind == PICO_CARTESIAN) {
    { Launch L(c, 2); pico::launch_cart_pmr_cols(c->cop, c->G, nb, seed, rep_begin, (float)sigma, c->stream); }
    { Launch L(c, 2); pico::launch_cart_rows_adjoint(c->cop, c->G, out, nb, c->stream); }
  } else {
    { Launch L(c, 2); pico::launch_grid_pmr(c->sop, c->G, nb, seed, rep_begin, (float)sigma, c->stream); }
    { Launch L(c, 2, 2); pico::launch_grid_adjoint_rest(c->sop, c->G, out, nb, c->stream); }
  }
}

// The dense Gram operator serves Cartesian phase-encode masks with ny a multiple
// of 16 and at least 128 (smaller images stay on the column-FFT kernel, which is
// latency-bound there anyway); PICO_NORMAL_OP=fft in the environment opts out.
bool want_gram(const pico_operator_desc* d) {
  if (d->kind != PICO_CARTESIAN || d->mask_2d) return false;
  const char* e = std::getenv("PICO_NORMAL_OP");
  if (e && std::string(e) == "fft") return false;
  return d->ny >= 128 && pico::gram_supported(d->ny, d->nx);
}

// Small phase-encode Cartesian images (ny = 32, 64, 96): the CG solves run on
// chip (G_j and the vectors in shared memory, one cooperative launch per
// solve); PICO_NORMAL_OP=fft keeps the column-FFT path.
bool want_onchip(const pico_operator_desc* d) {
  if (d->kind != PICO_CARTESIAN || d->mask_2d) return false;
  const char* e = std::getenv("PICO_NORMAL_OP");
  if (e && std::string(e) == "fft") return false;
  return pico::colcg_small_supported(d->ny);
}
// Image rows per block of the Toeplitz / 2-D-mask row passes: 4 (blocks of
// a quarter of the threads, four per SM) unless PICO_TOEP_ROWS=16 in the
// environment asks for one block of 16 rows per SM.  The p^H q partials per
// image are one per row block.
int toep_row_lines() {
  const char* e = std::getenv("PICO_TOEP_ROWS");
  return e && std::atoi(e) == 16 ? 16 : 4;
}

size_t onchip_extra_bytes(const pico_operator_desc* d, int64_t B) {
  return (size_t)d->nx * d->ny * d->ny * 8 + 4 + (size_t)d->ny * 16 + (size_t)B * d->nx * (8 + 8 + 4 + 16 + 16);
}

// G planes, second direction buffer and per-image scalars of the Gram mode
size_t gram_extra_bytes(const pico_operator_desc* d, int64_t B) {
  return pico::gram_bytes(d->ny, d->nx) + (size_t)B * d->ny * d->nx * 8 + (size_t)B * 8 + (size_t)d->ny * 16 + 16 +
         (size_t)B * 12 + (size_t)d->nx * 4;
}

// Small phase-encode images: G_j of every column (plain layout) and the
// per-(image, column) state of the on-chip solves; `global` adds the column
// partials and grid-barrier words of the whole-image solve.
pico_status small_setup(pico_ctx* c, bool global) {
  pico_status st = PICO_OK;
  const size_t n = (size_t)c->max_batch * c->nx;
  if (!c->col_G) {
    if ((st = dalloc(c, &c->col_G, (size_t)c->nx * c->ny * c->ny)) != PICO_OK) return st;
    if ((st = dalloc(c, &c->col_gmax, (size_t)1)) != PICO_OK) return st;
    if (!c->g_pbuf && (st = dalloc(c, &c->g_pbuf, (size_t)c->ny)) != PICO_OK) return st;
    pico::launch_colcg_small_build(c->smaps, c->gmask.data(), c->nc, c->ny, c->nx, c->col_G, c->col_gmax, c->g_pbuf,
                                   c->stream);
  }
  if ((!c->col_rr0 && (st = dalloc(c, &c->col_rr0, n)) != PICO_OK) ||
      (!c->col_rr && (st = dalloc(c, &c->col_rr, n)) != PICO_OK) ||
      (!c->col_iters && (st = dalloc(c, &c->col_iters, n)) != PICO_OK))
    return st;
  if (global && !c->sglob.part_pq) {
    if ((st = dalloc(c, &c->sglob.part_pq, n)) != PICO_OK || (st = dalloc(c, &c->sglob.part_rr, n)) != PICO_OK)
      return st;
    c->sglob.err = c->g_err;
  }
  return cuda_check(c, "on-chip CG set-up");
}

// (re)build the stage-tiled G_j for gop.kc and the tensor maps of the CG vectors
pico_status gram_configure(pico_ctx* c) {
  const int kc = c->gop.kc;
  // the format G is built in follows the stage shape: FP16 operands need 16-value
  // stages staged in shared memory
  c->gop.f16 = c->gram_f16 && kc == 16 && !c->gop.a_tmem && (size_t)c->nc * c->ny * 8 <= 200 * 1024;
  pico::launch_gram_build(c->smaps, c->gmask.data(), c->nc, c->gop, c->g_pbuf, c->stream);
  const int B = c->max_batch;
  const bool ok = pico::gram_encode_x(&c->mR, cpf(c->R), c->ny, c->nx, B, kc) &&
                  pico::gram_encode_x(&c->mX, cpf(c->X), c->ny, c->nx, B, kc) &&
                  pico::gram_encode_x(&c->mP0, cpf(c->P), c->ny, c->nx, B, kc) &&
                  pico::gram_encode_x(&c->mP1, c->P2, c->ny, c->nx, B, kc);
  if (!ok) return fail(c, PICO_E_CUDA, "tensor map encoding for the Gram operator failed");
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "Gram operator set-up");
  return cuda_check(c, "Gram operator set-up");
}

pico_status gram_setup(pico_ctx* c, const pico_operator_desc* d) {
  pico_status st = PICO_OK;
  float* gbuf = nullptr;  // room for the TF32 form (the FP16 form takes half)
  if ((st = dalloc(c, &gbuf, pico::gram_bytes(c->ny, c->nx) / sizeof(float))) != PICO_OK) return st;
  c->gop.G = gbuf;
  if ((st = dalloc(c, &c->P2, (size_t)2 * c->max_batch * c->n)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->g_beta, (size_t)c->max_batch)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->g_done, (size_t)c->max_batch)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->g_pn, (size_t)c->max_batch)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->g_pscale, (size_t)c->max_batch)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->gop.gscale, (size_t)c->nx)) != PICO_OK) return st;
  if (const char* e = std::getenv("PICO_GRAM_TF32")) c->gram_f16 = std::atoi(e) == 0;
  if (const char* e = std::getenv("PICO_COLCG_PERSIST")) c->persist_off = std::atoi(e) == 0;
  if (!c->g_err && (st = dalloc(c, &c->g_err, (size_t)4)) != PICO_OK) return st;
  if ((st = dalloc(c, &c->g_pbuf, (size_t)c->ny)) != PICO_OK) return st;
  cudaMemsetAsync(c->g_err, 0, 4 * sizeof(int), c->stream);
  if (const char* e = std::getenv("PICO_GRAM_MIN_BATCH")) c->gram_min_batch = std::max(1, std::atoi(e));
  c->gop.ny = c->ny;
  c->gop.nx = c->nx;
  c->gop.nt = pico::gram_tile(c->ny);
  c->gop.kc = 16;
  if (const char* e = std::getenv("PICO_GRAM_KC")) c->gop.kc = std::atoi(e) == 8 ? 8 : 16;
  // the direction's split can also be staged in tensor memory (measured about
  // 1 % slower than shared memory on the 320 x 320 knee operator; kept as an option)
  c->gop.a_tmem = 0;
  if (const char* e = std::getenv("PICO_GRAM_ATMEM")) c->gop.a_tmem = std::atoi(e) != 0;
  c->gmask.assign(d->mask, d->mask + c->ny);
  if ((st = gram_configure(c)) != PICO_OK) return st;
  c->gram = true;
  return PICO_OK;
}

pico_status wavelet_check(pico_ctx* c, int levels) {
  if (c->ny != c->nx || levels > 30 || (c->ny % (1 << levels)) != 0 || (c->ny >> levels) < 1)
    return fail(c, PICO_E_UNSUPPORTED, "the wavelet transform needs a square image divisible by 2^levels");
  return PICO_OK;
}

pico_status cs_check(pico_ctx* c) {
  if (!c || !c->smaps) return PICO_E_INVALID;
  if (!c->cs_ready) return fail(c, PICO_E_INVALID, "run pico_cs_recon first");
  select_path(c, 0);  // the CS iterations keep images in the natural layout
  return PICO_OK;
}
}  // namespace

extern "C" {

}  // extern "C"

namespace pico {

pico_status init_impl(const pico_operator_desc* d, void* cuda_stream, size_t hbm_budget, bool async_alloc,
                      pico_ctx** out) {
  if (!out) return PICO_E_INVALID;
  *out = nullptr;
  if (!d || !d->smaps) return PICO_E_INVALID;
  if (d->ny <= 0 || d->nx <= 0 || d->ncoils <= 0) return PICO_E_INVALID;
  if (d->kind != PICO_CARTESIAN && d->kind != PICO_SPIRAL) return PICO_E_INVALID;
  if (d->kind == PICO_CARTESIAN && !d->mask) return PICO_E_INVALID;
  if (d->kind == PICO_SPIRAL && (!d->traj || d->nsamp <= 0 || d->nsamp > (int64_t)1 << 30)) return PICO_E_INVALID;
  if (d->lambda < 0.0 || d->power_iters < 0 || d->max_batch < 0 || d->max_iter_cap < 0) return PICO_E_INVALID;

  auto* c = new pico_ctx();
  *out = c;
  c->async_alloc = async_alloc;
  c->kind = d->kind;
  c->ny = d->ny;
  c->nx = d->nx;
  c->nc = d->ncoils;
  c->n = (int64_t)d->ny * d->nx;
  c->stream = (cudaStream_t)cuda_stream;
  c->lam_rel = d->lambda;
  c->power_iters = d->power_iters;
  c->margin = d->power_margin > 0 ? d->power_margin : 1.01;
  c->max_batch = d->max_batch > 0 ? d->max_batch : 64;
  c->itmax = d->max_iter_cap > 0 ? d->max_iter_cap : 128;
  c->budget = hbm_budget;
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    c->cap = nullptr;
    c->use_graphs = false;
    cudaGetLastError();
  }
  const int nc = c->nc;
  const int64_t n = c->n, B = c->max_batch;
  const int PB = (int)((n + pico::kVecPerBlock - 1) / pico::kVecPerBlock);

  int N1 = 0, N2 = 0, M1 = 0, M2 = 0, P1 = 0, P2 = 0;
  int PA = 0;
  const int img = c->ny;  // spiral images are square
  const int L = 2 * img;
  const int kbw = d->kb_width > 0 ? d->kb_width : 6;
  const double os = d->oversamp > 0 ? (double)d->oversamp : 2.0;
  size_t extra = 0;
  c->mask2d = c->kind == PICO_CARTESIAN && d->mask_2d != 0;
  if (c->mask2d) {
    if (c->ny != c->nx) return fail(c, PICO_E_UNSUPPORTED, "2-D masks need square images");
    if (!pico::grid_split(img, &P1, &P2) || !pico::fft_length_supported(img))
      return fail(c, PICO_E_UNSUPPORTED, "image size has no 2-D FFT split in this build");
    c->toep_rl = toep_row_lines();
    PA = (img + c->toep_rl - 1) / c->toep_rl;
    extra = std::max((size_t)B * nc * n, (size_t)n) * 8 + (size_t)n * 5 + (size_t)img * 8;
  } else if (c->kind == PICO_CARTESIAN) {
    if (!pico::cart_supported(c->ny, c->nx, &N1, &N2, &M1, &M2))
      return fail(c, PICO_E_UNSUPPORTED, "ny has no FFT split in this build");
    PA = pico::cart_normal_tiles(c->nx);
    extra = (size_t)c->ny * 13 + (size_t)c->nx * 8;
    if (want_onchip(d)) extra += onchip_extra_bytes(d, B);
    if (want_gram(d)) {
      c->pa_gram = pico::gram_pa(c->ny, c->nx);
      c->pa_fft = PA;
      PA = std::max(PA, c->pa_gram);
      extra += gram_extra_bytes(d, B);
    }
  } else {
    if (c->ny != c->nx) return fail(c, PICO_E_UNSUPPORTED, "spiral images must be square");
    if (os != 2.0) return fail(c, PICO_E_UNSUPPORTED, "spiral gridding supports oversampling 2.0 only");
    if (kbw < 2 || kbw > 8 || (kbw & 1)) return fail(c, PICO_E_UNSUPPORTED, "kb_width must be 2, 4, 6 or 8");
    if (!pico::spiral_supported(img, &P1, &P2))
      return fail(c, PICO_E_UNSUPPORTED, "spiral image size has no 2N grid split in this build");
    c->toep_rl = toep_row_lines();
    PA = (img + c->toep_rl - 1) / c->toep_rl;
    c->nsamp = d->nsamp;
    extra = std::max((size_t)B * nc * img * L, (size_t)L * L) * 8 + (size_t)L * L * 4 + (size_t)img * 4 + (size_t)L * 8 +
            (size_t)c->nsamp * (8 + 8 + 8 + 16 + 88) + (size_t)(L / 16) * (L / 16) * 4 + 64;
  }

  // footprint check before allocating anything
  const size_t need = (size_t)nc * n * 8 + (size_t)nc * nc * 16 + (size_t)4 * B * n * 8 + (size_t)B * (c->itmax + 1) * PB * 8 +
                      (size_t)B * c->itmax * PA * 8 + (size_t)B * 16 + (size_t)PB * 8 + 64 + extra;
  if (hbm_budget && need > hbm_budget)
    return fail(c, PICO_E_OOM, "operator and workspace need " + std::to_string(need) + " bytes > hbm_budget");

  // whitening (Eq. 3): S' = L^-1 S with L L^H = Sigma_n.  L^-1 (nc x nc) is
  // formed on the host; the per-voxel product runs on the device (FP64) for up
  // to pico::kWhitenMaxCoils coils, on the host beyond that.
  std::vector<float2> S;
  std::vector<double2> Li_dev;
  if (d->noise_cov) {
    std::vector<cd> Lc((size_t)nc * nc);
    for (int i = 0; i < nc * nc; ++i) Lc[i] = cd(d->noise_cov[2 * i], d->noise_cov[2 * i + 1]);
    if (!cholesky(Lc, nc)) return fail(c, PICO_E_INVALID, "noise_cov is not Hermitian positive definite");
    const std::vector<cd> Li = tril_inverse(Lc, nc);
    if (nc <= pico::kWhitenMaxCoils) {
      Li_dev.resize((size_t)nc * nc);
      for (int i = 0; i < nc * nc; ++i) Li_dev[i] = make_double2(Li[i].real(), Li[i].imag());
    } else {
      S.resize((size_t)nc * n);
      std::memcpy(S.data(), d->smaps, S.size() * sizeof(float2));
      std::vector<float2> W((size_t)nc * n);
      std::vector<cd> col(nc);
      for (int64_t v = 0; v < n; ++v) {
        for (int k = 0; k < nc; ++k) col[k] = cd(S[(size_t)k * n + v].x, S[(size_t)k * n + v].y);
        for (int i = 0; i < nc; ++i) {
          cd acc = 0.0;
          for (int k = 0; k <= i; ++k) acc += Li[i * nc + k] * col[k];
          W[(size_t)i * n + v] = make_float2((float)acc.real(), (float)acc.imag());
        }
      }
      S.swap(W);
    }
  }

  pico_status st = PICO_OK;
#define TRY(x) \
  if ((st = (x)) != PICO_OK) return st;
  TRY(dalloc(c, &c->smaps, (size_t)nc * n));
  TRY(dalloc(c, &c->X, (size_t)B * n));
  TRY(dalloc(c, &c->R, (size_t)B * n));
  TRY(dalloc(c, &c->P, (size_t)B * n));
  TRY(dalloc(c, &c->Q, (size_t)B * n));
  TRY(dalloc(c, &c->rr_part, (size_t)B * (c->itmax + 1) * PB));
  TRY(dalloc(c, &c->pq_part, (size_t)B * c->itmax * PA));
  TRY(dalloc(c, &c->status, (size_t)B));
  TRY(dalloc(c, &c->d_iters, (size_t)B));
  TRY(dalloc(c, &c->cg_alpha, (size_t)B));
  TRY(dalloc(c, &c->cg_alpha2, (size_t)B));
  TRY(dalloc(c, &c->cg_state2, (size_t)B));
  if (const char* e = std::getenv("PICO_CG_PAIR_X")) c->pair_x = std::atoi(e) != 0;
  TRY(dalloc(c, &c->d_flag, (size_t)1));
  TRY(dalloc(c, &c->cg_done, (size_t)B));
  if (cudaMallocHost(&c->h_flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    c->h_flag = nullptr;  // no early stop: tolerance-stopped solves run all max_iter iterations
  }
  TRY(dalloc(c, &c->cg_state, (size_t)B));
  TRY(dalloc(c, &c->g_err, (size_t)4));  // first failure code of a bounded wait in any kernel
  cudaMemsetAsync(c->g_err, 0, 4 * sizeof(int), c->stream);
  TRY(dalloc(c, &c->d_relres, (size_t)B));
  TRY(dalloc(c, &c->d_norm, (size_t)PB + 1));
  cudaMemcpyAsync(c->smaps, S.empty() ? d->smaps : static_cast<const void*>(S.data()), (size_t)nc * n * sizeof(float2),
                  cudaMemcpyHostToDevice, c->stream);
  if (!Li_dev.empty()) {
    double2* li = nullptr;
    TRY(dalloc(c, &li, Li_dev.size()));
    cudaMemcpyAsync(li, Li_dev.data(), Li_dev.size() * sizeof(double2), cudaMemcpyHostToDevice, c->stream);
    { Launch L(c, 3); pico::launch_whiten(c->smaps, li, nc, n, c->stream); }
    // Li_dev lives on the host stack until the copy has run
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "pico_init whitening");
  }
  cudaMemsetAsync(c->status, 0, (size_t)B * sizeof(int), c->stream);
  if (!c->pa_gram) c->pa_fft = PA;
  c->cg = pico::CgArgs{n,     c->X,      c->R,     c->P,      c->Q,   c->rr_part, c->pq_part,
                       c->status, PB, c->pa_fft, c->itmax, 0.0, c->cg_done};

  if (c->mask2d) {
    TRY(cart2d_setup(c, d, img, P1, P2));
  } else if (c->kind == PICO_CARTESIAN) {
    TRY(dalloc(c, &c->ymul, (size_t)c->ny));
    TRY(dalloc(c, &c->tw, (size_t)c->ny));
    TRY(dalloc(c, &c->twx, (size_t)c->nx));
    TRY(dalloc(c, &c->mask, (size_t)c->ny));
    std::vector<float> ym(c->ny);
    for (int k = 0; k < c->ny; ++k) ym[k] = d->mask[k] ? (float)(1.0 / c->ny) : 0.f;
    const std::vector<float2> twy = twiddles(c->ny), twxv = twiddles(c->nx);
    cudaMemcpyAsync(c->ymul, ym.data(), ym.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->tw, twy.data(), twy.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->twx, twxv.data(), twxv.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->mask, d->mask, (size_t)c->ny, cudaMemcpyHostToDevice, c->stream);
    c->cop = pico::CartOp{c->ny, c->nx, nc, N1, N2, c->smaps, c->ymul, c->tw, c->mask, M1, M2, c->twx};
    c->gmask.assign(d->mask, d->mask + c->ny);
    // the host vectors above must outlive the asynchronous copies
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "pico_init upload");
  } else {
    TRY(spiral_setup(c, d, img, L, P1, P2, kbw));
  }

  // power method (Sec. 3.3): lambda_max of A^H A from a hash-drawn start vector
  c->lam_phys = c->lam_rel;
  if (c->power_iters > 0) {
    { Launch L(c, 3); pico::launch_fill_probe(c->X, n, kPowerSeed, 0, (float)(1.0 / std::sqrt((double)n)), c->stream); }
    for (int i = 0; i < c->power_iters; ++i) {
      op_apply(c, c->X, c->R, 1, 0.f);
      { Launch L(c, 3); pico::launch_norm2_part(c->R, n, c->d_norm + 1, c->stream); }
      { Launch L(c, 3); pico::launch_scale_by_norm(c->R, c->X, n, c->d_norm + 1, PB, c->d_norm, c->stream); }
    }
    double lmax = 0.0;
    cudaMemcpyAsync(&lmax, c->d_norm, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "pico_init power method");
    c->lambda_max = lmax;
    c->lam_phys = c->lam_rel * c->margin * lmax;
  }
  // the dense Gram operator takes over the CG normal operator once lambda_max is known
  if (!c->mask2d && c->kind == PICO_CARTESIAN && want_gram(d)) TRY(gram_setup(c, d));
  // small phase-encode images: every solve runs on chip, G_j in shared memory
  if (want_onchip(d)) {
    TRY(small_setup(c, true));
    c->onchip = true;
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "pico_init");
  if ((st = cuda_check(c, "pico_init")) != PICO_OK) return st;
#undef TRY
  return PICO_OK;
}

// Device bytes a context for `d` holds (the same sizes pico_init allocates);
// with_kbuf adds the k-space / grid buffer of PMR and the forward/adjoint calls.
size_t footprint_bytes(const pico_operator_desc* d, bool with_kbuf) {
  const int64_t B = d->max_batch > 0 ? d->max_batch : 64;
  const int64_t itmax = d->max_iter_cap > 0 ? d->max_iter_cap : 128;
  const int64_t nc = d->ncoils, n = (int64_t)d->ny * d->nx;
  const int64_t PB = (n + kVecPerBlock - 1) / kVecPerBlock;
  int64_t PA, extra, kbuf;
  if (d->kind == PICO_CARTESIAN && d->mask_2d) {
    PA = (d->ny + toep_row_lines() - 1) / toep_row_lines();
    extra = std::max(B * nc * n, n) * 8 + n * 5 + (int64_t)d->ny * 8;
    kbuf = B * nc * n * 8;
  } else if (d->kind == PICO_CARTESIAN) {
    PA = cart_normal_tiles(d->nx);
    extra = (int64_t)d->ny * 13 + (int64_t)d->nx * 8;
    kbuf = B * nc * n * 8;
    if (want_onchip(d)) extra += (int64_t)onchip_extra_bytes(d, B);
    if (want_gram(d)) {
      PA = std::max<int64_t>(PA, gram_pa(d->ny, d->nx));
      extra += (int64_t)gram_extra_bytes(d, B);
    }
  } else {
    const int64_t img = d->ny, L = 2 * img;
    PA = (img + toep_row_lines() - 1) / toep_row_lines();
    extra = std::max(B * nc * img * L, L * L) * 8 + L * L * 4 + img * 4 + L * 8 + d->nsamp * (56 + 88) +
            (L / 16) * (L / 16) * 4 + 64;
    kbuf = B * nc * 4 * n * 8;
  }
  const int64_t need = nc * n * 8 + nc * nc * 16 + 4 * B * n * 8 + B * (itmax + 1) * PB * 8 + B * itmax * PA * 8 + B * 16 +
                       PB * 8 + 64 + 16 + extra + (with_kbuf ? kbuf : 0);
  return (size_t)need;
}

}  // namespace pico

extern "C" {

pico_status pico_init(const pico_operator_desc* d, void* cuda_stream, size_t hbm_budget, pico_ctx** out) {
  return pico::init_impl(d, cuda_stream, hbm_budget, false, out);
}

pico_status pico_get_info(const pico_ctx* c, pico_info* info) {
  if (!c || !info) return PICO_E_INVALID;
  info->lambda_max = c->lambda_max;
  info->lambda_phys = c->lam_phys;
  info->kind = c->kind;
  info->ny = c->ny;
  info->nx = c->nx;
  info->ncoils = c->nc;
  info->max_batch = c->max_batch;
  info->max_iter_cap = c->itmax;
  info->nsamp = c->nsamp;
  info->device_bytes = c->device_bytes;
  info->normal_op = c->gram ? 1 : c->onchip ? 3 : (c->kind == PICO_CARTESIAN && !c->mask2d) ? 0 : 2;
  return PICO_OK;
}

pico_status pico_apply_normal(pico_ctx* c, const void* x, void* y, int32_t nbatch) {
  if (!c || !c->smaps) return PICO_E_INVALID;
  if (nbatch < 0 || (nbatch > 0 && (!x || !y))) return fail(c, PICO_E_INVALID, "bad batch or pointer");
  const bool gram = c->gram && std::min(nbatch, c->max_batch) >= c->gram_min_batch;
  const int chunk = c->kind == PICO_CARTESIAN && !gram ? 65535 : c->max_batch;
  for (int32_t b0 = 0; b0 < nbatch; b0 += chunk) {
    const int nb = std::min(chunk, nbatch - b0);
    const float2* xi = static_cast<const float2*>(x) + (size_t)b0 * c->n;
    float2* yo = static_cast<float2*>(y) + (size_t)b0 * c->n;
    select_path(c, nb);
    if (c->gram_on) {
      { Launch L(c, 3); pico::launch_to_cp(xi, cpf(c->R), c->ny, c->nx, nb, c->stream); }
      op_apply(c, c->R, c->Q, nb, (float)c->lam_phys);
      { Launch L(c, 3); pico::launch_from_cp(cpf(c->Q), yo, c->ny, c->nx, nb, c->stream); }
    } else {
      op_apply(c, xi, yo, nb, (float)c->lam_phys);
    }
  }
  return cuda_check(c, "pico_apply_normal");
}

pico_status pico_cg_batch(pico_ctx* c, const void* rhs, void* x, int32_t nbatch, int32_t max_iter, double rtol,
                          int32_t* iters_out, double* relres_out) {
  if (!c || !c->smaps) return PICO_E_INVALID;
  if (nbatch < 0 || (nbatch > 0 && (!rhs || !x))) return fail(c, PICO_E_INVALID, "bad batch or pointer");
  pico_status st = check_iter(c, max_iter, rtol);
  if (st != PICO_OK) return st;
  const size_t bytes_img = (size_t)c->n * sizeof(float2);
  for (int32_t b0 = 0; b0 < nbatch; b0 += c->max_batch) {
    const int nb = std::min(c->max_batch, nbatch - b0);
    const float2* rb = reinterpret_cast<const float2*>(static_cast<const char*>(rhs) + (size_t)b0 * bytes_img);
    float2* xb = reinterpret_cast<float2*>(static_cast<char*>(x) + (size_t)b0 * bytes_img);
    select_path(c, nb);
    if (c->gram_on) {
      Launch L(c, 3);
      pico::launch_to_cp(rb, cpf(c->R), c->ny, c->nx, nb, c->stream);
    } else {
      cudaMemcpyAsync(c->R, rb, (size_t)nb * bytes_img, cudaMemcpyDeviceToDevice, c->stream);
    }
    if ((st = run_cg(c, nb, max_iter, rtol, (float)c->lam_phys)) != PICO_OK) return st;
    if (c->gram_on) {
      Launch L(c, 3);
      pico::launch_from_cp(cpf(c->X), xb, c->ny, c->nx, nb, c->stream);
    } else {
      cudaMemcpyAsync(xb, c->X, (size_t)nb * bytes_img, cudaMemcpyDeviceToDevice, c->stream);
    }
    if (iters_out || relres_out) {
      if (column_mode(c) || small_path(c)) {
        Launch L(c, 3);
        pico::launch_colcg_report(col_args(c), c->nx, nb, c->d_iters, c->d_relres, c->stream);
      } else {
        Launch L(c, 3);
        pico::launch_cg_report(c->cg, nb, max_iter, c->d_iters, c->d_relres, c->stream);
      }
      std::vector<int> it(nb);
      std::vector<double> rr(nb);
      cudaMemcpyAsync(it.data(), c->d_iters, nb * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
      cudaMemcpyAsync(rr.data(), c->d_relres, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "pico_cg_batch");
      for (int i = 0; i < nb; ++i) {
        if (iters_out) iters_out[b0 + i] = it[i];
        if (relres_out) relres_out[b0 + i] = rr[i];
      }
    }
  }
  return cuda_check(c, "pico_cg_batch");
}

pico_status pico_variance_map(pico_ctx* c, uint64_t seed, int64_t probe_begin, int32_t nprobes, int32_t kind,
                              int32_t max_iter, double rtol, double* sum, double* sumsq, int32_t accumulate) {
  if (!c || !c->smaps) return PICO_E_INVALID;
  if (!sum || nprobes < 0 || probe_begin < 0) return fail(c, PICO_E_INVALID, "bad sum pointer or probe range");
  if (kind < 0 || kind > 2) return fail(c, PICO_E_INVALID, "unknown probe kind");
  pico_status st = check_iter(c, max_iter, rtol);
  if (st != PICO_OK) return st;
  if (!accumulate) {
    cudaMemsetAsync(sum, 0, (size_t)c->n * sizeof(double), c->stream);
    if (sumsq) cudaMemsetAsync(sumsq, 0, (size_t)c->n * sizeof(double), c->stream);
  }
  const float lam = (float)c->lam_phys;
  const int chunk = probe_chunk(c);
  for (int32_t b0 = 0; b0 < nprobes; b0 += chunk) {
    const int nb = std::min(chunk, nprobes - b0);
    select_path(c, nb);
    if ((st = run_cg_from_probe(c, nb, max_iter, rtol, lam, seed, probe_begin + b0, kind)) != PICO_OK) return st;
    if (c->lam_phys != 0.0) {
      // Sigma v = (M + lam)^-1 M (M + lam)^-1 v: apply M to the first solution, solve again
      op_apply(c, c->X, c->R, nb, 0.f);
      if ((st = run_cg(c, nb, max_iter, rtol, lam)) != PICO_OK) return st;
    }
    const float2* xs = c->X;
    if (c->gram_on) {  // back to the natural layout for the probe-indexed accumulation
      { Launch L(c, 3); pico::launch_from_cp(cpf(c->X), c->Q, c->ny, c->nx, nb, c->stream); }
      xs = c->Q;
    }
    { Launch L(c, 3); pico::launch_accum_pico(xs, c->n, nb, seed, probe_begin + b0, kind, sum, sumsq, c->stream); }
  }
  return cuda_check(c, "pico_variance_map");
}

pico_status pico_variance_map_adaptive(pico_ctx* c, uint64_t seed, int32_t probe_kind, int32_t chunk,
                                       int64_t max_probes, int32_t max_iter, double rtol, double target,
                                       double* sum, double* sumsq, int64_t* probes_used, double* rel_stderr) {
  if (!c || !c->smaps) return PICO_E_INVALID;
  if (!sum || !sumsq || !probes_used || chunk < 2 || max_probes < 2 || !(target > 0.0))
    return fail(c, PICO_E_INVALID, "adaptive map needs sum, sumsq, probes_used, chunk >= 2, target > 0");
  constexpr int kParts = 64;
  double* part = c->d_norm;  // PB + 1 >= 1 doubles; use a dedicated area below when too small
  pico_status st = PICO_OK;
  if (c->cg.PB + 1 < 2 * kParts) {
    if (!c->d_adapt && (st = dalloc(c, &c->d_adapt, (size_t)2 * kParts)) != PICO_OK) return st;
    part = c->d_adapt;
  }
  int64_t done = 0;
  double rel = INFINITY;
  std::vector<double> h(2 * kParts);
  while (done < max_probes) {
    const int32_t nb = (int32_t)std::min<int64_t>(chunk, max_probes - done);
    if ((st = pico_variance_map(c, seed, done, nb, probe_kind, max_iter, rtol, sum, sumsq, done > 0)) != PICO_OK)
      return st;
    done += nb;
    if (done < 2) continue;
    { Launch L(c, 3); pico::launch_stderr_parts(sum, sumsq, c->n, done, part, kParts, c->stream); }
    cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "pico_variance_map_adaptive");
    double a = 0.0, b = 0.0;
    for (int k = 0; k < kParts; ++k) {
      a += h[2 * k];
      b += h[2 * k + 1];
    }
    rel = a > 0.0 ? std::sqrt(b / a) : INFINITY;
    if (rel <= target) break;
  }
  *probes_used = done;
  if (rel_stderr) *rel_stderr = rel;
  return cuda_check(c, "pico_variance_map_adaptive");
}

pico_status pico_pmr(pico_ctx* c, uint64_t seed, int64_t rep_begin, int32_t nreps, double sigma, int32_t max_iter,
                     double rtol, double* sum, double* sumsq, int32_t accumulate) {
  if (!c || !c->smaps) return PICO_E_INVALID;
  if (!sum || nreps < 0 || rep_begin < 0) return fail(c, PICO_E_INVALID, "bad sum pointer or replica range");
  if (!(sigma > 0.0)) return fail(c, PICO_E_INVALID, "sigma must be > 0");
  if (c->kind == PICO_CARTESIAN && !c->mask2d && c->cop.M1 == 0)
    return fail(c, PICO_E_UNSUPPORTED, "nx has no FFT split in this build (PMR adjoint)");
  pico_status st = check_iter(c, max_iter, rtol);
  if (st != PICO_OK) return st;
  if ((st = ensure_kbuf(c)) != PICO_OK) return st;
  if (!accumulate) {
    cudaMemsetAsync(sum, 0, (size_t)c->n * sizeof(double), c->stream);
    if (sumsq) cudaMemsetAsync(sumsq, 0, (size_t)c->n * sizeof(double), c->stream);
  }
  const float lam = (float)c->lam_phys;
  const int chunk = probe_chunk(c);
  for (int32_t b0 = 0; b0 < nreps; b0 += chunk) {
    const int nb = std::min(chunk, nreps - b0);
    select_path(c, nb);
    if (c->gram_on) {
      noise_adjoint(c, c->Q, nb, seed, rep_begin + b0, sigma);
      { Launch L(c, 2); pico::launch_to_cp(c->Q, cpf(c->R), c->ny, c->nx, nb, c->stream); }
    } else {
      noise_adjoint(c, c->R, nb, seed, rep_begin + b0, sigma);
    }
    if ((st = run_cg(c, nb, max_iter, rtol, lam)) != PICO_OK) return st;
    const float2* xs = c->X;
    if (c->gram_on) {
      { Launch L(c, 3); pico::launch_from_cp(cpf(c->X), c->Q, c->ny, c->nx, nb, c->stream); }
      xs = c->Q;
    }
    { Launch L(c, 3); pico::launch_accum_pmr(xs, c->n, nb, (float)(1.0 / (sigma * sigma)), sum, sumsq, c->stream); }
  }
  return cuda_check(c, "pico_pmr");
}

pico_status pico_forward(pico_ctx* c, const void* x, void* y, int32_t nbatch) {
  if (!c || !c->smaps) return PICO_E_INVALID;
  if (nbatch < 0 || (nbatch > 0 && (!x || !y))) return fail(c, PICO_E_INVALID, "bad batch or pointer");
  const float2* xi = static_cast<const float2*>(x);
  float2* yo = static_cast<float2*>(y);
  pico_status st = PICO_OK;
  if (c->kind == PICO_CARTESIAN) {
    if (!pico::fft_length_supported(c->nx) || !pico::fft_length_supported(c->ny))
      return fail(c, PICO_E_UNSUPPORTED, "nx or ny has no FFT split in this build (forward operator)");
    const int chunk = std::max(1, 65535 / c->nc);
    const float scale = (float)(1.0 / std::sqrt((double)c->n));
    for (int32_t b0 = 0; b0 < nbatch; b0 += chunk) {
      const int nb = std::min(chunk, nbatch - b0);
      float2* yb = yo + (size_t)b0 * c->nc * c->n;
      { Launch L(c, 3); pico::launch_cart_smul(xi + (size_t)b0 * c->n, c->smaps, yb, nb, c->nc, c->n, c->stream); }
      { Launch L(c, 3); pico::launch_fft_rows(c->nx, yb, c->twx, c->ny, nb * c->nc, c->n, -1, c->stream); }
      { Launch L(c, 3); pico::launch_fft_cols(c->ny, yb, c->tw, c->nx, nb * c->nc, c->n, -1, c->stream); }
      if (c->mask2d) {
        Launch L(c, 3);
        pico::launch_mask2d(yb, yb, c->mask, scale, c->n, nb * c->nc, c->stream);
      } else {
        Launch L(c, 3);
        pico::launch_cart_mask_scale(yb, c->mask, nb * c->nc, c->ny, c->nx, scale, c->stream);
      }
    }
  } else {
    if ((st = ensure_kbuf(c)) != PICO_OK) return st;
    const int L = c->sop.L;
    for (int32_t b0 = 0; b0 < nbatch; b0 += c->max_batch) {
      const int nb = std::min(c->max_batch, nbatch - b0);
      { Launch Lk(c, 3); pico::launch_spiral_pad(c->sop, xi + (size_t)b0 * c->n, c->G, nb, c->stream); }
      { Launch Lk(c, 3); pico::launch_fft_rows(L, c->G, c->tw2, L, nb * c->nc, (int64_t)L * L, -1, c->stream); }
      { Launch Lk(c, 3); pico::launch_fft_cols(L, c->G, c->tw2, L, nb * c->nc, (int64_t)L * L, -1, c->stream); }
      { Launch Lk(c, 3); pico::launch_nufft_interp(c->sop, c->G, yo + (size_t)b0 * c->nc * c->nsamp, nb, c->stream); }
    }
  }
  return cuda_check(c, "pico_forward");
}

pico_status pico_adjoint(pico_ctx* c, const void* y, void* x, int32_t nbatch) {
  if (!c || !c->smaps) return PICO_E_INVALID;
  if (nbatch < 0 || (nbatch > 0 && (!x || !y))) return fail(c, PICO_E_INVALID, "bad batch or pointer");
  if (c->kind == PICO_CARTESIAN && !c->mask2d && c->cop.M1 == 0)
    return fail(c, PICO_E_UNSUPPORTED, "nx has no FFT split in this build (adjoint operator)");
  pico_status st = ensure_kbuf(c);
  if (st != PICO_OK) return st;
  const float2* yi = static_cast<const float2*>(y);
  float2* xo = static_cast<float2*>(x);
  const int64_t kper = c->kind == PICO_CARTESIAN ? c->n : c->nsamp;
  for (int32_t b0 = 0; b0 < nbatch; b0 += c->max_batch) {
    const int nb = std::min(c->max_batch, nbatch - b0);
    const float2* yb = yi + (size_t)b0 * c->nc * kper;
    if (c->mask2d) {
      { Launch L(c, 3); pico::launch_mask2d(yb, c->G, c->mask, (float)(1.0 / std::sqrt((double)c->n)), c->n,
                                            nb * c->nc, c->stream); }
      adjoint2d_from_kbuf(c, xo + (size_t)b0 * c->n, nb);
    } else if (c->kind == PICO_CARTESIAN) {
      { Launch L(c, 3); pico::launch_cart_pmr_cols(c->cop, c->G, nb, 0, 0, 0.f, c->stream, yb); }
      { Launch L(c, 3); pico::launch_cart_rows_adjoint(c->cop, c->G, xo + (size_t)b0 * c->n, nb, c->stream); }
    } else {
      { Launch L(c, 3); pico::launch_grid_pmr(c->sop, c->G, nb, 0, 0, 0.f, c->stream, yb); }
      { Launch L(c, 3, 2); pico::launch_grid_adjoint_rest(c->sop, c->G, xo + (size_t)b0 * c->n, nb, c->stream); }
    }
  }
  return cuda_check(c, "pico_adjoint");
}

pico_status pico_cs_recon(pico_ctx* c, const void* b_dev, double lambda_l1, int32_t iters, int32_t levels,
                          void* x_dev) {
  if (!c || !c->smaps) return PICO_E_INVALID;
  if (!b_dev || !x_dev || iters < 1 || levels < 1 || !(lambda_l1 >= 0.0))
    return fail(c, PICO_E_INVALID, "bad CS reconstruction arguments");
  pico_status st = wavelet_check(c, levels);
  if (st != PICO_OK) return st;
  if (!(c->lambda_max > 0.0)) return fail(c, PICO_E_INVALID, "CS needs the power-method lambda_max (power_iters > 0)");
  if ((st = cs_buffers(c)) != PICO_OK) return st;
  select_path(c, 0);  // the CS iterations keep images in the natural layout
  if (c->cs_traj_cap < iters) {
    if ((st = dalloc(c, &c->cs_traj, (size_t)iters * c->n)) != PICO_OK) return st;
    c->cs_traj_cap = iters;
  }
  c->cs_iters = iters;
  c->cs_levels = levels;
  c->cs_lam = lambda_l1;
  c->cs_lc = c->margin * c->lambda_max;
  c->cs_tau = lambda_l1 / c->cs_lc;
  c->cs_c.assign(iters, 0.f);
  double t = 1.0;
  for (int k = 0; k < iters; ++k) {
    const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
    c->cs_c[k] = (float)((t - 1.0) / tn);
    t = tn;
  }
  ++c->cs_generation;  // the stored linearisation point is replaced from here on
  if ((st = pico_adjoint(c, b_dev, c->cs_ahb, 1)) != PICO_OK) return st;
  cs_fista(c, c->cs_ahb, 0, 1, true);
  cudaMemcpyAsync(c->cs_x0, cs_e(c, 0), (size_t)c->n * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(x_dev, cs_e(c, 0), (size_t)c->n * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream);
  c->cs_ready = true;
  return cuda_check(c, "pico_cs_recon");
}

pico_status pico_cs_pmr(pico_ctx* c, uint64_t seed, int64_t rep_begin, int32_t nreps, double sigma, double* sum,
                        double* sumsq, int32_t accumulate) {
  pico_status st = cs_check(c);
  if (st != PICO_OK) return st;
  if (!sum || nreps < 0 || rep_begin < 0) return fail(c, PICO_E_INVALID, "bad sum pointer or replica range");
  if (!(sigma > 0.0)) return fail(c, PICO_E_INVALID, "sigma must be > 0");
  if (c->kind == PICO_CARTESIAN && !c->mask2d && c->cop.M1 == 0)
    return fail(c, PICO_E_UNSUPPORTED, "nx has no FFT split in this build (PMR adjoint)");
  if ((st = ensure_kbuf(c)) != PICO_OK) return st;
  if (!accumulate) {
    cudaMemsetAsync(sum, 0, (size_t)c->n * sizeof(double), c->stream);
    if (sumsq) cudaMemsetAsync(sumsq, 0, (size_t)c->n * sizeof(double), c->stream);
  }
  for (int32_t b0 = 0; b0 < nreps; b0 += c->max_batch) {
    const int nb = std::min(c->max_batch, nreps - b0);
    noise_adjoint(c, c->R, nb, seed, rep_begin + b0, sigma);                           // A^H n_i
    { Launch L(c, 3); pico::launch_axpy_bcast(c->R, c->cs_ahb, 1.f, c->n, nb, c->stream); }  // A^H (b + n_i)
    cs_fista(c, c->R, c->n, nb, false);                                               // f(b + n_i)
    { Launch L(c, 3); pico::launch_axpy_bcast(cs_e(c, 0), c->cs_x0, -1.f, c->n, nb, c->stream); }
    { Launch L(c, 3); pico::launch_accum_pmr(cs_e(c, 0), c->n, nb, (float)(1.0 / (sigma * sigma)), sum, sumsq,
                                             c->stream); }
  }
  return cuda_check(c, "pico_cs_pmr");
}

pico_status pico_wavelet(pico_ctx* c, const void* in_dev, void* out_dev, int32_t nbatch, int32_t levels,
                         int32_t inverse) {
  if (!c || !c->smaps) return PICO_E_INVALID;
  if (nbatch < 0 || (nbatch > 0 && (!in_dev || !out_dev)) || levels < 1)
    return fail(c, PICO_E_INVALID, "bad batch, pointer or level count");
  pico_status st = wavelet_check(c, levels);
  if (st != PICO_OK) return st;
  if ((st = cs_buffers(c)) != PICO_OK) return st;
  const float2* in = static_cast<const float2*>(in_dev);
  float2* out = static_cast<float2*>(out_dev);
  for (int32_t b0 = 0; b0 < nbatch; b0 += c->max_batch) {
    const int nb = std::min(c->max_batch, nbatch - b0);
    const size_t off = (size_t)b0 * c->n;
    if (inverse) cs_WH(c, in + off, out + off, cs_e(c, 2), nb, levels);
    else cs_W(c, in + off, out + off, cs_e(c, 2), nb, levels);
  }
  return cuda_check(c, "pico_wavelet");
}

pico_status pico_cs_jvp(pico_ctx* c, const void* db_dev, void* dx_dev, int32_t nbatch) {
  pico_status st = cs_check(c);
  if (st != PICO_OK) return st;
  if (nbatch < 0 || (nbatch > 0 && (!db_dev || !dx_dev))) return fail(c, PICO_E_INVALID, "bad batch or pointer");
  const int64_t kper = c->kind == PICO_CARTESIAN ? (int64_t)c->nc * c->n : (int64_t)c->nc * c->nsamp;
  for (int32_t b0 = 0; b0 < nbatch; b0 += c->max_batch) {
    const int nb = std::min(c->max_batch, nbatch - b0);
    if ((st = pico_adjoint(c, static_cast<const float2*>(db_dev) + (size_t)b0 * kper, c->Q, nb)) != PICO_OK)
      return st;
    cs_jvp_core(c, c->Q, nb);
    cudaMemcpyAsync(static_cast<float2*>(dx_dev) + (size_t)b0 * c->n, cs_e(c, 0), (size_t)nb * c->n * sizeof(float2),
                    cudaMemcpyDeviceToDevice, c->stream);
  }
  return cuda_check(c, "pico_cs_jvp");
}

pico_status pico_cs_vjp(pico_ctx* c, const void* xbar_dev, void* bbar_dev, int32_t nbatch) {
  pico_status st = cs_check(c);
  if (st != PICO_OK) return st;
  if (nbatch < 0 || (nbatch > 0 && (!xbar_dev || !bbar_dev))) return fail(c, PICO_E_INVALID, "bad batch or pointer");
  const int64_t kper = c->kind == PICO_CARTESIAN ? (int64_t)c->nc * c->n : (int64_t)c->nc * c->nsamp;
  for (int32_t b0 = 0; b0 < nbatch; b0 += c->max_batch) {
    const int nb = std::min(c->max_batch, nbatch - b0);
    cs_vjp_core(c, static_cast<const float2*>(xbar_dev) + (size_t)b0 * c->n, nb);
    if ((st = pico_forward(c, cs_e(c, 0), static_cast<float2*>(bbar_dev) + (size_t)b0 * kper, nb)) != PICO_OK)
      return st;
  }
  return cuda_check(c, "pico_cs_vjp");
}

pico_status pico_cs_variance_map(pico_ctx* c, uint64_t seed, int64_t probe_begin, int32_t nprobes, int32_t kind,
                                 double* sum, double* sumsq, int32_t accumulate) {
  pico_status st = cs_check(c);
  if (st != PICO_OK) return st;
  if (!sum || nprobes < 0 || probe_begin < 0 || kind < 0 || kind > 2)
    return fail(c, PICO_E_INVALID, "bad sum pointer, probe range or kind");
  if (!accumulate) {
    cudaMemsetAsync(sum, 0, (size_t)c->n * sizeof(double), c->stream);
    if (sumsq) cudaMemsetAsync(sumsq, 0, (size_t)c->n * sizeof(double), c->stream);
  }
  for (int32_t b0 = 0; b0 < nprobes; b0 += c->max_batch) {
    const int nb = std::min(c->max_batch, nprobes - b0);
    { Launch L(c, 1); pico::launch_cg_init_probe(c->cg, nb, seed, probe_begin + b0, kind, c->stream); }
    cs_vjp_core(c, c->R, nb);                   // E0 = J^T v  (as the image-domain A^H-side vector / Lc sum)
    op_apply(c, cs_e(c, 0), c->Q, nb, 0.f);     // A^H (A g) = M g: the tangent J needs, without k-space
    cs_jvp_core(c, c->Q, nb);                   // E0 = J J^T v
    { Launch L(c, 3); pico::launch_accum_pico(cs_e(c, 0), c->n, nb, seed, probe_begin + b0, kind, sum, sumsq,
                                              c->stream); }
  }
  return cuda_check(c, "pico_cs_variance_map");
}

pico_status pico_finalize(pico_ctx* c, const double* sum, const double* sumsq, int64_t count, float* var,
                          float* se) {
  if (!c || !sum || count <= 0) return c ? fail(c, PICO_E_INVALID, "bad finalize arguments") : PICO_E_INVALID;
  if (se && !sumsq) return fail(c, PICO_E_INVALID, "stderr needs sumsq");
  { Launch L(c, 3); pico::launch_finalize(sum, sumsq, c->n, count, var, se, c->stream); }
  return cuda_check(c, "pico_finalize");
}

pico_status pico_gfactor(pico_ctx* c, const float* va, const float* vr, double R, float* g) {
  if (!c || !va || !vr || !g || !(R > 0)) return c ? fail(c, PICO_E_INVALID, "bad gfactor arguments") : PICO_E_INVALID;
  { Launch L(c, 3); pico::launch_gfactor(va, vr, c->n, R, g, c->stream); }
  return cuda_check(c, "pico_gfactor");
}

pico_status pico_sync(pico_ctx* c) {
  if (!c) return PICO_E_INVALID;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "pico_sync");
  // read and clear the asynchronous status words on the context stream, then
  // report every class that is pending (a timeout ranks before a breakdown)
  int e = 0;
  std::vector<int> s;
  if (c->g_err && cudaMemcpyAsync(&e, c->g_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return cuda_check(c, "pico_sync");
  if (c->status) {
    s.assign(c->max_batch, 0);
    if (cudaMemcpyAsync(s.data(), c->status, s.size() * sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
        cudaSuccess)
      return cuda_check(c, "pico_sync");
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "pico_sync");
  int broken = 0;
  for (int v : s) broken += v != 0;
  if (e) cudaMemsetAsync(c->g_err, 0, sizeof(int), c->stream);
  if (broken) cudaMemsetAsync(c->status, 0, s.size() * sizeof(int), c->stream);
  if ((e || broken) && cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "pico_sync");
  std::string msg;
  if (e) msg = "a kernel's bounded pipeline wait timed out (code " + std::to_string(e) + ")";
  if (broken) {
    if (!msg.empty()) msg += "; ";
    msg += "CG breakdown (non-finite residual or p^H (M + lam) p <= 0) in " + std::to_string(broken) +
           " system(s) of the last batch";
  }
  if (e) return fail(c, PICO_E_TIMEOUT, msg);
  if (broken) return fail(c, PICO_E_BREAKDOWN, msg);
  return cuda_check(c, "pico_sync");
}

pico_status pico_set_solver(pico_ctx* c, int32_t solver) {
  if (!c || !c->smaps) return PICO_E_INVALID;
  if (solver != PICO_SOLVER_GLOBAL && solver != PICO_SOLVER_COLUMNS)
    return fail(c, PICO_E_INVALID, "solver must be PICO_SOLVER_GLOBAL or PICO_SOLVER_COLUMNS");
  if (solver == PICO_SOLVER_COLUMNS) {
    const bool phase_encode = c->kind == PICO_CARTESIAN && !c->mask2d && !c->gmask.empty();
    const bool small = phase_encode && !c->gram && pico::colcg_small_supported(c->ny);
    if (!small && (!c->gram || !pico::gram_colcg_supported(c->ny, c->nx)))
      return fail(c, PICO_E_UNSUPPORTED,
                  "per-column CG needs a Cartesian phase-encode context with ny = 32, 64 or 96, or one on the "
                  "tensor-core operator whose row tile is a multiple of 32 and at most 4 tiles per column");
    if (small) {
      const pico_status st = small_setup(c, false);
      if (st != PICO_OK) return st;
    }
    c->col_small = small;
    const size_t n = (size_t)c->max_batch * c->nx;
    pico_status st = PICO_OK;
    if ((!c->col_rr0 && (st = dalloc(c, &c->col_rr0, n)) != PICO_OK) ||
        (!c->col_rr && (st = dalloc(c, &c->col_rr, n)) != PICO_OK) ||
        (!c->col_beta && (st = dalloc(c, &c->col_beta, n)) != PICO_OK) ||
        (!c->col_done && (st = dalloc(c, &c->col_done, n)) != PICO_OK) ||
        (!c->col_iters && (st = dalloc(c, &c->col_iters, n)) != PICO_OK) ||
        (!c->col_pn && (st = dalloc(c, &c->col_pn, n)) != PICO_OK) ||
        (!c->col_pscale && (st = dalloc(c, &c->col_pscale, n)) != PICO_OK))
      return st;
  }
  clear_graphs(c);
  c->solver = solver;
  return cuda_check(c, "pico_set_solver");
}

pico_status pico_get_solver(const pico_ctx* c, int32_t* solver) {
  if (!c || !solver) return PICO_E_INVALID;
  *solver = c->solver;
  return PICO_OK;
}

pico_status pico_inject_error(pico_ctx* c, int32_t cls, int32_t code) {
  if (!c || !c->smaps || (cls != PICO_E_TIMEOUT && cls != PICO_E_BREAKDOWN) || code == 0)
    return c ? fail(c, PICO_E_INVALID, "inject PICO_E_TIMEOUT or PICO_E_BREAKDOWN with a nonzero code")
             : PICO_E_INVALID;
  int* word = cls == PICO_E_TIMEOUT ? c->g_err : c->status;
  if (!word) return fail(c, PICO_E_INVALID, "no status word of that class");
  if (cudaMemcpyAsync(word, &code, sizeof(int), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return cuda_check(c, "pico_inject_error");
  return PICO_OK;
}

pico_status pico_cs_generation(const pico_ctx* c, int64_t* generation) {
  if (!c || !generation) return PICO_E_INVALID;
  *generation = c->cs_generation;
  return PICO_OK;
}

pico_status pico_profile(pico_ctx* c, int32_t enable) {
  if (!c) return PICO_E_INVALID;
  prof_collect(c);
  if (enable) {
    for (int k = 0; k < 4; ++k) {
      c->prof_ms[k] = 0;
      c->prof_n[k] = 0;
    }
  }
  c->profiling = enable != 0;
  return cuda_check(c, "pico_profile");
}

pico_status pico_profile_read(pico_ctx* c, int32_t cls, double* total_ms, int64_t* launches) {
  if (!c || cls < 0 || cls > 3) return PICO_E_INVALID;
  prof_collect(c);
  if (total_ms) *total_ms = c->prof_ms[cls];
  if (launches) *launches = c->prof_n[cls];
  return cuda_check(c, "pico_profile_read");
}

pico_status pico_launch_count(pico_ctx* c, int64_t* count, int32_t reset) {
  if (!c || !count) return PICO_E_INVALID;
  *count = c->launches;
  if (reset) c->launches = 0;
  return PICO_OK;
}

pico_status pico_get_tuning(const pico_ctx* c, pico_tuning* out) {
  if (!c || !out) return PICO_E_INVALID;
  out->gram_min_batch = c->gram_min_batch;
  out->gram_kc = c->gop.kc ? c->gop.kc : 16;
  out->gram_a_tmem = c->gop.a_tmem;
  out->probe_batch = c->probe_batch;
  return PICO_OK;
}

pico_status pico_set_tuning(pico_ctx* c, const pico_tuning* t) {
  if (!c || !c->smaps || !t) return PICO_E_INVALID;
  if (t->gram_min_batch < 0 || !(t->gram_kc == 0 || t->gram_kc == 8 || t->gram_kc == 16) ||
      !(t->gram_a_tmem == 0 || t->gram_a_tmem == 1) || t->probe_batch < 0 || t->probe_batch > c->max_batch)
    return fail(c, PICO_E_INVALID, "tuning out of range (gram_kc 8/16, gram_a_tmem 0/1, probe_batch <= max_batch)");
  clear_graphs(c);
  if (t->gram_min_batch > 0) c->gram_min_batch = t->gram_min_batch;
  const bool rebuild = (t->gram_kc != 0 && t->gram_kc != c->gop.kc) || t->gram_a_tmem != c->gop.a_tmem;
  c->gop.a_tmem = t->gram_a_tmem;
  c->probe_batch = t->probe_batch;
  if (t->gram_kc != 0) c->gop.kc = t->gram_kc;
  if (rebuild && c->gram) return gram_configure(c);  // G's operand format follows (kc, a_tmem)
  return cuda_check(c, "pico_set_tuning");
}

pico_status pico_autotune(pico_ctx* c, int32_t iters, pico_tuning* out, double* times_us, int32_t ntimes) {
  if (!c || !c->smaps) return PICO_E_INVALID;
  if (c->onchip) {  // the on-chip solve has no launch shape to choose: report the current tuning
    if (times_us)
      for (int i = 0; i < ntimes; ++i) times_us[i] = NAN;
    if (out) pico_get_tuning(c, out);
    return PICO_OK;
  }
  if (iters == 0) iters = 4;
  if (iters < 2 || iters > 32 || iters > c->itmax) return fail(c, PICO_E_INVALID, "autotune iters must be 2..32");
  constexpr int kCand = 4, kNb = 6;
  const int cand_kc[kCand] = {0, 16, 16, 8}, cand_at[kCand] = {0, 0, 1, 0};
  int nbs[kNb] = {16, 32, 64, 128, 256, c->max_batch};
  bool nb_ok[kNb];
  for (int i = 0; i < kNb; ++i) {
    nb_ok[i] = nbs[i] <= c->max_batch;
    for (int k = 0; k < i; ++k) nb_ok[i] = nb_ok[i] && nbs[k] != nbs[i];
  }
  double t[kCand][kNb];
  for (auto& row : t)
    for (double& v : row) v = NAN;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_check(c, "pico_autotune");
  }
  const float lam = (float)c->lam_phys;
  const bool prof = c->profiling;
  const int solver = c->solver;
  c->profiling = false;
  c->solver = PICO_SOLVER_GLOBAL;  // the tuning is measured on the whole-image CG
  c->cg.rtol2 = 0.0;
  // us per image and iteration of `iters` CG iterations on nb probes: the
  // first run launches directly, the second captures the graph, the best of
  // the next two replays counts
  auto time_cg = [&](int nb, bool gram) -> double {
    c->gram_on = gram;
    c->cg.PA = gram ? c->pa_gram : c->pa_fft;
    float best = INFINITY;
    for (int rep = 0; rep < 4; ++rep) {
      init_from_probe(c, nb, 0x7a11ull, 0, PICO_PROBE_PHASE);
      cudaEventRecord(e0, c->stream);
      cg_range(c, nb, 0, iters, 0.0, lam);
      cudaEventRecord(e1, c->stream);
      float ms = INFINITY;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        return (double)NAN;
      if (rep >= 2) best = std::min(best, ms);
    }
    return 1e3 * (double)best / ((double)nb * iters);
  };
  pico_tuning cur{};
  pico_get_tuning(c, &cur);
  pico_status st = PICO_OK;
  for (int k = 0; k < kCand && st == PICO_OK; ++k) {
    if (k > 0) {
      if (!c->gram) break;
      clear_graphs(c);
      if (c->gop.kc != cand_kc[k] || c->gop.a_tmem != cand_at[k]) {
        c->gop.a_tmem = cand_at[k];
        c->gop.kc = cand_kc[k];
        if ((st = gram_configure(c)) != PICO_OK) break;
      }
    }
    for (int i = 0; i < kNb; ++i)
      if (nb_ok[i]) t[k][i] = time_cg(nbs[i], k > 0);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->profiling = prof;
  c->solver = solver;
  if (st != PICO_OK) return st;
  if ((st = cuda_check(c, "pico_autotune")) != PICO_OK) return st;
  double flat[kCand * kNb];
  for (int k = 0; k < kCand; ++k)
    for (int i = 0; i < kNb; ++i) flat[k * kNb + i] = t[k][i];
  pico_tuning best{};
  if ((st = pico_tune_select(flat, c->max_batch, c->gram ? 1 : 0, &best)) != PICO_OK)
    return fail(c, st, "no candidate could be timed");
  if (!c->gram) {  // nothing to choose for the Gram operator: keep its settings
    best.gram_min_batch = cur.gram_min_batch;
    best.gram_a_tmem = cur.gram_a_tmem;
  }
  if (times_us)
    for (int k = 0; k < kCand; ++k)
      for (int i = 0; i < kNb; ++i)
        if (k * kNb + i < ntimes) times_us[k * kNb + i] = t[k][i];
  if ((st = pico_set_tuning(c, &best)) != PICO_OK) return st;
  if (out) pico_get_tuning(c, out);
  return PICO_OK;
}

pico_status pico_tune_select(const double* t, int32_t max_batch, int32_t gram, pico_tuning* out) {
  if (!t || !out || max_batch < 1) return PICO_E_INVALID;
  constexpr int kCand = 4, kNb = 6;
  const int cand_kc[kCand] = {0, 16, 16, 8}, cand_at[kCand] = {0, 0, 1, 0};
  const int nbs[kNb] = {16, 32, 64, 128, 256, max_batch};
  bool ok[kNb];
  for (int i = 0; i < kNb; ++i) {
    ok[i] = nbs[i] <= max_batch && std::isfinite(t[i]);
    for (int k = 0; k < i; ++k) ok[i] = ok[i] && nbs[k] != nbs[i];
  }
  int top = -1;  // largest batch the column-FFT / Toeplitz operator was timed at
  for (int i = 0; i < kNb; ++i)
    if (ok[i] && (top < 0 || nbs[i] > nbs[top])) top = i;
  if (top < 0) return PICO_E_INVALID;
  pico_tuning best{};
  best.gram_min_batch = max_batch + 1;
  best.gram_kc = 0;
  best.gram_a_tmem = 0;
  int vg = 0;  // Gram candidate: the fastest at the largest batch
  if (gram)
    for (int k = 1; k < kCand; ++k)
      if (std::isfinite(t[k * kNb + top]) && (vg == 0 || t[k * kNb + top] < t[vg * kNb + top])) vg = k;
  if (vg) {
    best.gram_kc = cand_kc[vg];
    best.gram_a_tmem = cand_at[vg];
    // the smallest batch from which on the Gram operator is never slower
    int order[kNb], no = 0;
    for (int i = 0; i < kNb; ++i)
      if (ok[i]) order[no++] = i;
    std::sort(order, order + no, [&](int a, int b) { return nbs[a] > nbs[b]; });
    for (int j = 0; j < no; ++j) {
      const int i = order[j];
      if (!(t[vg * kNb + i] <= t[i])) break;
      best.gram_min_batch = nbs[i];
    }
  }
  auto chosen = [&](int i) { return (vg && nbs[i] >= best.gram_min_batch) ? t[vg * kNb + i] : t[i]; };
  // the largest batch within 3 % of the lowest time per image
  double tmin = INFINITY;
  for (int i = 0; i < kNb; ++i)
    if (ok[i] && std::isfinite(chosen(i))) tmin = std::min(tmin, chosen(i));
  int pb = -1;
  for (int i = 0; i < kNb; ++i)
    if (ok[i] && chosen(i) <= 1.03 * tmin && (pb < 0 || nbs[i] > nbs[pb])) pb = i;
  best.probe_batch = (pb >= 0 && nbs[pb] < max_batch) ? nbs[pb] : 0;
  *out = best;
  return PICO_OK;
}

const char* pico_last_error(const pico_ctx* c) { return c ? c->err.c_str() : "null context"; }

void pico_destroy(pico_ctx* c) {
  if (!c) return;
  if (!c->allocs.empty()) cudaStreamSynchronize(c->stream);
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.first);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->h_flag) cudaFreeHost(c->h_flag);
  for (void* p : c->allocs) {
    if (c->async_alloc)
      cudaFreeAsync(p, c->stream);
    else
      cudaFree(p);
  }
  delete c;
}

}  // extern "C"
