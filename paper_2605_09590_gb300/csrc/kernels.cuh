// Kernel launch interface shared by the C-ABI layer (api.cu) and the kernel
// translation units.  Host-side only declarations; no torch types anywhere.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pico {

// Threads and complex elements per block of the streaming vector kernels.
constexpr int kVecThreads = 256;
constexpr int kVecPerThread = 4;
constexpr int kVecPerBlock = kVecThreads * kVecPerThread;

// Batched CG state (Eq. 6 solved for many right-hand sides at once).
// Scalars are kept per iteration so that every value is written once:
// rr(b, it) = sum_j rr_part[(b*(itmax+1) + it)*PB + j]   (r^H r before update it)
// pq(b, it) = sum_j pq_part[(b*itmax + it)*PA + j]        (p^H (M+lam) p of update it)
struct CgArgs {
  int64_t n;         // voxels per image
  float2* X;         // [B][n] solution
  float2* R;         // [B][n] residual (holds the right-hand side before init)
  float2* P;         // [B][n] search direction
  float2* Q;         // [B][n] (M + lam) P
  double* rr_part;   // [B][itmax+1][PB]
  double* pq_part;   // [B][itmax][PA]
  int* status;       // [B] 0 ok, 5 breakdown
  int PB, PA, itmax;
  double rtol2;      // squared relative residual tolerance
  int* done;         // [B] or nullptr: stop flag of the current iteration, written by the
                     // first pass of the Toeplitz operator for the passes after it
};

// ---- encode.cu: pre-whitening of the sensitivities (Eq. 3) ----
constexpr int kWhitenMaxCoils = 64;
// S[c][v] <- sum_{k <= c} Li[c][k] S[k][v] in place, Li lower-triangular nc x nc (FP64)
void launch_whiten(float2* S, const double2* Li, int nc, int64_t n, cudaStream_t s);

// ---- cg.cu ----
void launch_cg_init_probe(const CgArgs& a, int nb, uint64_t seed, int64_t probe_begin, int kind, cudaStream_t s);
void launch_cg_init_rhs(const CgArgs& a, int nb, cudaStream_t s);
void launch_cg_update(const CgArgs& a, int nb, int it, cudaStream_t s);
// the same update as launch_cg_update with the per-system scalars computed once
// (two launches, 16-byte accesses); false (nothing launched) when n is odd
bool launch_cg_step(const CgArgs& a, int nb, int it, float* alpha, int* state, cudaStream_t s);
// The same with x advanced once per two iterations (operators that keep the
// previous direction p_prev intact through iteration it): even it updates r,
// odd it applies the pending x update of it - 1 and its own; alpha / state
// of it - 1 in alpha_prev / state_prev.  launch_cg_flush_pair applies a
// pending x update after a solve that ended on an even iteration.
bool launch_cg_step_pair(const CgArgs& a, int nb, int it, float* alpha, int* state, const float* alpha_prev,
                         const int* state_prev, const float2* p_prev, cudaStream_t s);
void launch_cg_flush_pair(const CgArgs& a, int nb, const float* alpha_prev, const int* state_prev,
                          const float2* p_prev, cudaStream_t s);
void launch_cg_report(const CgArgs& a, int nb, int max_iter, int* iters, double* relres, cudaStream_t s);
// *flag (device) != 0 iff every one of the nb systems has stopped at iteration it
void launch_cg_all_done(const CgArgs& a, int nb, int it, int* flag, cudaStream_t s);
void launch_accum_pico(const float2* X, int64_t n, int nb, uint64_t seed, int64_t probe_begin, int kind,
                       double* sum, double* sumsq, cudaStream_t s);
void launch_accum_pmr(const float2* X, int64_t n, int nb, float inv_sigma2, double* sum, double* sumsq,
                      cudaStream_t s);
void launch_finalize(const double* sum, const double* sumsq, int64_t n, int64_t count, float* var,
                     float* stderr_out, cudaStream_t s);
void launch_gfactor(const float* var_acc, const float* var_ref, int64_t n, double R, float* g, cudaStream_t s);
// per-block partials (sum of mean^2, sum of stderr^2) of running PICO sums over `count` probes
void launch_stderr_parts(const double* sum, const double* sumsq, int64_t n, int64_t count, double* part, int nblk,
                         cudaStream_t s);
void launch_norm2_part(const float2* x, int64_t n, double* part, cudaStream_t s);
void launch_scale_by_norm(const float2* y, float2* x, int64_t n, const double* part, int nparts,
                          double* norm_out, cudaStream_t s);
void launch_fill_probe(float2* x, int64_t n, uint64_t seed, int64_t index, float scale, cudaStream_t s);
void launch_copy_scaled(const float2* in, float2* out, int64_t n, cudaStream_t s);

// ---- cart.cu: Cartesian column-decoupled operators ----
struct CartOp {
  int ny, nx, nc;
  int N1, N2;               // ny = N1 * N2 split of the column FFT
  const float2* smaps;      // [nc][ny][nx] whitened sensitivities
  const float* ymul;        // [ny] mask(ky) / ny
  const float2* tw;         // [ny] exp(-2 pi i e / ny)
  const uint8_t* mask;      // [ny]
  // row transform for the PMR adjoint (length nx)
  int M1, M2;               // nx = M1 * M2
  const float2* twx;        // [nx] exp(-2 pi i e / nx)
};
bool cart_supported(int ny, int nx, int* N1, int* N2, int* M1, int* M2);
// Columns per CTA of the normal operator; the number of column tiles is also
// the number of p^H q partials per image and iteration.
constexpr int kNormTile = 8;
inline int cart_normal_tiles(int nx) { return (nx + kNormTile - 1) / kNormTile; }
// y = (A^H A + lam I) x for nb images
void launch_cart_apply(const CartOp& op, const float2* x, float2* y, int nb, float lam, cudaStream_t s);
// CG iteration `it`, normal-operator half: P = R + beta P; Q = (A^H A + lam) P; pq partials
void launch_cart_cg_normal(const CartOp& op, const CgArgs& a, int nb, int it, float lam, cudaStream_t s);
// PMR: G[b][c] = F^H_y (mask . n_{b,c}) (hybrid y, kx), scaled by 1/sqrt(ny nx);
// with data != nullptr the k-space values come from data [nb][nc][ny][nx] instead of the noise draw
void launch_cart_pmr_cols(const CartOp& op, float2* G, int nb, uint64_t seed, int64_t rep_begin, float sigma,
                          cudaStream_t s, const float2* data = nullptr);
// out[b] = sum_c conj(S_c) . F^H_x G[b][c]
void launch_cart_rows_adjoint(const CartOp& op, const float2* G, float2* out, int nb, cudaStream_t s);

// ---- gram.cu: dense per-column normal operator on the tensor cores ----
struct GramOp {
  int ny, nx, nt;           // nt: output rows per CTA (divides ny, <= 256)
  int kc;                   // contraction values per pipeline stage (16 or 8)
  int a_tmem;               // 1: the split direction is staged in tensor memory
  int f16;                  // 1 (with kc = 16, a_tmem = 0): FP16 head + remainder operands (kind::f16)
  // G_j split into a head and a remainder (TF32, or FP16 after scaling by
  // gscale[j]), stored as the kernel's pipeline stages consume it:
  // [j][y tile][chunk][re hi | im hi | re lo | im lo][nt rows][kc values,
  // 16-byte groups swizzled as in shared memory]
  void* G;
  float* gscale;            // [nx] power-of-two scale of G_j (FP16 form)
};
struct GramArgs {
  const float* in;          // r (CG) or x (apply), column-planar [B][nx][2][ny]
  const float* pold;        // previous direction (CG, it > 0)
  float* pnew;              // new direction (CG) or nullptr
  float* q;                 // (A^H A + lam) p; every vector 16-byte aligned (bulk copies)
  const float* beta;        // [B] (CG)
  const int* done;          // [B] (CG)
  double* pq;               // pq partials [B][itmax][PA] or nullptr
  int itmax, PA, it, nb, cg;
  float lam;
  int* err;                 // first failure code (bounded waits)
  const float* pscale;      // FP16 form: power-of-two scale of each image's operand [B]
                            // (per-column CG: ColCgArgs::pscale instead)
  // filled by the launcher
  const void* G;
  const float* gscale;
  int ny, nx, nt, nyt, stages, tmem_cols;
  int tma_epi;              // epilogue moves p and q by tensor copies (nt a multiple of 32)
};

// State of CG run separately on every readout column (phase-encode Cartesian
// contexts): one step length and one stopping test per (image, column).
// Arrays are [B][nx], image-major; the solution x and residual r are the
// context's column-planar X and R.
struct ColCgArgs {
  float* x;                 // [B][nx][2][ny] solution, updated in place
  float* r;                 // [B][nx][2][ny] residual (holds the right-hand side before init)
  const double* rr0;        // ||r_j||^2 of the right-hand side
  double* rr;               // ||r_j||^2 before the next update
  float* beta;              // step of the next direction update (0 before the first)
  int* done;                // 1 once the column met the stopping rule or broke down
  int* iters;               // updates taken by the column
  int* status;              // [B] 5 when any column of the image broke down
  double rtol2;             // squared relative residual tolerance
  double* pn;               // bound on the next direction's entries, sqrt(rr) + beta pn
  float* pscale;            // its power-of-two FP16 scale
};
bool gram_supported(int ny, int nx);
int gram_tile(int ny);
size_t gram_bytes(int ny, int nx);  // both G planes, head and remainder
int gram_pa(int ny, int nx);
bool gram_encode_x(CUtensorMap* m, float* base, int ny, int nx, int B, int kc);
void launch_gram_build(const float2* smaps, const uint8_t* mask_host, int nc, const GramOp& op, double2* pbuf,
                       cudaStream_t s);
// per image: beta, the stop flag, and (FP16 operands) the bound pn on the
// direction's entries, sqrt(rr) + beta pn_prev, with its power-of-two scale
void launch_gram_scalars(const CgArgs& a, int nb, int it, float* beta, int* done, double* pn, float* pscale,
                         cudaStream_t s);
// FP16 operands of an operator application: pscale[b] from max |x_b| (column-planar input)
void launch_gram_apply_scale(const float* x, int ny, int nx, int nb, float* pscale, cudaStream_t s);
void launch_gram_normal(const GramOp& op, const CUtensorMap& mIn, const CUtensorMap& mPold, GramArgs g,
                        cudaStream_t s);
// Per-column CG on the tensor-core operator.  Supported when the output-row
// tile is a multiple of 32 and a column spans at most 4 tiles (one thread-
// block cluster per column and image tile).
bool gram_colcg_supported(int ny, int nx);
// x = 0, rr0 = rr = ||b_j||^2, beta = 0, iters = 0, done where b_j = 0 (or
// non-finite: breakdown, status 5), for the nb right-hand sides in cg.r
void launch_colcg_init(const ColCgArgs& cg, int ny, int nx, int nb, cudaStream_t s);
// one CG update on every column of nb images: p = r + beta p_old (it > 0) or
// r, q = (A^H A + lam) p on the tensor cores, alpha = rr / p^H q, x += alpha p,
// r -= alpha q, beta = ||r||^2_new / rr -- all in one launch
// false (nothing launched) if a tile map cannot be encoded
bool launch_gram_colcg(const GramOp& op, const CUtensorMap& mIn, const CUtensorMap& mPold, GramArgs g,
                       const ColCgArgs& cg, cudaStream_t s);
// *flag (device) = 1 if any column of the nb images is still iterating, else 0
void launch_colcg_any_live(const ColCgArgs& cg, int nx, int nb, int* flag, cudaStream_t s);
// per image: the most updates any column took, and ||r|| / ||b|| over the image
void launch_colcg_report(const ColCgArgs& cg, int nx, int nb, int* iters, double* relres, cudaStream_t s);
void launch_to_cp(const float2* in, float* out, int ny, int nx, int nb, cudaStream_t s);

// ---- colcg_small.cu: per-column CG with the whole solve on chip (ny <= 96) ----
bool colcg_small_supported(int ny);
// G_j of every column, plain layout [nx][ny][ny] complex64 (pbuf: ny double2 of device scratch)
// Per-column CG of phase-encode images with the whole solve in one launch:
// clusters of ny / NT CTAs (NT = colcg_persist_rows(ny), 0 if unsupported)
// own a column and 128 images; G in the FP16 stage tiling of row blocks of NT
// (launch_gram_build with nt = NT); psplit of colcg_persist_split_bytes().
// R, X column-planar; rr0 / rr / iters per (image, column).
int colcg_persist_rows(int ny);
size_t colcg_persist_split_bytes(int ny, int nx, int B);
bool launch_colcg_persist(const void* G, const float* gscale, const float* R, float* X, uint8_t* psplit, double* rr0,
                          double* rr, int* iters, int* status, int* err, int ny, int nx, int nb, int max_iter,
                          double rtol2, float lam, cudaStream_t s);
void launch_colcg_small_build(const float2* smaps, const uint8_t* mask_host, int nc, int ny, int nx, float2* G,
                              float* gmax, double2* pbuf, cudaStream_t s);
// Whole-image CG on the on-chip kernel: per-column partial sums exchanged
// between the blocks of an image group (two tagged 64-bit words per sum)
struct SmallGlobal {
  ulonglong2* part_pq;  // [B][nx]
  ulonglong2* part_rr;  // [B][nx]
  int* err;             // error word of a bounded wait
};
// every CG update of nb right-hand sides rhs [nb][ny][nx] (natural layout) in
// one launch; x [nb][ny][nx]; rr0 / rr / iters per (image, column) [nb][nx]
// (column sums); gmax from launch_colcg_small_build.  glob == nullptr: CG per
// column; otherwise CG on the whole image (cooperative launches).  false if
// nothing could be launched.
bool launch_colcg_small(const float2* G, const float* gmax, const float2* rhs, float2* X, int ny, int nx, int nb,
                        int max_iter, double rtol2, float lam, double* rr0, double* rr, int* iters, int* status,
                        const SmallGlobal* glob, cudaStream_t s);
void launch_from_cp(const float* in, float2* out, int ny, int nx, int nb, cudaStream_t s);

// ---- spiral.cu: non-Cartesian (Toeplitz normal operator, KB gridding) ----
struct SpiralOp {
  int n;                    // image is n x n
  int L;                    // grid 2n
  int nc;
  int P1, P2;               // L = P1 * P2 split
  const float2* smaps;      // [nc][n][n] whitened
  const float2* tw2;        // [L] exp(-2 pi i e / L)
  const float* That;        // [L][L] real Toeplitz kernel, includes 1/L^2
  const float* deapod;      // [n] 1 / (phi^((x - n/2)/L) sqrt(n))
  // gridding
  int64_t M;                // samples
  const float2* u;          // [M] sample positions in grid units (2 k)
  const float2* cphase;     // [M] e^{i pi (kx + ky)} (image-centre shift)
  const int* tile_ptr;      // [ntiles + 1] CSR over 16x16 grid tiles
  const int* tile_idx;      // samples touching each tile (with the kernel half-width)
  float beta, halfw, inv_i0beta;
  int* err;                 // first failure code of a bounded wait (device), or nullptr
  int row_lines;            // image rows per block of the Toeplitz row passes: 4 or 16 (0 = 16)
  const float* gw;          // [M][2][kMaxTaps] Kaiser-Bessel weights of each sample's window (x, then y)
  const int2* go;           // [M] wrapped first grid index (x, y) of each sample's window
};
// 3-D tensor map over `planes` planes of rows x L complex64 values (8-byte
// elements), boxes of `cols` x `box_rows` values (the column pass's staging)
bool encode_plane_map(CUtensorMap* m, const void* base, int rows, int L, int64_t planes, int cols, int box_rows);
bool spiral_supported(int n, int* P1, int* P2);
bool grid_split(int L, int* P1, int* P2);  // split of a 2-D pass length (Toeplitz or 2-D Cartesian)
void launch_toep_h(const float* traj, int64_t M, int n, float2* c, cudaStream_t s);
void launch_toep_fft2(const SpiralOp& op, float2* c, cudaStream_t s);  // c <- DFT_2D(c)
void launch_toep_finalize(const float2* c, int L, float scale, float* That, cudaStream_t s);
void launch_toep_apply(const SpiralOp& op, const float2* x, float2* y, float2* G, int nb, float lam, cudaStream_t s);
void launch_toep_cg_normal(const SpiralOp& op, const CgArgs& a, float2* G, int nb, int it, float lam,
                           cudaStream_t s);
// the per-sample gridding windows (set-up; gw holds grid_table_floats(M) floats)
size_t grid_table_floats(int64_t M);
void launch_grid_table(const SpiralOp& op, float* gw, int2* go, cudaStream_t s);
void launch_grid_pmr(const SpiralOp& op, float2* Qgrid, int nb, uint64_t seed, int64_t rep_begin, float sigma,
                     cudaStream_t s, const float2* data = nullptr);
void launch_grid_adjoint_rest(const SpiralOp& op, float2* Qgrid, float2* out, int nb, cudaStream_t s);

// ---- cs.cu: nonlinear CS (L1-wavelet FISTA) and its Jacobian ----
struct Wavelet {
  float h[8], g[8];  // scaling / wavelet filters, g[m] = (-1)^m h[L-1-m]
  int L;
};
// coef = W x (levels, periodised, in place layout), tmp: scratch of the same size
void launch_dwt(const float2* x, float2* coef, float2* tmp, int n, int levels, int nb, const Wavelet& w,
                cudaStream_t s);
void launch_idwt(const float2* coef, float2* x, float2* tmp, int n, int levels, int nb, const Wavelet& w,
                 cudaStream_t s);
int dwt_kernels(int levels);
int idwt_kernels(int levels, bool in_place);
void launch_cs_gradstep(const float2* z, const float2* Mz, const float2* rhs, int64_t rhs_stride, float inv_lc,
                        float2* y, int64_t n, int nb, cudaStream_t s);
void launch_cs_soft(const float2* c, float2* keep, float2* out, float tau, int64_t n, int nb, cudaStream_t s);
void launch_axpy_bcast(float2* x, const float2* y, float alpha, int64_t n, int nb, cudaStream_t s);
void launch_cs_soft_tan(const float2* at, float2* dc, float tau, int64_t n, int nb, cudaStream_t s);
void launch_cs_momentum(const float2* xn, float2* x, float2* z, float c, int64_t n, int nb, cudaStream_t s);
void launch_vjp_a(float2* xbn, const float2* zb, float2* xk1, float c, int64_t n, int nb, cudaStream_t s);
void launch_vjp_b(const float2* yb, const float2* Myb, float inv_lc, float2* zb, float2* ysum, int64_t n, int nb,
                  cudaStream_t s);
void launch_scale(float2* x, float sc, int64_t n, int nb, cudaStream_t s);
void launch_mask2d(const float2* in, float2* out, const uint8_t* mask, float scale, int64_t n, int planes,
                   cudaStream_t s);
void launch_coil_combine(const float2* G, const float2* S, int nc, float2* x, int64_t n, int nb, cudaStream_t s);
void launch_noise_kspace2d(float2* G, const uint8_t* mask, int nc, int64_t n, int nb, uint64_t seed,
                           int64_t rep_begin, float sigma, cudaStream_t s);

// ---- fft_generic.cu: batched 1-D FFTs along rows / columns of row-major planes ----
bool fft_length_supported(int L);
bool launch_fft_rows(int L, float2* data, const float2* tw, int nrows, int planes, int64_t plane_stride, int sign,
                     cudaStream_t s);
bool launch_fft_cols(int L, float2* data, const float2* tw, int ncols, int planes, int64_t plane_stride, int sign,
                     cudaStream_t s);

// ---- encode.cu: forward encoding operator pieces ----
void launch_cart_smul(const float2* x, const float2* S, float2* G, int nb, int nc, int64_t n, cudaStream_t s);
void launch_cart_mask_scale(float2* G, const uint8_t* mask, int planes, int ny, int nx, float scale, cudaStream_t s);
void launch_spiral_pad(const SpiralOp& op, const float2* x, float2* G, int nb, cudaStream_t s);
void launch_nufft_interp(const SpiralOp& op, const float2* G, float2* y, int nb, cudaStream_t s);

}  // namespace pico
