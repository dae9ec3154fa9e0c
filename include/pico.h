/*
 * pico.h -- C ABI of libpico, the GPU hot path of PICO (Probing Image-space
 * COvariance) voxelwise noise-variance estimation for linear MRI
 * reconstructions (Dalmaz et al., "Fast Voxelwise SNR Estimation for
 * Iterative MRI Reconstructions").
 *
 * Problem (Sec. 2.1): pre-whitened multi-coil data b_w = A x + n_w with
 * n_w ~ CN(0, I) (Eq. 3), Tikhonov CG-SENSE reconstruction
 * x = (A^H A + lam I)^-1 A^H b_w (Eqs. 4-6), image-domain noise covariance
 * Sigma = (M + lam I)^-1 M (M + lam I)^-1 with M = A^H A (Eq. 8), variance
 * map diag(Sigma) (Eq. 10).  PICO (Alg. 1) estimates diag(Sigma) by
 * averaging Re(conj(v) . Sigma v) over random-phase probe images v (Eq. 20);
 * Sigma v is applied with CG on the normal equations (Sec. 2.2.3).  PMR
 * (Sec. 1) re-solves with synthetic k-space noise for comparison.
 *
 * Conventions (all entry points):
 *  - Images are complex64 (interleaved float re, im), row-major [ny][nx],
 *    voxel (y, x); batches are contiguous [nbatch][ny][nx].
 *  - "_dev" pointers are CUDA device pointers owned by the caller; they must
 *    stay valid until the work is finished (pico_sync).  Host pointers are
 *    read during the call only.
 *  - All GPU work is stream-ordered on the stream given to pico_init; results
 *    are valid after pico_sync (or any later synchronisation of that stream).
 *  - Every call returns a pico_status; no exceptions cross the ABI.  On error
 *    pico_last_error(ctx) describes the cause.  A failed call leaves the
 *    context usable unless the status is PICO_E_CUDA.
 *  - Results are deterministic: identical inputs give identical bits,
 *    independent of how probes are split into calls (probe_begin/accumulate).
 */
#ifndef PICO_H
#define PICO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pico_ctx pico_ctx;

typedef enum {
  PICO_OK = 0,
  PICO_E_INVALID = 1,     /* bad argument or descriptor                            */
  PICO_E_OOM = 2,         /* footprint above hbm_budget, or cudaMalloc failed      */
  PICO_E_CUDA = 3,        /* a CUDA runtime error; the context should be destroyed */
  PICO_E_TIMEOUT = 4,     /* a bounded device-side wait gave up                    */
  PICO_E_BREAKDOWN = 5,   /* CG met p^H (M + lam) p <= 0 for some right-hand side  */
  PICO_E_UNSUPPORTED = 6  /* valid request this build does not implement           */
} pico_status;

typedef enum { PICO_CARTESIAN = 0, PICO_SPIRAL = 1 } pico_kind;

/* How CG solves the normal equations (Eq. 6), see pico_set_solver. */
typedef enum { PICO_SOLVER_GLOBAL = 0, PICO_SOLVER_COLUMNS = 1 } pico_solver;

/* Probe families of Sec. 2.2.4: random phase (Eq. 20), real Rademacher
 * (Eq. 19), complex Gaussian (Eq. 18). */
typedef enum { PICO_PROBE_PHASE = 0, PICO_PROBE_RADEMACHER = 1, PICO_PROBE_GAUSS = 2 } pico_probe;

/* Acquisition and reconstruction description (Sec. 2.1.1-2.1.3). */
typedef struct {
  int32_t kind;             /* pico_kind                                                     */
  int32_t ny, nx;           /* image matrix                                                   */
  int32_t ncoils;           /* receive channels                                               */
  const void* smaps;        /* host complex64 [ncoils][ny][nx] coil sensitivities (copied)    */
  const double* noise_cov;  /* host complex128 [ncoils][ncoils] Hermitian PD channel noise
                               covariance Sigma_n (Eq. 2), or NULL for white noise; folded
                               into the sensitivities as L^-1 S with L L^H = Sigma_n (Eq. 3) */
  const uint8_t* mask;      /* Cartesian: host [ny] phase-encode mask, natural DFT order
                               (index ky, 0 = DC); every kx of a kept line is sampled;
                               with mask_2d: host [ny][nx] mask (ky, kx), square images      */
  int32_t mask_2d;          /* 0: phase-encode mask; 1: 2-D mask (e.g. Poisson disc)          */
  const float* traj;        /* spiral: host [nsamp][2] (kx, ky) in cycles/FOV                 */
  int64_t nsamp;            /* spiral samples                                                 */
  float oversamp;           /* spiral gridding oversampling (2.0)                             */
  int32_t kb_width;         /* spiral Kaiser-Bessel width (6)                                 */
  double lambda;            /* Tikhonov weight relative to the spectrally normalised operator:
                               lam_phys = lambda * power_margin * lambda_max(A^H A) (Sec. 3.3);
                               with power_iters == 0, lambda is taken as physical            */
  int32_t power_iters;      /* power-method steps for lambda_max (15 in the paper), 0 = none  */
  double power_margin;      /* safety factor on lambda_max (1.01 in the paper)                */
  int32_t max_batch;        /* right-hand sides solved together (0 = 64)                      */
  int32_t max_iter_cap;     /* largest max_iter accepted later (0 = 128)                      */
} pico_operator_desc;

typedef struct {
  double lambda_max;        /* power-method estimate (0 if power_iters == 0)                  */
  double lambda_phys;       /* Tikhonov weight applied to A^H A                               */
  int32_t kind, ny, nx, ncoils, max_batch, max_iter_cap;
  int64_t nsamp;
  uint64_t device_bytes;    /* device memory held by the context                              */
  int32_t normal_op;        /* how (A^H A + lam I) is applied inside CG: 0 column FFTs,
                               1 dense per-column Gram matrices on the tensor cores for
                               batches of at least gram_min_batch images (64 unless
                               tuned, pico_set_tuning / PICO_GRAM_MIN_BATCH) and
                               column FFTs below (phase-encode masks, ny % 16 == 0,
                               ny >= 128; PICO_NORMAL_OP=fft in the environment selects 0),
                               2 Toeplitz 2-D FFT passes                                   */
} pico_info;

/* Create a context: validates the descriptor, whitens the sensitivities,
 * uploads the operator, sizes the workspace for max_batch right-hand sides
 * and runs the power method (Sec. 3.3).  cuda_stream: a cudaStream_t (NULL =
 * legacy default stream).  hbm_budget: bytes the context may hold on the
 * device, 0 = unlimited; PICO_E_OOM is returned before any allocation if the
 * footprint exceeds it.  Synchronises the stream before returning.
 * On failure *out may still receive a context that only carries the error
 * text (pico_last_error); release it with pico_destroy. */
pico_status pico_init(const pico_operator_desc* desc, void* cuda_stream, size_t hbm_budget, pico_ctx** out);

/* Operator sizes and the normalisation actually used. */
pico_status pico_get_info(const pico_ctx* ctx, pico_info* info);

/* y = (A^H A + lam_phys I) x for nbatch images (Eq. 6 left-hand side).
 * x_dev, y_dev: device complex64 [nbatch][ny][nx]; must not overlap. */
pico_status pico_apply_normal(pico_ctx* ctx, const void* x_dev, void* y_dev, int32_t nbatch);

/* Forward encoding operator y = A x (Sec. 2.1.1, Eq. 1, pre-whitened as in
 * Eq. 3: A = L^-1 A~, so y is whitened k-space).  x_dev: device complex64
 * [nbatch][ny][nx].  y_dev: device complex64, Cartesian [nbatch][ncoils][ny][nx]
 * (orthonormal 2-D DFT, zero off the mask); spiral [nbatch][ncoils][nsamp]
 * (NUDFT e^{-2 pi i k.r/n}/n with r = (x, y) from 0, evaluated by a
 * Kaiser-Bessel NUFFT of width kb_width on the 2n grid). */
pico_status pico_forward(pico_ctx* ctx, const void* x_dev, void* y_dev, int32_t nbatch);

/* Adjoint y -> A^H y (layouts as pico_forward; Cartesian entries off the mask
 * are ignored).  With whitened data b_w, A^H b_w is the right-hand side of the
 * CG-SENSE normal equations (Eq. 6). */
pico_status pico_adjoint(pico_ctx* ctx, const void* y_dev, void* x_dev, int32_t nbatch);

/* Solve (A^H A + lam_phys I) x = rhs by CG from x0 = 0 for nbatch right-hand
 * sides (Eq. 6, CG-SENSE).  Each system stops after max_iter updates or once
 * ||r|| <= rtol ||rhs|| (rtol = 0: exactly max_iter updates).  Inner products
 * are accumulated in FP64.  rhs_dev, x_dev: device complex64 [nbatch][ny][nx].
 * iters_out (int32 [nbatch]) and relres_out (double [nbatch]) are HOST arrays
 * or NULL; if either is given the call synchronises the stream.
 * max_iter must be in [0, max_iter_cap]. */
pico_status pico_cg_batch(pico_ctx* ctx, const void* rhs_dev, void* x_dev, int32_t nbatch, int32_t max_iter,
                          double rtol, int32_t* iters_out, double* relres_out);

/* Choose the CG of every solve of this context (pico_cg_batch, pico_variance_map,
 * pico_variance_map_adaptive, pico_pmr):
 *   PICO_SOLVER_GLOBAL   CG on the whole image (Sec. 2.1.3, Eq. 6), the default;
 *   PICO_SOLVER_COLUMNS  Cartesian phase-encode masks: A^H A is block diagonal
 *                        over the nx readout columns (the mask acts on ky only,
 *                        F^H M F = (F_y^H M_y F_y) (x) I), so Eq. 6 splits into nx
 *                        independent ny x ny systems and CG runs on each one with
 *                        its own step lengths and its own stopping test
 *                        ||r_j|| <= rtol ||rhs_j||.  The fixed point is the same
 *                        (the exact solution); the iterates after a fixed number
 *                        of updates differ from the global CG's (each column's
 *                        iterate minimises that column's error in its own energy
 *                        norm, so no column converges slower).  With FP16
 *                        operands and ny a multiple of a row block of 80,
 *                        64, 48 or 32 rows with at most 8 blocks (ny = 128,
 *                        160, 192, 256, 320, 384, 512, ...) a whole solve is
 *                        one launch (x, r, p stay on chip for every update;
 *                        PICO_COLCG_PERSIST=0 in the environment at
 *                        pico_init turns this off); otherwise every update is
 *                        one fused launch on the tensor cores.  relres_out of
 *                        pico_cg_batch is ||r|| / ||rhs|| over the image and
 *                        iters_out the most updates any column took.
 * PICO_E_UNSUPPORTED for PICO_SOLVER_COLUMNS unless the context runs the
 * tensor-core operator (pico_info.normal_op == 1) with a row tile that is a
 * multiple of 32 and at most 4 tiles per column, or keeps its solves on chip
 * (normal_op == 3).  Drops the context's captured CUDA graphs; allocates
 * 28 bytes per (image, column) on first use, and for the one-launch solve
 * the FP16 G_j in its row tiling (8 nx ny^2 bytes) and the shared split
 * direction (ny / 16 x 16 KB per column and 128-image tile), unless that
 * would pass the context's hbm_budget (then the per-update kernel runs). */
pico_status pico_set_solver(pico_ctx* ctx, int32_t solver);
pico_status pico_get_solver(const pico_ctx* ctx, int32_t* solver);

/* PICO running sums (Alg. 1) over probes probe_begin .. probe_begin+nprobes-1
 * drawn under seed (probe_kind: pico_probe):
 *   sum_dev[k]   (+)= sum_i Re(conj(v_i[k]) (Sigma v_i)[k])
 *   sumsq_dev[k] (+)= sum_i Re(...)^2                (nullable)
 * Sigma v is one CG solve when lam_phys == 0, else solve / apply A^H A /
 * solve (Sec. 2.2.3).  sum_dev, sumsq_dev: device float64 [ny][nx];
 * accumulate = 0 overwrites them, 1 adds to them (checkpoint/resume and
 * splitting probes across calls give bit-identical totals).
 * The variance map is sum / (number of probes); see pico_finalize. */
pico_status pico_variance_map(pico_ctx* ctx, uint64_t seed, int64_t probe_begin, int32_t nprobes,
                              int32_t probe_kind, int32_t max_iter, double rtol, double* sum_dev,
                              double* sumsq_dev, int32_t accumulate);

/* Adaptive PICO (Sec. 5, stopping from the estimator's own variance): runs
 * probes 0, 1, ... under seed in chunks of `chunk` (>= 2) and stops once the
 * relative standard error of the running mean map,
 *   ||stderr||_2 / ||sum / N||_2  with  stderr = sqrt((sumsq/N - (sum/N)^2)/(N-1)),
 * is <= target, or after max_probes.  sum_dev and sumsq_dev (required,
 * device float64 [ny][nx]) are overwritten with the running sums;
 * probes_used (host) receives N, rel_stderr (host, nullable) the final
 * statistic.  Synchronises once per chunk. */
pico_status pico_variance_map_adaptive(pico_ctx* ctx, uint64_t seed, int32_t probe_kind, int32_t chunk,
                                       int64_t max_probes, int32_t max_iter, double rtol, double target,
                                       double* sum_dev, double* sumsq_dev, int64_t* probes_used,
                                       double* rel_stderr);

/* PMR running sums (Sec. 1; Sec. 3.2.2): replica i draws whitened k-space
 * noise n_i ~ CN(0, sigma^2 I) on the sampled positions, solves
 * x_i = (A^H A + lam_phys I)^-1 A^H n_i by CG and accumulates
 *   sum_dev[k] (+)= |x_i[k]|^2 / sigma^2,  sumsq_dev[k] (+)= (|x_i[k]|^2/sigma^2)^2.
 * Arguments as for pico_variance_map. */
pico_status pico_pmr(pico_ctx* ctx, uint64_t seed, int64_t rep_begin, int32_t nreps, double sigma,
                     int32_t max_iter, double rtol, double* sum_dev, double* sumsq_dev, int32_t accumulate);

/* ---- Nonlinear compressed sensing (Sec. 2.2.5) -----------------------------
 * Reconstruction f: b -> x by L1-wavelet FISTA (Beck & Teboulle; the paper's
 * FISTA of Sec. 3.2.3 with a db4 wavelet penalty):
 *   min_x 1/2 ||A x - b||^2 + lambda_l1 ||W x||_1,
 * W the periodised orthonormal 2-D Daubechies-4 DWT with `levels` levels, x0 = 0,
 * step 1/Lc with Lc = power_margin * lambda_max (Sec. 3.3; needs power_iters > 0),
 * standard momentum, complex soft threshold, `iters` iterations.  b_dev is
 * whitened k-space (layout of pico_forward, one acquisition), x_dev the image
 * [ny][nx].  The iterates are kept on the device for the Jacobian calls below;
 * the image must be square with ny divisible by 2^levels. */
pico_status pico_cs_recon(pico_ctx* ctx, const void* b_dev, double lambda_l1, int32_t iters, int32_t levels,
                          void* x_dev);

/* Number of pico_cs_recon calls this context has started (0 before the
 * first).  The Jacobian calls below linearise around the most recent one; a
 * caller that keeps a reconstruction's output for a later pico_cs_jvp /
 * pico_cs_vjp compares the generation it recorded with this value (the
 * torch.autograd.Function of the Python binding raises on a mismatch). */
pico_status pico_cs_generation(const pico_ctx* ctx, int64_t* generation);

/* Jacobian-vector product dx = J db of the last pico_cs_recon (tangent of the
 * unrolled iterations; the soft threshold's derivative is R-linear:
 * dS[dc] = (1 - tau/|c|) dc + (tau/|c|) u Re(conj(u) dc), u = c/|c|, for
 * |c| > tau, else 0).  db_dev: k-space [nbatch][...] as pico_forward;
 * dx_dev: [nbatch][ny][nx]. */
pico_status pico_cs_jvp(pico_ctx* ctx, const void* db_dev, void* dx_dev, int32_t nbatch);

/* Vector-Jacobian product bbar = J^T xbar, the adjoint of pico_cs_jvp for the
 * real inner product Re<a, b> (reverse sweep over the stored iterates).
 * xbar_dev [nbatch][ny][nx] -> bbar_dev k-space [nbatch][...]. */
pico_status pico_cs_vjp(pico_ctx* ctx, const void* xbar_dev, void* bbar_dev, int32_t nbatch);

/* Jacobian PICO (Sec. 2.2.5 with Alg. 1): running sums of Re(conj(v) . J J^T v)
 * over probes probe_begin.. of seed; arguments as pico_variance_map (the CG
 * settings do not apply).  Needs a prior pico_cs_recon. */
pico_status pico_cs_variance_map(pico_ctx* ctx, uint64_t seed, int64_t probe_begin, int32_t nprobes,
                                 int32_t probe_kind, double* sum_dev, double* sumsq_dev, int32_t accumulate);

/* PMR for the nonlinear reconstruction (Sec. 3.2.3): for replicas
 * rep_begin .. rep_begin + nreps - 1 of `seed`, draw whitened k-space noise n_i
 * (the draw of pico_pmr), rerun the last pico_cs_recon's FISTA on b + n_i with
 * the same lambda_l1, step, levels and iteration count, and accumulate
 *   sum_dev[k] (+)= |f(b + n_i)[k] - f(b)[k]|^2 / sigma^2,   sumsq_dev[k] (+)= (.)^2
 * (float64 [ny][nx], caller-owned; sumsq_dev nullable).  Needs a prior
 * pico_cs_recon.  For small sigma the mean tends to the same E|J n|^2 that
 * pico_cs_variance_map estimates. */
pico_status pico_cs_pmr(pico_ctx* ctx, uint64_t seed, int64_t rep_begin, int32_t nreps, double sigma,
                        double* sum_dev, double* sumsq_dev, int32_t accumulate);

/* The sparsifying transform W of the CS reconstruction as an operator: the
 * periodised orthonormal 2-D Daubechies-4 DWT with `levels` levels (inverse = 0)
 * or its inverse W^H (inverse = 1), coefficients in the in-place layout (the
 * approximation band top-left).  in_dev / out_dev: device complex64
 * [nbatch][ny][nx], caller-owned, may be equal.  Needs a square image divisible
 * by 2^levels (PICO_E_UNSUPPORTED otherwise). */
pico_status pico_wavelet(pico_ctx* ctx, const void* in_dev, void* out_dev, int32_t nbatch, int32_t levels,
                         int32_t inverse);

/* Finalise running sums over `count` samples (Alg. 1 output; the standard
 * error of the running mean per voxel, the convergence diagnostic of Sec. 5):
 *   var_dev[k] = sum[k] / count                                   (float32, nullable)
 *   stderr_dev[k] = sqrt((sumsq/count - (sum/count)^2) / (count-1)) (float32, nullable;
 *                                                                   needs sumsq_dev) */
pico_status pico_finalize(pico_ctx* ctx, const double* sum_dev, const double* sumsq_dev, int64_t count,
                          float* var_dev, float* stderr_dev);

/* g-factor map g = sigma_acc / (sqrt(R) sigma_ref) (Eq. 11) from two variance
 * maps (device float32 [ny][nx]); R is the acceleration factor. */
pico_status pico_gfactor(pico_ctx* ctx, const float* var_acc_dev, const float* var_ref_dev, double R,
                         float* g_dev);

/* Batched CG-SENSE solve that allocates no device memory.  The paper has no
 * counterpart: this is an interface for callers that cannot call cudaMalloc
 * while they run -- code inside a host application that owns all device
 * memory through its own fixed pool, or that must avoid the allocator's
 * implicit synchronisation.  It runs the same kernels as pico_cg_batch for a
 * Cartesian phase-encode mask but needs no context:
 *   smaps_dev  caller's device complex64 [ncoils][ny][nx] sensitivities,
 *              already pre-whitened (no noise covariance is applied here)
 *   mask_dev   caller's device uint8 [ny] phase-encode mask (natural DFT order)
 *   lam        physical Tikhonov weight added to A^H A
 *   rhs_dev, x_dev, nbatch, max_iter (<= 128), rtol  as in pico_cg_batch
 *              (no iteration report; a CG breakdown is not reported either:
 *              such a system keeps the iterate reached before it)
 *   cuda_stream  stream the work is enqueued on (NULL = legacy default)
 * Every temporary lives in one file-scope device array of
 * pico_cg_batch_static_capacity() bytes (64 MiB) that each GPU loading the
 * library keeps until the process exits.  A request whose temporaries do not
 * fit returns PICO_E_INVALID; pico_static_last_error() then states the bytes
 * needed.  The first call on a device looks the array's address up, so make
 * one call before any stream capture.  All calls share the array and it keeps
 * the previous call's contents: calls whose GPU work overlaps (other streams
 * or threads) race and must be serialised by the caller. */
pico_status pico_cg_batch_static(const void* smaps_dev, const uint8_t* mask_dev, int32_t ny, int32_t nx,
                                 int32_t ncoils, double lam, const void* rhs_dev, void* x_dev, int32_t nbatch,
                                 int32_t max_iter, double rtol, void* cuda_stream);
size_t pico_cg_batch_static_capacity(void);
const char* pico_static_last_error(void);

/* Device bytes a context for `desc` holds (what pico_init allocates, plus the
 * k-space / grid buffer of pico_pmr, pico_forward and pico_adjoint when
 * with_kspace != 0).  Host-only; for admission control. */
pico_status pico_footprint(const pico_operator_desc* desc, int32_t with_kspace, size_t* bytes);

/* ---- Serving runtime ------------------------------------------------------
 * A request asks for one PICO variance map (and optionally a PMR map) of one
 * acquisition.  Requests of different sizes, coil counts and trajectories may
 * be submitted at any time from any thread; a scheduler thread admits them in
 * arrival order while a slot is free (max_active) and their footprint fits
 * hbm_budget (0 = unlimited), builds each request's operator on its own CUDA
 * stream with stream-ordered allocation, enqueues its probes in batches of
 * `chunk`, and retires it when its work completes.  Work of admitted requests
 * overlaps on the GPU.  A request's result depends only on its own inputs, seed
 * and the chunk size: it is bit-identical in any mix and alone on a context with
 * max_batch = chunk (batches of at least 64 images of a Cartesian phase-encode
 * operator run on the tensor-core Gram operator, smaller ones on the column-FFT
 * kernel; the two agree to about 1e-6 relative, not bitwise).  The server uses the device
 * current at pico_server_create.  Overlap on the GPU covers fixed-count solves
 * (rtol = 0): a request with rtol > 0 synchronises its stream after every few
 * CG iterations to test the stopping rule, and the single scheduler thread
 * admits or retires no other request meanwhile. */
typedef struct pico_server pico_server;

typedef struct {
  pico_operator_desc op;    /* acquisition; its host arrays are copied at submit            */
  uint64_t seed;            /* probes 0..nprobes-1 and replicas 0..pmr_reps-1 of this seed */
  int32_t nprobes;          /* PICO probes (0 = no PICO map)                               */
  int32_t probe_kind;       /* pico_probe                                                  */
  int32_t max_iter;         /* CG iterations per solve                                     */
  double rtol;              /* CG relative-residual stop (0 = max_iter exactly)            */
  int32_t pmr_reps;         /* PMR replicas (0 = no PMR map)                               */
  double pmr_sigma;         /* PMR noise standard deviation                                */
  /* Nonlinear CS request (Sec. 2.2.5): with cs_data != NULL the maps are those
   * of the L1-wavelet FISTA reconstruction of cs_data (whitened k-space, layout
   * of pico_forward, host, copied at submit) -- Jacobian PICO and CS PMR --
   * with weight cs_lambda, cs_iters iterations and cs_levels DWT levels
   * (max_iter and rtol do not apply; the descriptor needs power_iters > 0). */
  const void* cs_data;
  double cs_lambda;
  int32_t cs_iters, cs_levels;
} pico_request;

typedef struct {
  int64_t id;
  int32_t status;           /* pico_status of the request                                  */
  double t_arrival, t_admit, t_done;  /* seconds on the server's clock                     */
  int64_t footprint_bytes;
} pico_request_info;

pico_status pico_server_create(size_t hbm_budget, int32_t max_active, int32_t chunk, pico_server** out);
/* Queue a request; returns at once with its id (PICO_E_OOM if it can never fit). */
pico_status pico_server_submit(pico_server* server, const pico_request* request, int64_t* id);
/* Block until request `id` is done; copy its maps (host float64 [ny][nx]: the
 * variance map sum/N and the PMR map, each nullable) and timing; forget it. */
pico_status pico_server_wait(pico_server* server, int64_t id, double* var_out, double* pmr_out,
                             pico_request_info* info);
/* Finish all queued work, stop the scheduler, free the server. */
pico_status pico_server_destroy(pico_server* server);

/* Device timing of this context's kernels by class, from CUDA events recorded
 * on the context stream around every launch while profiling is enabled.
 * pico_profile(ctx, 1) clears the totals and starts recording, (ctx, 0) stops.
 * Classes: 0 = SENSE normal operator (incl. the fused CG direction update),
 * 1 = CG init/update vector kernels, 2 = PMR noise + adjoint, 3 = accumulate /
 * finalize / small kernels.  pico_profile_read synchronises the stream and
 * returns the summed milliseconds and the number of launches of a class. */
pico_status pico_profile(pico_ctx* ctx, int32_t enable);
pico_status pico_profile_read(pico_ctx* ctx, int32_t kernel_class, double* total_ms, int64_t* launches);

/* Kernels launched by this context so far (all classes); reset = 1 zeroes the
 * counter after reading it. */
pico_status pico_launch_count(pico_ctx* ctx, int64_t* count, int32_t reset);

/* ---- Tuning ----------------------------------------------------------------
 * Launch shapes a context picks at run time.  Not a step of the method (the
 * paper has no counterpart): every setting gives the same result up to
 * rounding (bitwise the same for a given setting).
 *   gram_min_batch  CG batches of at least this many images use the tensor-core
 *                   Gram operator, smaller ones the column-FFT kernel (Cartesian
 *                   phase-encode contexts with normal_op == 1; 0 keeps the
 *                   current value, a value above max_batch disables the Gram path)
 *   gram_kc         contraction values per pipeline stage of the Gram operator,
 *                   16 or 8 (a change rebuilds the stage-tiled G_j, ~1 ms)
 *   gram_a_tmem     1: the split direction is staged in tensor memory and read
 *                   by the MMA from there (tiles that fit), 0: shared memory
 *   probe_batch     probes / replicas per CG batch in pico_variance_map and
 *                   pico_pmr, 1..max_batch (0 = max_batch)
 * pico_set_tuning validates every field (PICO_E_INVALID, nothing changed) and
 * drops the context's captured CUDA graphs.  Fields that do not apply to the
 * context's operator are kept but have no effect. */
typedef struct {
  int32_t gram_min_batch;
  int32_t gram_kc;
  int32_t gram_a_tmem;
  int32_t probe_batch;
} pico_tuning;
pico_status pico_get_tuning(const pico_ctx* ctx, pico_tuning* out);
pico_status pico_set_tuning(pico_ctx* ctx, const pico_tuning* in);

/* Measure and apply the fastest tuning for this context on this GPU.  Each
 * candidate runs `iters` CG iterations (2..32; 0 = 4) on a batch of random-phase
 * probes with CUDA events on the context stream (one untimed run first, which
 * also captures the iteration graph); the time per image and iteration is
 * compared.  Candidates: batch sizes 16, 32, 64, 128, 256 up to max_batch (and
 * max_batch itself) for the column-FFT or Toeplitz operator and, on contexts
 * with normal_op == 1, for the Gram operator with (kc, a_tmem) = (16, 0),
 * (16, 1), (8, 0).  The Gram variant is the fastest at the largest batch;
 * gram_min_batch the smallest batch from which on the Gram operator is at
 * least as fast as the column FFTs; probe_batch the batch with the lowest
 * time per image on the chosen operator.
 *   out       receives the applied tuning (may be NULL)
 *   times_us  NULL or room for `ntimes` doubles: [candidate][batch] microseconds
 *             per image and iteration, candidates (column FFT / Toeplitz, Gram
 *             16/0, Gram 16/1, Gram 8/0) x batches (16, 32, 64, 128, 256,
 *             max_batch); NaN where not measured (ntimes >= 24 for all)
 * Overwrites the context's CG workspace; synchronises the stream. */
pico_status pico_autotune(pico_ctx* ctx, int32_t iters, pico_tuning* out, double* times_us, int32_t ntimes);

/* The choice pico_autotune makes from its measurements, as a host-only pure
 * function (no context, no GPU): times_us is the [4][6] table described above
 * (NaN = not measured; a batch counts only where the column-FFT / Toeplitz
 * time is finite), max_batch the batch capacity, gram != 0 if the Gram rows
 * may be chosen.  Fills every field of *out (gram_kc = 0 and gram_min_batch =
 * max_batch + 1 when no Gram candidate applies; probe_batch = 0 when the
 * choice is max_batch).  PICO_E_INVALID without any measured batch. */
pico_status pico_tune_select(const double* times_us, int32_t max_batch, int32_t gram, pico_tuning* out);

/* Wait for all work of the context and report its asynchronous status:
 * PICO_E_CUDA for a CUDA error; otherwise every pending class is named in
 * pico_last_error and the status is PICO_E_TIMEOUT if a kernel's bounded
 * pipeline wait (the tensor-core Gram operator, the TMA-staged Toeplitz column
 * pass) gave up, else PICO_E_BREAKDOWN if a CG system broke down (a non-finite
 * residual -- NaN or Inf in a right-hand side or the operator -- or
 * p^H (M + lam) p <= 0) since the last pico_sync.  Broken-down systems keep the
 * iterate reached before the breakdown (x = 0 for a non-finite right-hand
 * side).  Both status words are cleared on the context stream, so the context
 * stays usable. */
pico_status pico_sync(pico_ctx* ctx);

/* Host-side fault injection for tests of the failure paths: sets the device
 * status word of class `cls` (PICO_E_TIMEOUT: the bounded-wait error word;
 * PICO_E_BREAKDOWN: the CG status of system 0) to `code` (nonzero), stream-
 * ordered and synchronised, exactly as a kernel would; the next pico_sync
 * reports and clears it.  No kernel is made to fail.  PICO_E_INVALID for any
 * other class or a zero code.  (No counterpart in the paper.) */
pico_status pico_inject_error(pico_ctx* ctx, int32_t cls, int32_t code);

/* Text of the last error of this context ("" if none).  Owned by the context. */
const char* pico_last_error(const pico_ctx* ctx);

/* Release every device and host resource of the context (NULL is ignored). */
void pico_destroy(pico_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PICO_H */
