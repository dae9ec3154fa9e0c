// pico_cg_batch_static: batched CG-SENSE solves that allocate no device memory.
//
// Some callers cannot call cudaMalloc while they run: code that executes
// inside an already-running frame of a host application whose device memory
// is fully managed by someone else (a scanner reconstruction pipeline with a
// fixed memory pool, a plug-in loaded into another process, or code that must
// not trigger the allocator's implicit synchronisation).  For them this entry
// point runs the same kernels as pico_cg_batch but keeps every temporary
// (residual, search direction, operator output, the per-iteration inner-
// product partials and the FFT tables) in one file-scope device array of fixed
// size, kStaticBytes.  Inputs and outputs stay the caller's.
//
// The array is part of the library's device image: every GPU that loads the
// library holds it until the process exits.  Its address is looked up once per
// device, on the first call made while that device is current; make that first
// call before any CUDA stream capture.  Every call uses the same array and it
// keeps the contents of the last call, so calls whose GPU work overlaps (two
// streams, two host threads) race and give wrong results: serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "pico.h"

namespace {

constexpr size_t kStaticBytes = (size_t)64 << 20;  // 64 MiB of scratch
constexpr int kMaxDevices = 64;
constexpr int kStaticItMax = 128;

static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
thread_local char g_err[256] = "";

pico_status static_fail(pico_status st, const char* msg) {
  std::snprintf(g_err, sizeof(g_err), "%s", msg);
  return st;
}

// Device address of g_scratch for the current device (looked up once).
pico_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return static_fail(PICO_E_CUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return static_fail(PICO_E_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return static_fail(PICO_E_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PICO_OK;
}

// mask(ky)/ny and the twiddles exp(-2 pi i e / ny), written into the scratch
__global__ void k_static_tables(const uint8_t* mask, int ny, float* ymul, float2* tw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ny) return;
  ymul[i] = mask[i] ? 1.0f / (float)ny : 0.0f;
  float s, c;
  sincospif(-2.0f * (float)i / (float)ny, &s, &c);
  tw[i] = make_float2(c, s);
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

size_t pico_cg_batch_static_capacity(void) { return kStaticBytes; }

const char* pico_static_last_error(void) { return g_err; }

pico_status pico_cg_batch_static(const void* smaps_dev, const uint8_t* mask_dev, int32_t ny, int32_t nx,
                                 int32_t ncoils, double lam, const void* rhs_dev, void* x_dev, int32_t nbatch,
                                 int32_t max_iter, double rtol, void* cuda_stream) {
  g_err[0] = 0;
  if (!smaps_dev || !mask_dev || !rhs_dev || !x_dev) return static_fail(PICO_E_INVALID, "null pointer argument");
  if (ny <= 0 || nx <= 0 || ncoils <= 0 || nbatch < 0) return static_fail(PICO_E_INVALID, "bad sizes");
  if (max_iter < 0 || max_iter > kStaticItMax) return static_fail(PICO_E_INVALID, "max_iter outside [0, 128]");
  if (!(rtol >= 0.0) || !(lam >= 0.0)) return static_fail(PICO_E_INVALID, "rtol and lam must be >= 0");
  int N1, N2, M1, M2;
  if (!pico::cart_supported(ny, nx, &N1, &N2, &M1, &M2))
    return static_fail(PICO_E_UNSUPPORTED, "ny has no FFT split in this build");
  if (nbatch == 0) return PICO_OK;

  const int64_t n = (int64_t)ny * nx;
  const int PB = (int)((n + pico::kVecPerBlock - 1) / pico::kVecPerBlock);
  const int PA = pico::cart_normal_tiles(nx);
  // layout of the scratch array for this call
  const size_t vec = align256((size_t)nbatch * n * sizeof(float2));
  const size_t off_R = 0, off_P = vec, off_Q = 2 * vec;
  const size_t off_rr = 3 * vec;
  const size_t off_pq = off_rr + align256((size_t)nbatch * (kStaticItMax + 1) * PB * sizeof(double));
  const size_t off_st = off_pq + align256((size_t)nbatch * kStaticItMax * PA * sizeof(double));
  const size_t off_ym = off_st + align256((size_t)nbatch * sizeof(int));
  const size_t off_tw = off_ym + align256((size_t)ny * sizeof(float));
  const size_t need = off_tw + align256((size_t)ny * sizeof(float2));
  if (need > kStaticBytes) {
    std::snprintf(g_err, sizeof(g_err),
                  "nbatch=%d images of %dx%d need %zu bytes of scratch; the static array holds %zu",
                  nbatch, ny, nx, need, kStaticBytes);
    return PICO_E_INVALID;
  }

  void* base = nullptr;
  pico_status st = scratch_address(&base);
  if (st != PICO_OK) return st;
  unsigned char* sb = static_cast<unsigned char*>(base);
  cudaStream_t s = (cudaStream_t)cuda_stream;

  float* ymul = reinterpret_cast<float*>(sb + off_ym);
  float2* tw = reinterpret_cast<float2*>(sb + off_tw);
  k_static_tables<<<(ny + 127) / 128, 128, 0, s>>>(mask_dev, ny, ymul, tw);
  cudaMemsetAsync(sb + off_st, 0, (size_t)nbatch * sizeof(int), s);
  cudaMemcpyAsync(sb + off_R, rhs_dev, (size_t)nbatch * n * sizeof(float2), cudaMemcpyDeviceToDevice, s);

  pico::CartOp op{ny, nx, ncoils, N1, N2, static_cast<const float2*>(smaps_dev), ymul, tw, mask_dev, M1, M2,
                  nullptr};
  pico::CgArgs a{n,
                 static_cast<float2*>(x_dev),
                 reinterpret_cast<float2*>(sb + off_R),
                 reinterpret_cast<float2*>(sb + off_P),
                 reinterpret_cast<float2*>(sb + off_Q),
                 reinterpret_cast<double*>(sb + off_rr),
                 reinterpret_cast<double*>(sb + off_pq),
                 reinterpret_cast<int*>(sb + off_st),
                 PB,
                 PA,
                 kStaticItMax,
                 rtol * rtol};
  pico::launch_cg_init_rhs(a, nbatch, s);
  for (int it = 0; it < max_iter; ++it) {
    pico::launch_cart_cg_normal(op, a, nbatch, it, (float)lam, s);
    pico::launch_cg_update(a, nbatch, it, s);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(PICO_E_CUDA, cudaGetErrorString(e));
  return PICO_OK;
}

}  // extern "C"
