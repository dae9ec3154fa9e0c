// Noise-map serving runtime: requests for PICO (and optionally PMR) maps of
// uneven size, coil count and trajectory arrive at any time; a scheduler
// thread admits them in arrival order while their device footprint fits the
// memory budget and a slot is free, builds each request's operator on its own
// CUDA stream (stream-ordered allocation, so admitting or retiring a request
// never synchronises the device), enqueues its probe batches, and retires it
// when its completion event fires.  Work of admitted requests overlaps on the
// GPU.  Every request's result depends only on its own inputs and seed, so it
// is bit-identical alone or in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "pico.h"

namespace pico {
pico_status init_impl(const pico_operator_desc* d, void* cuda_stream, size_t hbm_budget, bool async_alloc,
                      pico_ctx** out);
size_t footprint_bytes(const pico_operator_desc* d, bool with_kbuf);
}  // namespace pico

namespace {

using clk = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  pico_request req{};
  // owned copies of the host arrays of the descriptor
  std::vector<float> smaps, traj;
  std::vector<double> cov;
  std::vector<uint8_t> mask;
  std::vector<float> cs_data;  // whitened k-space of a CS request
  size_t footprint = 0;
  double t_arrival = 0, t_admit = 0, t_done = 0;
  // device state while active
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  pico_ctx* ctx = nullptr;
  double *d_sum = nullptr, *d_sumsq = nullptr, *d_psum = nullptr;
  float* d_cs = nullptr;  // device copy of the CS data and the reconstruction
  // results
  std::vector<double> var, pmr;
  pico_status status = PICO_OK;
  bool finished = false;
};

}  // namespace

struct pico_server {
  size_t budget = 0, in_use = 0;
  int max_active = 4;
  int chunk = 64;
  clk::time_point t0 = clk::now();
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::vector<std::shared_ptr<Request>> active;
  std::map<int64_t, std::shared_ptr<Request>> all;
  int64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  int device = 0;
};

namespace {

double now_s(const pico_server* s) { return std::chrono::duration<double>(clk::now() - s->t0).count(); }

// Build the operator and enqueue all of the request's work on its stream.
pico_status launch_request(pico_server* sv, Request& r) {
  if (cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking) != cudaSuccess) return PICO_E_CUDA;
  if (cudaEventCreateWithFlags(&r.done_ev, cudaEventDisableTiming) != cudaSuccess) return PICO_E_CUDA;
  pico_status st = pico::init_impl(&r.req.op, r.stream, 0, true, &r.ctx);
  if (st != PICO_OK) return st;
  const size_t n = (size_t)r.req.op.ny * r.req.op.nx;
  if (cudaMallocAsync((void**)&r.d_sum, 3 * n * sizeof(double), r.stream) != cudaSuccess) return PICO_E_OOM;
  r.d_sumsq = r.d_sum + n;
  r.d_psum = r.d_sum + 2 * n;
  if (r.req.cs_data) {
    const size_t kf = r.cs_data.size();
    if (cudaMallocAsync((void**)&r.d_cs, (kf + 2 * n) * sizeof(float), r.stream) != cudaSuccess) return PICO_E_OOM;
    if (cudaMemcpyAsync(r.d_cs, r.cs_data.data(), kf * sizeof(float), cudaMemcpyHostToDevice, r.stream) != cudaSuccess)
      return PICO_E_CUDA;
    st = pico_cs_recon(r.ctx, r.d_cs, r.req.cs_lambda, r.req.cs_iters, r.req.cs_levels, r.d_cs + kf);
    if (st != PICO_OK) return st;
    for (int32_t b = 0; b < r.req.nprobes; b += sv->chunk) {
      const int32_t nb = std::min(sv->chunk, r.req.nprobes - b);
      st = pico_cs_variance_map(r.ctx, r.req.seed, b, nb, r.req.probe_kind, r.d_sum, r.d_sumsq, b > 0);
      if (st != PICO_OK) return st;
    }
    for (int32_t b = 0; b < r.req.pmr_reps; b += sv->chunk) {
      const int32_t nb = std::min(sv->chunk, r.req.pmr_reps - b);
      st = pico_cs_pmr(r.ctx, r.req.seed, b, nb, r.req.pmr_sigma, r.d_psum, nullptr, b > 0);
      if (st != PICO_OK) return st;
    }
    if (cudaEventRecord(r.done_ev, r.stream) != cudaSuccess) return PICO_E_CUDA;
    return PICO_OK;
  }
  for (int32_t b = 0; b < r.req.nprobes; b += sv->chunk) {
    const int32_t nb = std::min(sv->chunk, r.req.nprobes - b);
    st = pico_variance_map(r.ctx, r.req.seed, b, nb, r.req.probe_kind, r.req.max_iter, r.req.rtol, r.d_sum,
                           r.d_sumsq, b > 0);
    if (st != PICO_OK) return st;
  }
  for (int32_t b = 0; b < r.req.pmr_reps; b += sv->chunk) {
    const int32_t nb = std::min(sv->chunk, r.req.pmr_reps - b);
    st = pico_pmr(r.ctx, r.req.seed, b, nb, r.req.pmr_sigma, r.req.max_iter, r.req.rtol, r.d_psum, nullptr, b > 0);
    if (st != PICO_OK) return st;
  }
  if (cudaEventRecord(r.done_ev, r.stream) != cudaSuccess) return PICO_E_CUDA;
  return PICO_OK;
}

void release_request(Request& r) {
  if (r.d_sum) cudaFreeAsync(r.d_sum, r.stream);
  r.d_sum = nullptr;
  if (r.d_cs) cudaFreeAsync(r.d_cs, r.stream);
  r.d_cs = nullptr;
  if (r.ctx) pico_destroy(r.ctx);
  r.ctx = nullptr;
  if (r.stream) cudaStreamSynchronize(r.stream);
  if (r.done_ev) cudaEventDestroy(r.done_ev);
  if (r.stream) cudaStreamDestroy(r.stream);
  r.done_ev = nullptr;
  r.stream = nullptr;
}

void finish(pico_server* sv, Request& r, pico_status st) {
  r.status = st;
  r.t_done = now_s(sv);
  r.finished = true;
}

void scheduler(pico_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    // admit in arrival order while a slot is free and the footprint fits
    while (!sv->queue.empty() && (int)sv->active.size() < sv->max_active) {
      auto r = sv->queue.front();
      if (sv->budget && sv->in_use + r->footprint > sv->budget && !sv->active.empty()) break;
      sv->queue.pop_front();
      sv->in_use += r->footprint;
      r->t_admit = now_s(sv);
      lk.unlock();
      const pico_status st = launch_request(sv, *r);
      lk.lock();
      if (st != PICO_OK) {
        release_request(*r);
        sv->in_use -= r->footprint;
        finish(sv, *r, st);
        sv->cv_done.notify_all();
        continue;
      }
      sv->active.push_back(r);
    }
    // retire finished requests
    for (size_t i = 0; i < sv->active.size();) {
      auto r = sv->active[i];
      const cudaError_t q = cudaEventQuery(r->done_ev);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      lk.unlock();
      pico_status st = q == cudaSuccess ? PICO_OK : PICO_E_CUDA;
      const size_t n = (size_t)r->req.op.ny * r->req.op.nx;
      if (st == PICO_OK) {
        std::vector<double> h(3 * n);
        if (cudaMemcpyAsync(h.data(), r->d_sum, h.size() * sizeof(double), cudaMemcpyDeviceToHost, r->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(r->stream) != cudaSuccess)
          st = PICO_E_CUDA;
        r->var.assign(n, 0.0);
        if (r->req.nprobes > 0)
          for (size_t k = 0; k < n; ++k) r->var[k] = h[k] / (double)r->req.nprobes;
        if (r->req.pmr_reps > 0) {
          r->pmr.assign(n, 0.0);
          for (size_t k = 0; k < n; ++k) r->pmr[k] = h[2 * n + k] / (double)r->req.pmr_reps;
        }
        if (st == PICO_OK) st = pico_sync(r->ctx);
      }
      release_request(*r);
      lk.lock();
      sv->in_use -= r->footprint;
      finish(sv, *r, st);
      sv->active.erase(sv->active.begin() + i);
      sv->cv_done.notify_all();
    }
    if (sv->stop && sv->queue.empty() && sv->active.empty()) break;
    if (sv->active.empty() && sv->queue.empty()) {
      sv->cv_sched.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
    } else {
      sv->cv_sched.wait_for(lk, std::chrono::microseconds(200));
    }
  }
}

}  // namespace

extern "C" {

pico_status pico_footprint(const pico_operator_desc* desc, int32_t with_kspace, size_t* bytes) {
  if (!desc || !bytes || desc->ny <= 0 || desc->nx <= 0 || desc->ncoils <= 0) return PICO_E_INVALID;
  *bytes = pico::footprint_bytes(desc, with_kspace != 0);
  return PICO_OK;
}

pico_status pico_server_create(size_t hbm_budget, int32_t max_active, int32_t chunk, pico_server** out) {
  if (!out || max_active < 1 || chunk < 1) return PICO_E_INVALID;
  auto* sv = new pico_server();
  sv->budget = hbm_budget;
  sv->max_active = max_active;
  sv->chunk = chunk;
  cudaGetDevice(&sv->device);
  sv->worker = std::thread(scheduler, sv);
  *out = sv;
  return PICO_OK;
}

pico_status pico_server_submit(pico_server* sv, const pico_request* rq, int64_t* id) {
  if (!sv || !rq || !id) return PICO_E_INVALID;
  const pico_operator_desc& d = rq->op;
  if (!d.smaps || d.ny <= 0 || d.nx <= 0 || d.ncoils <= 0 || rq->nprobes < 0 || rq->pmr_reps < 0)
    return PICO_E_INVALID;
  if (d.kind == PICO_CARTESIAN && !d.mask) return PICO_E_INVALID;
  if (d.kind == PICO_SPIRAL && (!d.traj || d.nsamp <= 0)) return PICO_E_INVALID;
  auto r = std::make_shared<Request>();
  r->req = *rq;
  const size_t n = (size_t)d.ny * d.nx;
  r->smaps.assign((const float*)d.smaps, (const float*)d.smaps + 2 * (size_t)d.ncoils * n);
  r->req.op.smaps = r->smaps.data();
  if (d.noise_cov) {
    r->cov.assign(d.noise_cov, d.noise_cov + 2 * (size_t)d.ncoils * d.ncoils);
    r->req.op.noise_cov = r->cov.data();
  }
  if (d.mask) {
    r->mask.assign(d.mask, d.mask + (size_t)d.ny * (d.mask_2d ? d.nx : 1));
    r->req.op.mask = r->mask.data();
  }
  if (d.traj) {
    r->traj.assign(d.traj, d.traj + 2 * (size_t)d.nsamp);
    r->req.op.traj = r->traj.data();
  }
  r->footprint = pico::footprint_bytes(&r->req.op, rq->pmr_reps > 0) + 3 * n * sizeof(double);
  if (rq->cs_data) {
    if (d.kind != PICO_CARTESIAN || d.power_iters <= 0 || rq->cs_iters < 1 || rq->cs_levels < 1)
      return PICO_E_INVALID;
    const size_t kf = 2 * (size_t)d.ncoils * n;  // k-space floats (layout of pico_forward)
    r->cs_data.assign((const float*)rq->cs_data, (const float*)rq->cs_data + kf);
    r->req.cs_data = r->cs_data.data();
    // k-space buffer (the adjoint of the data), six CS work images per batch
    // slot, the iterates' coefficients, A^H b and f(b), the data and the image
    const size_t B = d.max_batch > 0 ? (size_t)d.max_batch : 64;
    r->footprint = pico::footprint_bytes(&r->req.op, true) + 3 * n * sizeof(double) + 6 * B * n * 8 +
                   (size_t)rq->cs_iters * n * 8 + 2 * n * 8 + (kf + 2 * n) * sizeof(float);
  }
  if (sv->budget && r->footprint > sv->budget) return PICO_E_OOM;
  std::lock_guard<std::mutex> lk(sv->mu);
  r->id = sv->next_id++;
  r->t_arrival = now_s(sv);
  sv->queue.push_back(r);
  sv->all[r->id] = r;
  *id = r->id;
  sv->cv_sched.notify_all();
  return PICO_OK;
}

pico_status pico_server_wait(pico_server* sv, int64_t id, double* var_out, double* pmr_out,
                             pico_request_info* info) {
  if (!sv) return PICO_E_INVALID;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(id);
  if (it == sv->all.end()) return PICO_E_INVALID;
  auto r = it->second;
  sv->cv_done.wait(lk, [&] { return r->finished; });
  const size_t n = (size_t)r->req.op.ny * r->req.op.nx;
  if (var_out && r->status == PICO_OK && !r->var.empty()) std::memcpy(var_out, r->var.data(), n * sizeof(double));
  if (pmr_out && r->status == PICO_OK && !r->pmr.empty()) std::memcpy(pmr_out, r->pmr.data(), n * sizeof(double));
  if (info) {
    info->id = r->id;
    info->status = r->status;
    info->t_arrival = r->t_arrival;
    info->t_admit = r->t_admit;
    info->t_done = r->t_done;
    info->footprint_bytes = (int64_t)r->footprint;
  }
  sv->all.erase(it);
  return r->status;
}

pico_status pico_server_destroy(pico_server* sv) {
  if (!sv) return PICO_E_INVALID;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv_sched.notify_all();
  }
  sv->worker.join();
  delete sv;
  return PICO_OK;
}

}  // extern "C"
