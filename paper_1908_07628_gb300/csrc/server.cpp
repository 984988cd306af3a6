// Map server: a request loop with continuous batching for STEM-EELS maps.
//
// Requests of different grids, thicknesses, interpolation factors, transition
// sets and scans are queued in arrival order.  A request is admitted when a worker
// slot is free and its device footprint (dominated by the scattering matrices) fits
// in the HBM budget still unclaimed; admission is first-fit in arrival order, and a
// request that has been bypassed kMaxBypass times blocks further bypassing until it
// is admitted.  Each worker owns a context and a CUDA stream and runs the request's
// S-matrix build and map on it, so admitted requests overlap on the device; the
// request's S_in stays resident on the device until its map is complete.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "stem_eels.h"

namespace {

constexpr int kMaxBypass = 8;
constexpr int64_t kContractionCap = (int64_t)4 << 30;   // tensor-core buffers + FP32 M buffer

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t id = 0;
  eels_request in{};              // borrowed input pointers
  int64_t footprint = 0;
  int64_t pixel_slices = 0;
  std::vector<double> map;
  eels_status status = EELS_OK;
  std::string err;
  double t_submit = 0, t_start = 0, t_done = 0;
  bool done = false;
  int bypassed = 0;
};

int beams(int n, double cell, double lam, int f, double angle) {
  return eels_count_beams(n, cell, lam, f, angle);
}

}  // namespace

struct eels_server {
  int device = 0;
  int64_t budget = 0;
  int slots = 0;
  std::mutex mu;
  std::condition_variable cv;       // work available / request finished / stop
  std::deque<Request*> pending;
  std::map<int64_t, Request*> requests;
  int64_t in_use = 0, peak = 0, next_id = 1;
  bool stop = false;
  double t_first = -1, t_last = 0;
  std::vector<std::thread> workers;
};

namespace {

// First admissible pending request (arrival order, respecting the bypass limit).
Request* take_admissible(eels_server* sv) {
  for (size_t k = 0; k < sv->pending.size(); ++k) {
    Request* r = sv->pending[k];
    if (r->footprint <= sv->budget - sv->in_use) {
      for (size_t q = 0; q < k; ++q) sv->pending[q]->bypassed++;
      sv->pending.erase(sv->pending.begin() + k);
      return r;
    }
    if (r->bypassed >= kMaxBypass) return nullptr;   // oldest waits: no more bypassing
  }
  return nullptr;
}

void run_request(eels_ctx* ctx, cudaStream_t st, Request* r) {
  eels_smatrix* sm = nullptr;
  eels_status s = eels_build_smatrix(ctx, &r->in.spec, &r->in.optics, st, &sm);
  if (s == EELS_OK) {
    s = eels_inelastic_map(ctx, sm, &r->in.tr, &r->in.scan, r->in.beta, r->in.precision,
                           r->map.data(), 0, st);
  }
  if (s != EELS_OK) r->err = eels_last_error(ctx);
  eels_smatrix_free(sm);
  r->status = s;
}

void worker_main(eels_server* sv) {
  cudaSetDevice(sv->device);
  eels_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  const bool ok = eels_create(sv->device, &ctx) == EELS_OK &&
                  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      sv->cv.wait(lock, [&] { return sv->stop || (r = take_admissible(sv)) != nullptr; });
      if (!r) break;   // stopping
      sv->in_use += r->footprint;
      sv->peak = std::max(sv->peak, sv->in_use);
      r->t_start = now_s();
    }
    if (ok) {
      run_request(ctx, st, r);
    } else {
      r->status = EELS_ERR_CUDA;
      r->err = "worker could not create its context or stream";
    }
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      sv->in_use -= r->footprint;
      r->t_done = now_s();
      sv->t_last = std::max(sv->t_last, r->t_done);
      r->done = true;
    }
    sv->cv.notify_all();
  }
  if (st) cudaStreamDestroy(st);
  eels_destroy(ctx);
}

}  // namespace

extern "C" {

int64_t eels_request_footprint(const eels_request* q) {
  if (!q || q->spec.n <= 0 || q->spec.n_z <= 0 || q->optics.f < 1) return -1;
  const int n = q->spec.n, nz = q->spec.n_z;
  const int n_in = beams(n, q->spec.cell, q->optics.lambda, q->optics.f, q->optics.alpha);
  const int n_out = beams(n, q->spec.cell, q->optics.lambda, q->optics.f, q->beta);
  if (n_in < 0 || n_out < 0) return -1;
  const int64_t c = 8, nn = (int64_t)n * n, plane = (int64_t)(n / 2) * (n / 2);
  const int64_t resident = c * nz * nn + c * plane + c * (int64_t)nz * n_in * plane;
  const int64_t forward = 2 * c * (int64_t)n_in * n * (n / 2) + 4 * (int64_t)nz * nn;
  const int64_t h = (int64_t)(q->tr.h_shared ? 1 : q->tr.n_sites) * q->tr.n_types * q->tr.w *
                    q->tr.w * 8;
  const int64_t backward = 2 * c * (int64_t)n_out * n * (n / 2) + c * (int64_t)n_out * plane +
                           kContractionCap + h;
  return resident + std::max(forward, backward);
}

eels_status eels_server_create(int device, int64_t hbm_budget, int slots, eels_server** out) {
  if (!out || slots < 1 || hbm_budget <= 0) return EELS_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return EELS_ERR_CUDA;
  eels_server* sv = new eels_server();
  sv->device = device;
  sv->budget = hbm_budget;
  sv->slots = slots;
  for (int k = 0; k < slots; ++k) sv->workers.emplace_back(worker_main, sv);
  *out = sv;
  return EELS_OK;
}

eels_status eels_server_submit(eels_server* sv, const eels_request* q, int64_t* id) {
  if (!sv || !q || !id) return EELS_ERR_ARG;
  if (q->spec.vproj_on_device || q->tr.on_device) return EELS_ERR_ARG;   // host inputs only
  const int64_t fp = eels_request_footprint(q);
  if (fp < 0) return EELS_ERR_ARG;
  if (fp > sv->budget) return EELS_ERR_OOM;   // can never be admitted
  Request* r = new Request();
  r->in = *q;
  r->footprint = fp;
  r->pixel_slices = (int64_t)q->scan.n_sx * q->scan.n_sy * q->spec.n_z;
  r->map.assign((size_t)q->tr.n_types * q->scan.n_sx * q->scan.n_sy, 0.0);
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    r->id = sv->next_id++;
    r->t_submit = now_s();
    if (sv->t_first < 0) sv->t_first = r->t_submit;
    sv->requests[r->id] = r;
    sv->pending.push_back(r);
  }
  sv->cv.notify_all();
  *id = r->id;
  return EELS_OK;
}

eels_status eels_server_wait(eels_server* sv, int64_t id, double* map_out, double timeout_s,
                             double* latency_s) {
  if (!sv) return EELS_ERR_ARG;
  std::unique_lock<std::mutex> lock(sv->mu);
  auto it = sv->requests.find(id);
  if (it == sv->requests.end()) return EELS_ERR_ARG;
  Request* r = it->second;
  const bool finished = sv->cv.wait_for(
      lock, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9), [&] { return r->done; });
  if (!finished) return EELS_ERR_TIMEOUT;
  if (map_out && r->status == EELS_OK)
    std::memcpy(map_out, r->map.data(), r->map.size() * sizeof(double));
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  return r->status;
}

eels_status eels_server_stats_get(eels_server* sv, eels_server_stats* st) {
  if (!sv || !st) return EELS_ERR_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  std::vector<double> lat;
  int64_t px = 0, failed = 0;
  double wait = 0;
  for (auto& kv : sv->requests) {
    const Request* r = kv.second;
    if (!r->done) continue;
    if (r->status != EELS_OK) {
      failed++;
      continue;
    }
    lat.push_back(r->t_done - r->t_submit);
    wait += r->t_start - r->t_submit;
    px += r->pixel_slices;
  }
  std::memset(st, 0, sizeof(*st));
  st->submitted = (int64_t)sv->requests.size();
  st->completed = (int64_t)lat.size();
  st->failed = failed;
  st->peak_bytes = sv->peak;
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) {
      const double pos = p * (lat.size() - 1);
      const size_t a = (size_t)std::floor(pos), b = std::min(a + 1, lat.size() - 1);
      return lat[a] + (lat[b] - lat[a]) * (pos - a);
    };
    st->p50_ms = 1e3 * pct(0.50);
    st->p99_ms = 1e3 * pct(0.99);
    st->max_ms = 1e3 * lat.back();
    double s = 0;
    for (double v : lat) s += v;
    st->mean_ms = 1e3 * s / lat.size();
    st->mean_wait_ms = 1e3 * wait / lat.size();
    st->makespan_s = sv->t_last - sv->t_first;
    st->pixel_slices_per_s = st->makespan_s > 0 ? px / st->makespan_s : 0;
  }
  return EELS_OK;
}

void eels_server_destroy(eels_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto& t : sv->workers) t.join();
  for (auto& kv : sv->requests) delete kv.second;
  delete sv;
}

}  // extern "C"
