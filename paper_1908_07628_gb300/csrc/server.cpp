// Map server: a request loop with continuous batching for STEM-EELS maps.
//
// Requests of different grids, thicknesses, interpolation factors, transition sets and
// scans are queued in arrival order.  A request is admitted as soon as its device
// footprint (dominated by the scattering matrices) fits in the HBM budget still
// unclaimed; admission is first-fit in arrival order, and a request that has been
// bypassed kMaxBypass times blocks further bypassing until it is admitted.  Every
// admitted request runs on its own host thread, context and CUDA stream, and its S_in
// stays resident on the device until its map is complete.
//
// Work is issued in tiles: one tile is a few slices of the S-matrix build or a few
// depths of the map (the backward S_out step and the contraction of the sites there).
// `slots` issue tokens gate the device: a request holds a token while it issues one
// tile, waits for that tile to finish on its stream, hands the token to the request
// that has waited longest, and queues again.  Tiles of different requests therefore
// interleave and overlap on the device, a request that arrives while long ones run
// starts after at most one tile of each, and a cancelled request, or one past its
// deadline, is dropped at its next tile boundary with its memory released.
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

#include "internal.h"
#include "stem_eels.h"

namespace {

constexpr int kMaxBypass = 8;
constexpr int kTileSteps = 4;                            // slices or depths per tile
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
  int n_in = 0, n_out = 0;        // probe and detector beams
  int64_t wave_steps = 0;         // multislice wave-slice steps the request issues
  double flops = 0;               // the map's contraction flops, once it has finished
  std::vector<double> map;
  eels_status status = EELS_OK;
  std::string err;
  double t_submit = 0, t_admit = 0, t_first_tile = -1, t_done = 0;
  bool done = false, cancel = false, holds_token = false;
  int bypassed = 0;
  int tiles = 0;                  // tiles issued so far
  eels_server* sv = nullptr;
  cudaStream_t st = nullptr;
};

int beams(int n, double cell, double lam, int f, double angle) {
  return eels_count_beams(n, cell, lam, f, angle);
}

}  // namespace

struct eels_server {
  int device = 0;
  int64_t budget = 0;
  int slots = 0;                    // issue tokens
  std::mutex mu;
  std::condition_variable cv;       // admission, tokens, completion, stop
  std::deque<Request*> pending;     // submitted, not yet admitted
  std::deque<Request*> gate;        // admitted, waiting for a token (FIFO)
  std::map<int64_t, Request*> requests;
  int64_t in_use = 0, peak = 0, next_id = 1;
  int tokens = 0;                   // free issue tokens
  int running = 0;                  // admitted requests not yet finished
  bool stop = false;
  double t0 = 0, t_first = -1, t_last = 0;
  std::thread admitter;
  std::vector<std::thread> threads;
};

namespace {

bool expired(const Request* r, double t) {
  return r->cancel || (r->in.deadline_s > 0 && t - r->t_submit > r->in.deadline_s);
}

// Wait (holding the lock) until r is first in the gate queue and a token is free.
// False if the request was cancelled or expired meanwhile (then it holds no token).
bool acquire_token(eels_server* sv, Request* r, std::unique_lock<std::mutex>& lock) {
  sv->gate.push_back(r);
  sv->cv.notify_all();
  // woken by token hand-overs and cancellations; deadlines pass silently, so re-check
  while (!(expired(r, now_s()) || (sv->tokens > 0 && sv->gate.front() == r)))
    sv->cv.wait_for(lock, std::chrono::milliseconds(20));
  sv->gate.erase(std::find(sv->gate.begin(), sv->gate.end(), r));
  if (expired(r, now_s())) {
    sv->cv.notify_all();
    return false;
  }
  sv->tokens--;
  r->holds_token = true;
  if (r->t_first_tile < 0) r->t_first_tile = now_s();
  return true;
}

void release_token(eels_server* sv, Request* r) {
  if (!r->holds_token) return;
  r->holds_token = false;
  sv->tokens++;
  sv->cv.notify_all();
}

// Tile boundary of a request's build or map: let the tile finish on the request's
// stream, pass the token on and queue for the next tile.
int tile_gate(void* user, int /*phase*/, int done, int total) {
  Request* r = static_cast<Request*>(user);
  if (done % kTileSteps != 0 && done != total) return 0;   // inside a tile
  cudaStreamSynchronize(r->st);
  eels_server* sv = r->sv;
  std::unique_lock<std::mutex> lock(sv->mu);
  r->tiles++;
  release_token(sv, r);
  return acquire_token(sv, r, lock) ? 0 : 1;
}

void run_request(eels_server* sv, Request* r) {
  cudaSetDevice(sv->device);
  eels_ctx* ctx = nullptr;
  eels_status s = eels_create(sv->device, &ctx);
  if (s == EELS_OK && cudaStreamCreateWithFlags(&r->st, cudaStreamNonBlocking) != cudaSuccess)
    s = EELS_ERR_CUDA;
  if (s == EELS_OK) {
    // the grouping follows from the request alone, never from the load (EELS_ASSOC_MODEL)
    eels_set_option(ctx, EELS_OPT_ASSOCIATION, EELS_ASSOC_MODEL);
    eels_set_option(ctx, EELS_OPT_SIN_CHECKPOINT, r->in.sin_checkpoint);
    // operand buffers within the footprint's contraction allowance (kContractionCap)
    eels_set_option(ctx, EELS_OPT_OPERAND_MIB, 3072);
    eels::set_tile_hook(ctx, tile_gate, r);
    bool go;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      go = acquire_token(sv, r, lock);
    }
    if (!go) {
      s = EELS_ERR_CANCELLED;
    } else {
      eels_smatrix* sm = nullptr;
      s = eels_build_smatrix(ctx, &r->in.spec, &r->in.optics, r->st, &sm);
      if (s == EELS_OK)
        s = eels_inelastic_map(ctx, sm, &r->in.tr, &r->in.scan, r->in.beta, r->in.precision,
                               r->map.data(), 0, r->st);
      if (s != EELS_OK) r->err = eels_last_error(ctx);
      const double flops = s == EELS_OK ? eels::last_map_flops(ctx) : 0.0;
      {
        std::lock_guard<std::mutex> lock(sv->mu);
        r->flops = flops;
      }
      eels_smatrix_free(sm);
    }
  } else {
    r->err = "could not create the request's context or stream";
  }
  if (r->st) cudaStreamDestroy(r->st);
  eels_destroy(ctx);
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    release_token(sv, r);
    r->status = s;
    sv->in_use -= r->footprint;
    sv->running--;
    r->t_done = now_s();
    sv->t_last = std::max(sv->t_last, r->t_done);
    r->done = true;
  }
  sv->cv.notify_all();
}

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

void admit_loop(eels_server* sv) {
  std::unique_lock<std::mutex> lock(sv->mu);
  for (;;) {
    Request* r = nullptr;
    sv->cv.wait(lock, [&] { return sv->stop || (r = take_admissible(sv)) != nullptr; });
    if (!r) break;   // stopping
    sv->in_use += r->footprint;
    sv->peak = std::max(sv->peak, sv->in_use);
    sv->running++;
    r->t_admit = now_s();
    sv->threads.emplace_back(run_request, sv, r);
  }
}

}  // namespace

extern "C" {

int64_t eels_request_footprint(const eels_request* q) {
  if (!q || q->spec.n <= 0 || q->spec.n_z <= 0 || q->optics.f < 1) return -1;
  const int n = q->spec.n, nz = q->spec.n_z;
  const int n_in = beams(n, q->spec.cell, q->optics.lambda, q->optics.f, q->optics.alpha);
  const int n_out = beams(n, q->spec.cell, q->optics.lambda, q->optics.f, q->beta);
  if (n_in < 0 || n_out < 0) return -1;
  const int k = q->sin_checkpoint >= 2 ? q->sin_checkpoint : 0;
  const int64_t c = 8, nn = (int64_t)n * n, plane = (int64_t)(n / 2) * (n / 2);
  const int64_t wave = c * (int64_t)n * (n / 2);   // one row-spectrum wave
  // transmissions, propagator table and S_in (every depth, or the checkpoints)
  const int64_t resident = c * nz * nn + c * plane +
                           (k ? (int64_t)((nz + k - 1) / k) * n_in * wave
                              : c * (int64_t)nz * n_in * plane);
  const int64_t forward = 2 * (int64_t)n_in * wave + 4 * (int64_t)nz * nn;
  const int64_t h = (int64_t)(q->tr.h_shared ? 1 : q->tr.n_sites) * q->tr.n_types * q->tr.w *
                    q->tr.w * 8;
  // the map: backward work arrays, one S_out depth, contraction buffers, H, and with
  // checkpoints the forward work arrays and one segment of S_in
  const int64_t backward = 2 * (int64_t)n_out * wave + c * (int64_t)n_out * plane +
                           kContractionCap + h +
                           (k ? 2 * (int64_t)n_in * wave + c * (int64_t)k * n_in * plane : 0);
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
  sv->tokens = slots;
  sv->t0 = now_s();
  sv->admitter = std::thread(admit_loop, sv);
  *out = sv;
  return EELS_OK;
}

eels_status eels_server_submit(eels_server* sv, const eels_request* q, int64_t* id) {
  if (!sv || !q || !id) return EELS_ERR_ARG;
  if (q->spec.vproj_on_device || q->tr.on_device) return EELS_ERR_ARG;   // host inputs only
  if (!(q->deadline_s >= 0) || q->sin_checkpoint < -1) return EELS_ERR_ARG;
  eels_request in = *q;
  if (in.sin_checkpoint == -1) {
    // checkpoint S_in only when storing every depth would take more than half the budget
    in.sin_checkpoint = 0;
    const int64_t whole = eels_request_footprint(&in);
    if (whole > sv->budget / 2)
      in.sin_checkpoint = std::max(2, (int)std::ceil(std::sqrt(2.0 * in.spec.n_z)));
  }
  const int64_t fp = eels_request_footprint(&in);
  if (fp < 0) return EELS_ERR_ARG;
  if (fp > sv->budget) return EELS_ERR_OOM;   // can never be admitted
  Request* r = new Request();
  r->in = in;
  r->sv = sv;
  r->footprint = fp;
  r->pixel_slices = (int64_t)q->scan.n_sx * q->scan.n_sy * q->spec.n_z;
  r->n_in = beams(in.spec.n, in.spec.cell, in.optics.lambda, in.optics.f, in.optics.alpha);
  r->n_out = beams(in.spec.n, in.spec.cell, in.optics.lambda, in.optics.f, in.beta);
  r->wave_steps = ((int64_t)r->n_in * (in.sin_checkpoint >= 2 ? 2 : 1) + r->n_out) * in.spec.n_z;
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

eels_status eels_server_cancel(eels_server* sv, int64_t id) {
  if (!sv) return EELS_ERR_ARG;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->requests.find(id);
    if (it == sv->requests.end()) return EELS_ERR_ARG;
    Request* r = it->second;
    if (r->done) return EELS_OK;
    r->cancel = true;
    auto p = std::find(sv->pending.begin(), sv->pending.end(), r);
    if (p != sv->pending.end()) {   // never admitted: finished here
      sv->pending.erase(p);
      r->status = EELS_ERR_CANCELLED;
      r->err = "cancelled before admission";
      r->t_done = now_s();
      r->done = true;
    }
  }
  sv->cv.notify_all();
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

eels_status eels_server_request_info(eels_server* sv, int64_t id, eels_request_info* out) {
  if (!sv || !out) return EELS_ERR_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->requests.find(id);
  if (it == sv->requests.end()) return EELS_ERR_ARG;
  const Request* r = it->second;
  std::memset(out, 0, sizeof(*out));
  out->done = r->done ? 1 : 0;
  out->status = r->done ? r->status : EELS_OK;
  out->t_submit = r->t_submit - sv->t0;
  out->t_admit = r->t_admit > 0 ? r->t_admit - sv->t0 : -1;
  out->t_first_tile = r->t_first_tile >= 0 ? r->t_first_tile - sv->t0 : -1;
  out->t_done = r->done ? r->t_done - sv->t0 : -1;
  out->tiles = r->tiles;
  out->footprint = r->footprint;
  out->n_in = r->n_in;
  out->n_out = r->n_out;
  out->pixel_slices = r->pixel_slices;
  out->wave_steps = r->wave_steps;
  out->contraction_flops = r->flops;
  return EELS_OK;
}

eels_status eels_server_stats_get(eels_server* sv, eels_server_stats* st) {
  if (!sv || !st) return EELS_ERR_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  std::vector<double> lat;
  int64_t px = 0, failed = 0, cancelled = 0;
  double wait = 0;
  for (auto& kv : sv->requests) {
    const Request* r = kv.second;
    if (!r->done) continue;
    if (r->status == EELS_ERR_CANCELLED) {
      cancelled++;
      continue;
    }
    if (r->status != EELS_OK) {
      failed++;
      continue;
    }
    lat.push_back(r->t_done - r->t_submit);
    wait += r->t_first_tile - r->t_submit;
    px += r->pixel_slices;
  }
  std::memset(st, 0, sizeof(*st));
  st->submitted = (int64_t)sv->requests.size();
  st->completed = (int64_t)lat.size();
  st->failed = failed;
  st->cancelled = cancelled;
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
    for (Request* r : sv->pending) {   // never admitted: dropped
      r->status = EELS_ERR_CANCELLED;
      r->t_done = now_s();
      r->done = true;
    }
    sv->pending.clear();
  }
  sv->cv.notify_all();
  sv->admitter.join();
  // admitted requests run to completion; the admitter has stopped adding threads
  for (auto& t : sv->threads) t.join();
  for (auto& kv : sv->requests) delete kv.second;
  delete sv;
}

}  // extern "C"
