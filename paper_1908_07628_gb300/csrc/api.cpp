// Host side of the C ABI declared in include/stem_eels.h: argument checks, beam
// lists, PRISM window lists, device buffers and the launch order of the kernels.
// Compiled with -ffp-contract=off so that the FP64 decisions taken here (beam
// inside an aperture, site inside a probe's PRISM window) are the plain IEEE
// sequence of operations the definitions state.
#include "stem_eels.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

struct eels_ctx {
  int device = 0;
  int assoc = EELS_ASSOC_AUTO;
  int shard_count = 1, shard_index = 0;   // detector-beam shard of eels_inelastic_map
  int sout_scheme = EELS_SOUT_STREAM;     // how S_out reaches each depth
  bool keep_exit = false;                 // builds also store S_in at the exit surface
  int sin_ckpt = 0;                       // builds checkpoint the waves every K slices (K >= 2)
  int64_t operand_budget = (int64_t)8 << 30;   // tensor-core operand buffers of one batch
  int tile_width = 0;                     // GEMM output tile columns: 0 chosen, 128 or 256
  int batch_sites = 0;                    // cap on sites per contraction batch (0: by memory)
  int wait_test = 0;                      // failure test: short pipeline waits, loads withheld
  int check_test = 0;                     // bounds-checked build test: a bad window origin
  // flops of the last map's contraction as grouped (8 per complex product, one product per
  // complex multiply-add whatever the operand split), for per-request metrics
  double last_map_flops = 0;
  // called between tiles of work (after each slice of a build, after each depth of a map);
  // a non-zero return abandons the call with EELS_ERR_CANCELLED (the map server's gate)
  eels::TileHook hook = nullptr;
  void* hook_user = nullptr;
  // measured choice of grouping per contraction shape (EELS_ASSOC_AUTO)
  // measured choice per contraction shape: grouping, and narrow (128-column) tiles for
  // the grouping's first and second GEMM
  struct Choice { int assoc; int narrow1, narrow2; };
  std::map<std::vector<int64_t>, Choice> assoc_cache;
  std::string err;
  std::map<int, float2*> tw;   // device twiddle table exp(-2 pi i k/N), by N
  // kernel timing records (eels_profile_enable)
  bool profiling = false;
  struct Rec { const char* name; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> spare;
  std::map<std::string, std::pair<int64_t, double>> prof_totals;
};

struct eels_smatrix {
  eels_ctx* ctx = nullptr;
  int device = 0;              // freeing the handle must not depend on the context
  int n = 0, n_z = 0, f = 1;
  double cell = 0, lam = 0, sigma = 0, dz = 0, alpha = 0;
  std::vector<int> bp, bq;     // probe beams, f-lattice integer indices
  float2* t = nullptr;         // [n_z][n][n]
  float2* ptab = nullptr;      // [n/2][n/2] box order, forward propagator / N^2
  float2* s_in = nullptr;      // [n_z][n_in][n/2][n/2]
  float2* s_exit = nullptr;    // [n_in][n/2][n/2] exit surface, N Dec(psi_j(n_z)), or null
  // checkpointed form (s_in null): the probe waves psi_j(cK) in row-spectrum form,
  // [ceil(n_z/K)][n_in][n][n/2]; S_in of a segment of K depths is recomputed from them
  int ckpt_k = 0;
  float2* ckpt = nullptr;
  cudaStream_t st = nullptr;   // stream the handle's memory is ordered on
};

namespace {

using eels::launch_col_pass;
using eels::launch_row_pass;

constexpr double kPi = 3.14159265358979323846;

eels_status fail(eels_ctx* ctx, eels_status code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

eels_status cuda_fail(eels_ctx* ctx, cudaError_t e, const char* where) {
  const eels_status code = (e == cudaErrorMemoryAllocation) ? EELS_ERR_OOM : EELS_ERR_CUDA;
  return fail(ctx, code, std::string(where) + ": " + cudaGetErrorString(e));
}

// Brackets one kernel launch with events when the context is profiling.
struct Prof {
  eels_ctx* ctx;
  const char* name;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  Prof(eels_ctx* c, const char* n, cudaStream_t s) : ctx(c), name(n), st(s) {
    if (ctx->profiling) { a = get(); cudaEventRecord(a, st); }
  }
  ~Prof() {
    if (!a) return;
    cudaEvent_t b = get();
    cudaEventRecord(b, st);
    ctx->recs.push_back({name, a, b});
  }
  cudaEvent_t get() {
    if (!ctx->spare.empty()) { cudaEvent_t e = ctx->spare.back(); ctx->spare.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};

// NVTX range over a scope (visible in nsys / ncu timelines; free when no tool attaches).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

// Select the context's device and drop a non-sticky error another library (or an
// unrelated failed call) left on this thread, so that the launch checks of this call
// report only this call's failures.  A sticky error (a faulted context) persists and
// is reported by the next CUDA call anyway.
cudaError_t enter(const eels_ctx* ctx) {
  const cudaError_t e = cudaSetDevice(ctx->device);
  (void)cudaGetLastError();
  return e;
}

#define EELS_CK(call)                                          \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
  } while (0)

// Stream-ordered device buffer freed at scope exit.
template <typename T>
struct DevBuf {
  T* p = nullptr;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { if (p) cudaFreeAsync(p, s); }
  cudaError_t alloc(size_t count, cudaStream_t st) {
    s = st;
    if (count == 0) count = 1;
    return cudaMallocAsync((void**)&p, count * sizeof(T), st);
  }
  cudaError_t upload(const T* host, size_t count, cudaStream_t st) {
    cudaError_t e = alloc(count, st);
    if (e != cudaSuccess || count == 0) return e;
    return cudaMemcpyAsync(p, host, count * sizeof(T), cudaMemcpyHostToDevice, st);
  }
};

// f-lattice beams (p, q), k = f(p, q)/L, with lambda |k| <= angle (Sec. III).
void lattice_beams(int n, double cell, double lam, int f, double angle, std::vector<int>& p,
                   std::vector<int>& q) {
  p.clear();
  q.clear();
  const int pmax = (int)std::ceil(angle * cell / (lam * f)) + 1;
  for (int b = -pmax; b <= pmax; ++b)
    for (int a = -pmax; a <= pmax; ++a)
      if (lam * f * std::sqrt((double)(a * a + b * b)) / cell <= angle) {
        p.push_back(a);
        q.push_back(b);
      }
  (void)n;
}

// Bounds-checked debug build: moves every translation unit's check flag into bit 4 of
// *status (stream-ordered after the call's kernels); nothing in the normal build.
cudaError_t collect_checks(int* status, cudaStream_t st) {
  cudaError_t e;
  if ((e = eels::collect_checks_tc(status, st)) != cudaSuccess) return e;
  if ((e = eels::collect_checks_fp32(status, st)) != cudaSuccess) return e;
  if ((e = eels::collect_checks_ms(status, st)) != cudaSuccess) return e;
  return eels::collect_checks_elastic(status, st);
}

// The same for calls without a status word of their own: EELS_ERR_BOUNDS if a kernel's
// check failed since the flags were last collected.  The flags are per process, so a
// violation is reported by the next checked call on any context.
eels_status checked_status(eels_ctx* ctx, cudaStream_t st) {
#ifdef STEM_CHECK
  DevBuf<int> flag;
  EELS_CK(flag.alloc(1, st));
  EELS_CK(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
  EELS_CK(collect_checks(flag.p, st));
  int h = 0;
  EELS_CK(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  EELS_CK(cudaStreamSynchronize(st));
  if (h & 4) return fail(ctx, EELS_ERR_BOUNDS, "a bounds check of the debug build failed");
#else
  (void)ctx;
  (void)st;
#endif
  return EELS_OK;
}

bool inside_band(int n, int f, const std::vector<int>& p, const std::vector<int>& q) {
  for (size_t i = 0; i < p.size(); ++i) {
    const int64_t k2 = (int64_t)f * f * ((int64_t)p[i] * p[i] + (int64_t)q[i] * q[i]);
    if (16 * k2 >= (int64_t)n * n) return false;
  }
  return true;
}

// PRISM window along one axis: minimum-image s - r in [-L/(2f), L/(2f)).
bool axis_in_window(double s, double r, double cell, int f) {
  double d = s - r;
  d = d - cell * std::floor(d / cell + 0.5);
  const double h = cell / (2 * f);
  return d >= -h && d < h;
}

eels_status twiddles(eels_ctx* ctx, int n, float2** out) {
  auto it = ctx->tw.find(n);
  if (it != ctx->tw.end()) {
    *out = it->second;
    return EELS_OK;
  }
  const int len = eels::twiddle_table_size(n);
  std::vector<float2> h(len);
  eels::fill_twiddle_tables(n, h.data());
  float2* d = nullptr;
  EELS_CK(cudaMalloc((void**)&d, len * sizeof(float2)));
  EELS_CK(cudaMemcpy(d, h.data(), len * sizeof(float2), cudaMemcpyHostToDevice));
  ctx->tw[n] = d;
  *out = d;
  return EELS_OK;
}

eels_status check_specimen(eels_ctx* ctx, const eels_specimen* spec, const eels_optics* op) {
  if (!spec || !op || !spec->vproj) return fail(ctx, EELS_ERR_ARG, "null specimen/optics");
  if (spec->n_z <= 0 || !(spec->cell > 0)) return fail(ctx, EELS_ERR_ARG, "bad n_z or cell");
  if (!eels::grid_supported(spec->n))
    return fail(ctx, EELS_ERR_UNSUPPORTED, "grid size " + std::to_string(spec->n) + " not built");
  if (op->f < 1 || !(op->lambda > 0) || !(op->dz > 0) || !(op->alpha > 0))
    return fail(ctx, EELS_ERR_ARG, "bad optics");
  return EELS_OK;
}

// Transmission functions t_i and the forward propagator table for a specimen.
eels_status build_slices(eels_ctx* ctx, const eels_specimen* spec, const eels_optics* op,
                         cudaStream_t st, float2* t, float2* ptab) {
  const int n = spec->n;
  const int64_t count = (int64_t)spec->n_z * n * n;
  const float* v = spec->vproj;
  DevBuf<float> vtmp;
  if (!spec->vproj_on_device) {
    EELS_CK(vtmp.upload(spec->vproj, (size_t)count, st));
    v = vtmp.p;
  }
  { Prof pr(ctx, "transmission", st); EELS_CK(eels::launch_transmission(v, op->sigma, t, count, st)); }
  EELS_CK(eels::launch_propagator_table(ptab, n, spec->cell, op->lambda, op->dz,
                                        (float)(1.0 / ((double)n * n)), st));
  return EELS_OK;
}

// Tile boundary: true if the hook asks to abandon the call.
bool cancelled(eels_ctx* ctx, int phase, int done, int total) {
  return ctx->hook && ctx->hook(ctx->hook_user, phase, done, total) != 0;
}

}  // namespace

void eels::set_tile_hook(eels_ctx* ctx, TileHook fn, void* user) {
  ctx->hook = fn;
  ctx->hook_user = user;
}

double eels::last_map_flops(const eels_ctx* ctx) { return ctx ? ctx->last_map_flops : 0.0; }

extern "C" {

eels_status eels_create(int device, eels_ctx** out) {
  if (!out) return EELS_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return EELS_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return EELS_ERR_CUDA;
  eels_ctx* c = new eels_ctx();
  c->device = device;
  // keep freed stream-ordered allocations cached between calls
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  *out = c;
  return EELS_OK;
}

void eels_destroy(eels_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  for (auto& kv : ctx->tw) cudaFree(kv.second);
  for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : ctx->spare) cudaEventDestroy(e);
  delete ctx;
  (void)cudaGetLastError();
}

const char* eels_last_error(const eels_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

eels_status eels_set_option(eels_ctx* ctx, int option, int value) {
  if (!ctx) return EELS_ERR_ARG;
  if (option == EELS_OPT_ASSOCIATION) {
    if (value < EELS_ASSOC_AUTO || value > EELS_ASSOC_MODEL)
      return fail(ctx, EELS_ERR_ARG, "unknown association");
    ctx->assoc = value;
    return EELS_OK;
  }
  if (option == EELS_OPT_SOUT_SCHEME) {
    if (value < EELS_SOUT_STREAM || value > EELS_SOUT_INVERSE)
      return fail(ctx, EELS_ERR_ARG, "unknown S_out scheme");
    ctx->sout_scheme = value;
    return EELS_OK;
  }
  if (option == EELS_OPT_TILE_WIDTH) {
    if (value != 0 && value != 128 && value != 256)
      return fail(ctx, EELS_ERR_ARG, "tile width is 0, 128 or 256");
    ctx->tile_width = value;
    return EELS_OK;
  }
  if (option == EELS_OPT_OPERAND_MIB) {
    if (value < 64) return fail(ctx, EELS_ERR_ARG, "operand budget must be >= 64 MiB");
    ctx->operand_budget = (int64_t)value << 20;
    return EELS_OK;
  }
  if (option == EELS_OPT_SIN_CHECKPOINT) {
    if (value < 0) return fail(ctx, EELS_ERR_ARG, "checkpoint interval must be >= 0");
    ctx->sin_ckpt = value >= 2 ? value : 0;
    return EELS_OK;
  }
  if (option == EELS_OPT_EXIT_PLANE) {
    if (value != 0 && value != 1) return fail(ctx, EELS_ERR_ARG, "exit plane option is 0 or 1");
    ctx->keep_exit = value == 1;
    return EELS_OK;
  }
  if (option == EELS_OPT_BATCH_SITES) {
    if (value < 0) return fail(ctx, EELS_ERR_ARG, "batch site cap must be >= 0");
    ctx->batch_sites = value;
    return EELS_OK;
  }
  if (option == EELS_OPT_WAIT_TEST) {
    if (value < 0) return fail(ctx, EELS_ERR_ARG, "wait test value must be >= 0");
    ctx->wait_test = value;
    return EELS_OK;
  }
  if (option == EELS_OPT_CHECK_TEST) {
#ifdef STEM_CHECK
    if (value != 0 && value != 1) return fail(ctx, EELS_ERR_ARG, "check test value is 0 or 1");
    ctx->check_test = value;
    return EELS_OK;
#else
    return fail(ctx, EELS_ERR_UNSUPPORTED, "needs the bounds-checked build (-DSTEM_CHECK)");
#endif
  }
  if (option == EELS_OPT_SHARD_COUNT) {
    if (value < 1) return fail(ctx, EELS_ERR_ARG, "shard count must be >= 1");
    ctx->shard_count = value;
    return EELS_OK;
  }
  if (option == EELS_OPT_SHARD_INDEX) {
    if (value < 0) return fail(ctx, EELS_ERR_ARG, "shard index must be >= 0");
    ctx->shard_index = value;
    return EELS_OK;
  }
  return fail(ctx, EELS_ERR_ARG, "unknown option");
}

eels_status eels_profile_enable(eels_ctx* ctx, int on) {
  if (!ctx) return EELS_ERR_ARG;
  ctx->profiling = on != 0;
  return EELS_OK;
}

int eels_profile_read(eels_ctx* ctx, char* buf, int cap) {
  if (!ctx) return -1;
  cudaSetDevice(ctx->device);
  // fold pending event pairs into the running totals
  for (auto& r : ctx->recs) {
    float ms = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& e = ctx->prof_totals[r.name];
    e.first += 1;
    e.second += ms;
    ctx->spare.push_back(r.a);
    ctx->spare.push_back(r.b);
  }
  ctx->recs.clear();
  std::string out = "{";
  for (auto& kv : ctx->prof_totals) {
    char tmp[256];
    std::snprintf(tmp, sizeof tmp, "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f}",
                  out.size() > 1 ? ", " : "", kv.first.c_str(), (long long)kv.second.first,
                  kv.second.second);
    out += tmp;
  }
  out += "}";
  const int need = (int)out.size() + 1;
  if (buf && cap >= need) {
    std::memcpy(buf, out.c_str(), (size_t)need);
    ctx->prof_totals.clear();   // totals are handed over once, then start again
  } else if (buf && cap > 0) {
    buf[0] = 0;
  }
  return need;
}

int eels_tuning_read(eels_ctx* ctx, char* buf, int cap) {
  if (!ctx) return -1;
  std::string out = "[";
  for (auto& kv : ctx->assoc_cache) {
    const auto& k = kv.first;
    const auto& c = kv.second;
    char tmp[320];
    std::snprintf(tmp, sizeof tmp,
                  "%s{\"precision\": \"%s\", \"n\": %lld, \"n_out\": %lld, \"n_in\": %lld, "
                  "\"w\": %lld, \"nr_max\": %lld, \"n_types\": %lld, \"grouping\": \"%s\", "
                  "\"tile_first\": %d, \"tile_second\": %d}",
                  out.size() > 1 ? ", " : "", k[0] == EELS_TC_BF16X3 ? "bf16x3" : "tf32",
                  (long long)k[1], (long long)k[2], (long long)k[3], (long long)k[4],
                  (long long)k[5], (long long)k[6],
                  c.assoc == EELS_ASSOC_PROBE_FIRST ? "probe_first" : "transition_first",
                  eels::tc_tile_width(c.narrow1), eels::tc_tile_width(c.narrow2));
    out += tmp;
  }
  out += "]";
  const int need = (int)out.size() + 1;
  if (buf && cap >= need) std::memcpy(buf, out.c_str(), (size_t)need);
  else if (buf && cap > 0) buf[0] = 0;
  return need;
}

int eels_checked_build(void) {
#ifdef STEM_CHECK
  return 1;
#else
  return 0;
#endif
}

int eels_count_beams(int n, double cell, double lambda, int f, double angle) {
  if (f < 1 || !(cell > 0) || !(lambda > 0) || angle < 0) return -1;
  std::vector<int> p, q;
  lattice_beams(n, cell, lambda, f, angle, p, q);
  return (int)p.size();
}

eels_status eels_memory_model(int n, int n_z, int planes_in, int planes_out, int64_t out[3]) {
  if (!out || n <= 0 || n % 2 || n_z < 0 || planes_in < 0 || planes_out < 0) return EELS_ERR_ARG;
  const int64_t c = 8;   // bytes of a single-precision complex value
  out[0] = 4 * c * (int64_t)n * n;
  out[1] = c * (int64_t)n_z * n * n;
  out[2] = c * (int64_t)(planes_in + planes_out) * (n / 2) * (n / 2);
  return EELS_OK;
}

int64_t eels_footprint_bytes(int n, int n_z, int n_in, int n_out, int chunk) {
  int64_t mm[3];
  if (eels_memory_model(n, n_z, 0, 0, mm) != EELS_OK || n_in < 0 || n_out < 0 || chunk < 0)
    return -1;
  const int64_t plane = 8 * (int64_t)(n / 2) * (n / 2);
  return mm[1] + plane * ((int64_t)n_z * n_in + n_out) + 2 * 8 * (int64_t)chunk * n * (n / 2);
}

eels_status eels_build_smatrix(eels_ctx* ctx, const eels_specimen* spec, const eels_optics* op,
                               void* stream, eels_smatrix** out) {
  if (!ctx || !out) return EELS_ERR_ARG;
  *out = nullptr;
  Range nvtx_range("eels_build_smatrix");
  eels_status r = check_specimen(ctx, spec, op);
  if (r != EELS_OK) return r;
  EELS_CK(enter(ctx));
  cudaStream_t st = (cudaStream_t)stream;
  const int n = spec->n, nh = n / 2, n_z = spec->n_z;
  std::vector<int> bp, bq;
  lattice_beams(n, spec->cell, op->lambda, op->f, op->alpha, bp, bq);
  if (bp.empty()) return fail(ctx, EELS_ERR_ARG, "no probe beam inside the aperture");
  if (!inside_band(n, op->f, bp, bq))
    return fail(ctx, EELS_ERR_ARG, "probe aperture extends beyond the band limit");
  const int n_in = (int)bp.size();
  float2* tw = nullptr;
  if ((r = twiddles(ctx, n, &tw)) != EELS_OK) return r;

  eels_smatrix* sm = new eels_smatrix();
  sm->ctx = ctx;
  sm->device = ctx->device;
  sm->n = n; sm->n_z = n_z; sm->f = op->f;
  sm->cell = spec->cell; sm->lam = op->lambda; sm->sigma = op->sigma; sm->dz = op->dz;
  sm->alpha = op->alpha;
  sm->bp = bp; sm->bq = bq;
  sm->ckpt_k = ctx->sin_ckpt;
  auto bail = [&](eels_status code) { eels_smatrix_free(sm); return code; };
  const int64_t plane = (int64_t)nh * nh;
  cudaError_t e;
  sm->st = st;
  // stream-ordered: no device-wide synchronisation against other streams' work
  if ((e = cudaMallocAsync((void**)&sm->t, sizeof(float2) * (size_t)n_z * n * n, st)) !=
          cudaSuccess ||
      (e = cudaMallocAsync((void**)&sm->ptab, sizeof(float2) * (size_t)plane, st)) != cudaSuccess ||
      (!ctx->sin_ckpt &&
       (e = cudaMallocAsync((void**)&sm->s_in,
                            sizeof(float2) * (size_t)(n_z * (int64_t)n_in * plane), st)) !=
           cudaSuccess) ||
      (ctx->sin_ckpt &&
       (e = cudaMallocAsync((void**)&sm->ckpt,
                            sizeof(float2) * (size_t)((n_z + ctx->sin_ckpt - 1) / ctx->sin_ckpt) *
                                n_in * n * nh,
                            st)) != cudaSuccess) ||
      (ctx->keep_exit &&
       (e = cudaMallocAsync((void**)&sm->s_exit, sizeof(float2) * (size_t)(n_in * plane), st)) !=
           cudaSuccess))
    return bail(cuda_fail(ctx, e, "S-matrix allocation"));
  if ((r = build_slices(ctx, spec, op, st, sm->t, sm->ptab)) != EELS_OK) return bail(r);

  std::vector<int> px(n_in), py(n_in);
  std::vector<float2> amp(n_in, make_float2(1.f, 0.f));
  for (int j = 0; j < n_in; ++j) { px[j] = op->f * bp[j]; py[j] = op->f * bq[j]; }
  DevBuf<int> dpx, dpy;
  DevBuf<float2> damp, W, Phi;
  if ((e = dpx.upload(px.data(), n_in, st)) != cudaSuccess ||
      (e = dpy.upload(py.data(), n_in, st)) != cudaSuccess ||
      (e = damp.upload(amp.data(), n_in, st)) != cudaSuccess ||
      (e = W.alloc((size_t)n_in * n * nh, st)) != cudaSuccess ||
      (e = Phi.alloc((size_t)n_in * n * nh, st)) != cudaSuccess)
    return bail(cuda_fail(ctx, e, "S_in work buffers"));
  {
    Prof pr(ctx, "init_plane_waves", st);
    if ((e = eels::launch_init_plane_waves(W.p, n, n_in, dpx.p, dpy.p, damp.p, tw, st)) != cudaSuccess)
      return bail(cuda_fail(ctx, e, "init plane waves"));
  }
  const int K = sm->ckpt_k;
  for (int i = 0; i < n_z; ++i) {
    const bool last = (i == n_z - 1) && !sm->s_exit;   // the exit plane needs one more half step
    if (K && i % K == 0) {   // checkpoint psi_j(i), the row pass input of slice i
      e = cudaMemcpyAsync(sm->ckpt + (int64_t)(i / K) * n_in * n * nh, W.p,
                          sizeof(float2) * (size_t)n_in * n * nh, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "checkpoint"));
    }
    if (K && last) break;    // nothing after the last checkpoint is stored
    {
      Prof pr(ctx, "row_pass", st);
      e = launch_row_pass(n, n_in, W.p, Phi.p, sm->t + (int64_t)i * n * n, 0, K ? 0 : 1,
                          K ? nullptr : sm->s_in + (int64_t)i * n_in * plane, K ? 0 : n_in, plane,
                          last ? 0 : 1, tw, st);
    }
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "row pass"));
    if (!last) {
      Prof pr(ctx, "col_pass", st);
      e = launch_col_pass(n, n_in, Phi.p, W.p, sm->ptab, 0, 0, nullptr, nullptr, nullptr, 0.0, tw,
                          st);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "column pass"));
    }
    if (cancelled(ctx, 0, i + 1, n_z)) return bail(fail(ctx, EELS_ERR_CANCELLED, "cancelled"));
  }
  if (sm->s_exit) {   // psi_j(n_z) = F^-1 P F (t psi_j(n_z - 1)) is in W: store N Dec of it
    Prof pr(ctx, "row_pass_store", st);
    e = launch_row_pass(n, n_in, W.p, nullptr, sm->t, 0, 2, sm->s_exit, n_in, plane, 0, tw, st);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "exit plane store"));
  }
  if ((r = checked_status(ctx, st)) != EELS_OK) return bail(r);
  *out = sm;
  return EELS_OK;
}

void eels_smatrix_free(eels_smatrix* sm) {
  if (!sm) return;
  cudaSetDevice(sm->device);
  cudaStreamSynchronize(sm->st);
  if (sm->t) cudaFreeAsync(sm->t, sm->st);
  if (sm->ptab) cudaFreeAsync(sm->ptab, sm->st);
  if (sm->s_exit) cudaFreeAsync(sm->s_exit, sm->st);
  if (sm->ckpt) cudaFreeAsync(sm->ckpt, sm->st);
  if (sm->s_in) cudaFreeAsync(sm->s_in, sm->st);
  delete sm;
  (void)cudaGetLastError();   // a void call leaves no error for the caller's next call
}

eels_status eels_smatrix_info(const eels_smatrix* sm, int* n, int* n_z, int* n_in) {
  if (!sm) return EELS_ERR_ARG;
  if (n) *n = sm->n;
  if (n_z) *n_z = sm->n_z;
  if (n_in) *n_in = (int)sm->bp.size();
  return EELS_OK;
}

eels_status eels_smatrix_beams(const eels_smatrix* sm, int32_t* p, int32_t* q) {
  if (!sm || !p || !q) return EELS_ERR_ARG;
  for (size_t j = 0; j < sm->bp.size(); ++j) { p[j] = sm->bp[j]; q[j] = sm->bq[j]; }
  return EELS_OK;
}

eels_status eels_smatrix_copy_depth(const eels_smatrix* sm, int depth, float* dst, void* stream) {
  if (!sm || !dst || depth < 0 || depth >= sm->n_z) return EELS_ERR_ARG;
  if (!sm->s_in) return EELS_ERR_UNSUPPORTED;   // checkpointed: S_in is not stored
  eels_ctx* ctx = sm->ctx;
  EELS_CK(enter(ctx));
  const int64_t per = (int64_t)sm->bp.size() * (sm->n / 2) * (sm->n / 2);
  EELS_CK(cudaMemcpyAsync(dst, sm->s_in + depth * per, per * sizeof(float2),
                          cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return EELS_OK;
}

namespace {

struct SiteLists {
  std::vector<int> xoff, xcnt, xlist, yoff, ycnt, ylist;
  int max_nr = 0;
};

// A rectangle of the scan: positions ix0 .. ix0 + nx - 1 by iy0 .. iy0 + ny - 1, indexed
// from 0 within it (a scan tile; the whole scan is {0, 0, n_sx, n_sy}).
struct ScanWin {
  int ix0, iy0, nx, ny;
};

SiteLists window_lists(const eels_transitions* tr, const eels_scan* sc, const ScanWin& win,
                       double cell, int f) {
  SiteLists L;
  const int S = tr->n_sites;
  L.xoff.resize(S); L.xcnt.resize(S); L.yoff.resize(S); L.ycnt.resize(S);
  for (int s = 0; s < S; ++s) {
    L.xoff[s] = (int)L.xlist.size();
    for (int ix = 0; ix < win.nx; ++ix)
      if (axis_in_window(tr->x[s], sc->x0 + (double)(win.ix0 + ix) * sc->step_x, cell, f))
        L.xlist.push_back(ix);
    L.xcnt[s] = (int)L.xlist.size() - L.xoff[s];
    L.yoff[s] = (int)L.ylist.size();
    for (int iy = 0; iy < win.ny; ++iy)
      if (axis_in_window(tr->y[s], sc->y0 + (double)(win.iy0 + iy) * sc->step_y, cell, f))
        L.ylist.push_back(iy);
    L.ycnt[s] = (int)L.ylist.size() - L.yoff[s];
    L.max_nr = std::max(L.max_nr, L.xcnt[s] * L.ycnt[s]);
  }
  return L;
}

eels_status check_transitions(eels_ctx* ctx, const eels_transitions* tr, const eels_scan* sc,
                              int n, int n_z) {
  if (!tr || !sc) return fail(ctx, EELS_ERR_ARG, "null transitions/scan");
  if (tr->n_sites < 0 || tr->n_types <= 0 || tr->w < 1 || tr->w > n / 2)
    return fail(ctx, EELS_ERR_ARG, "bad transition sizes (need 1 <= w <= N/2)");
  if (tr->h_shared != 0 && tr->h_shared != 1) return fail(ctx, EELS_ERR_ARG, "bad h_shared");
  if (tr->n_sites > 0 &&
      (!tr->H || !tr->slice || !tr->win_x0 || !tr->win_y0 || !tr->x || !tr->y))
    return fail(ctx, EELS_ERR_ARG, "null transition array");
  for (int s = 0; s < tr->n_sites; ++s) {
    if (tr->slice[s] < 0 || tr->slice[s] >= n_z) return fail(ctx, EELS_ERR_ARG, "site slice out of range");
    if (tr->win_x0[s] < 0 || tr->win_x0[s] >= n / 2 || tr->win_y0[s] < 0 || tr->win_y0[s] >= n / 2)
      return fail(ctx, EELS_ERR_ARG, "window origin outside the N/2 grid");
  }
  if (sc->n_sx <= 0 || sc->n_sy <= 0) return fail(ctx, EELS_ERR_ARG, "empty scan");
  return EELS_OK;
}

}  // namespace

namespace {

// The map over one rectangle of the scan, map_out [n_types][win.ny][win.nx]; the
// arguments are checked by the callers.
eels_status map_window(eels_ctx* ctx, const eels_smatrix* sm, const eels_transitions* tr,
                       const eels_scan* sc, const ScanWin& win, double beta, int precision,
                       double* map_out, int map_on_device, void* stream) {
  eels_status r = EELS_OK;
  bool nonfinite = false;
  ctx->last_map_flops = 0;
  const bool tc = precision != EELS_PREC_FP32;
  const int tc_prec = precision == EELS_PREC_BF16X3 ? EELS_TC_BF16X3 : EELS_TC_TF32;
  EELS_CK(enter(ctx));
  cudaStream_t st = (cudaStream_t)stream;
  const int n = sm->n, nh = n / 2, n_z = sm->n_z, f = sm->f;
  const int n_in = (int)sm->bp.size();
  const int T = tr->n_types, w = tr->w, S = tr->n_sites;
  const int64_t plane = (int64_t)nh * nh;
  const int64_t n_map = (int64_t)T * win.nx * win.ny;

  std::vector<int> dp, dq;
  lattice_beams(n, sm->cell, sm->lam, f, beta, dp, dq);
  if (dp.empty()) return fail(ctx, EELS_ERR_ARG, "no detector beam inside beta");
  if (!inside_band(n, f, dp, dq))
    return fail(ctx, EELS_ERR_ARG, "detector aperture extends beyond the band limit");
  if (ctx->shard_index >= ctx->shard_count)
    return fail(ctx, EELS_ERR_ARG, "shard index not below the shard count");
  if (ctx->shard_count > 1) {   // keep beams d with d mod G == g
    size_t k = 0;
    for (size_t d = (size_t)ctx->shard_index; d < dp.size(); d += (size_t)ctx->shard_count, ++k) {
      dp[k] = dp[d];
      dq[k] = dq[d];
    }
    dp.resize(k);
    dq.resize(k);
    if (dp.empty()) {   // nothing of this shard: the map is zero
      if (map_on_device) EELS_CK(cudaMemsetAsync(map_out, 0, sizeof(double) * n_map, st));
      else std::memset(map_out, 0, sizeof(double) * n_map);
      return EELS_OK;
    }
  }
  const int n_out = (int)dp.size();
  float2* tw = nullptr;
  if ((r = twiddles(ctx, n, &tw)) != EELS_OK) return r;

  // PRISM windows and the transitions of each slice (sites reached by some probe)
  SiteLists L = window_lists(tr, sc, win, sm->cell, f);
  std::vector<std::vector<int>> tr_site(n_z), tr_type(n_z);
  for (int s = 0; s < S; ++s) {
    if (L.xcnt[s] == 0 || L.ycnt[s] == 0) continue;
    for (int m = 0; m < T; ++m) {
      tr_site[tr->slice[s]].push_back(s);
      tr_type[tr->slice[s]].push_back(m);
    }
  }

  DevBuf<float2> dH, Sout, W, Phi, M, ax, ay, damp;
  DevBuf<int> dwx, dwy, dxoff, dxcnt, dxlist, dyoff, dycnt, dylist, dpx, dpy, dbp, dbq, dts, dtt;
  DevBuf<double> dmap;
  const float2* H = (const float2*)tr->H;
  const int h_mul = tr->h_shared ? 0 : 1;
  const size_t hcount = (size_t)(tr->h_shared ? 1 : S) * T * w * w;
  if (!tr->on_device) {
    EELS_CK(dH.upload((const float2*)tr->H, hcount, st));
    H = dH.p;
  }
  EELS_CK(dwx.upload(tr->win_x0, S, st));
  EELS_CK(dwy.upload(tr->win_y0, S, st));
#ifdef STEM_CHECK
  if (ctx->check_test) {   // origin N/2 for the first site some probe reaches; a periodic
    int s0 = 0;              // walk from there still stays inside the plane
    while (s0 < S && (L.xcnt[s0] == 0 || L.ycnt[s0] == 0)) ++s0;
    if (s0 < S) {
      const int bad = nh;
      EELS_CK(cudaMemcpyAsync(dwx.p + s0, &bad, sizeof(int), cudaMemcpyHostToDevice, st));
      EELS_CK(cudaStreamSynchronize(st));
    }
  }
#endif
  EELS_CK(dxoff.upload(L.xoff.data(), S, st));
  EELS_CK(dxcnt.upload(L.xcnt.data(), S, st));
  EELS_CK(dxlist.upload(L.xlist.data(), L.xlist.size(), st));
  EELS_CK(dyoff.upload(L.yoff.data(), S, st));
  EELS_CK(dycnt.upload(L.ycnt.data(), S, st));
  EELS_CK(dylist.upload(L.ylist.data(), L.ylist.size(), st));
  EELS_CK(dbp.upload(sm->bp.data(), n_in, st));
  EELS_CK(dbq.upload(sm->bq.data(), n_in, st));
  EELS_CK(ax.alloc((size_t)n_in * win.nx, st));
  EELS_CK(ay.alloc((size_t)n_in * win.ny, st));
  EELS_CK(eels::launch_phase_table(ax.p, dbp.p, n_in, f, sm->cell, sc->x0, sc->step_x, win.nx, st,
                                   0, win.ix0));
  EELS_CK(eels::launch_phase_table(ay.p, dbq.p, n_in, f, sm->cell, sc->y0, sc->step_y, win.ny, st,
                                   0, win.iy0));
  DevBuf<float2> axT, ayT;   // [pos][n_in]: the tensor-core gathers read along the beams
  if (tc) {
    EELS_CK(axT.alloc((size_t)n_in * win.nx, st));
    EELS_CK(ayT.alloc((size_t)n_in * win.ny, st));
    EELS_CK(eels::launch_phase_table(axT.p, dbp.p, n_in, f, sm->cell, sc->x0, sc->step_x,
                                     win.nx, st, 1, win.ix0));
    EELS_CK(eels::launch_phase_table(ayT.p, dbq.p, n_in, f, sm->cell, sc->y0, sc->step_y,
                                     win.ny, st, 1, win.iy0));
  }

  // flattened transition lists of all slices
  std::vector<int> all_site, all_type, slice_off(n_z + 1, 0);
  for (int i = 0; i < n_z; ++i) {
    slice_off[i] = (int)all_site.size();
    all_site.insert(all_site.end(), tr_site[i].begin(), tr_site[i].end());
    all_type.insert(all_type.end(), tr_type[i].begin(), tr_type[i].end());
  }
  slice_off[n_z] = (int)all_site.size();
  EELS_CK(dts.upload(all_site.data(), all_site.size(), st));
  EELS_CK(dtt.upload(all_type.data(), all_type.size(), st));

  // detector plane waves at the exit surface, carried back by conj(P) first:
  // beta_d(n_z - 1) = conj(P(k_d)) |k_d>
  std::vector<int> px(n_out), py(n_out);
  std::vector<float2> amp(n_out);
  for (int d = 0; d < n_out; ++d) {
    px[d] = f * dp[d];
    py[d] = f * dq[d];
    double a = sm->lam * sm->dz * (double)((int64_t)px[d] * px[d] + (int64_t)py[d] * py[d]) /
               (sm->cell * sm->cell);
    a -= 2.0 * std::floor(0.5 * a);
    amp[d] = make_float2((float)std::cos(kPi * a), (float)std::sin(kPi * a));
  }
  EELS_CK(dpx.upload(px.data(), n_out, st));
  EELS_CK(dpy.upload(py.data(), n_out, st));
  EELS_CK(damp.upload(amp.data(), n_out, st));
  EELS_CK(Sout.alloc((size_t)n_out * plane, st));
  EELS_CK(W.alloc((size_t)n_out * n * nh, st));
  EELS_CK(Phi.alloc((size_t)n_out * n * nh, st));
  EELS_CK(dmap.alloc((size_t)n_map, st));
  EELS_CK(cudaMemsetAsync(dmap.p, 0, sizeof(double) * n_map, st));
  // checkpointed S-matrix: forward work arrays and one segment of K depths of S_in
  const int K = sm->ckpt_k;
  DevBuf<float2> Wf, Phif, seg;
  if (sm->ckpt) {
    if (ctx->sout_scheme != EELS_SOUT_STREAM)
      return fail(ctx, EELS_ERR_UNSUPPORTED, "a checkpointed S-matrix needs the stream scheme");
    EELS_CK(Wf.alloc((size_t)n_in * n * nh, st));
    EELS_CK(Phif.alloc((size_t)n_in * n * nh, st));
    EELS_CK(seg.alloc((size_t)K * n_in * plane, st));
  }

  // M buffer: a batch of transitions, at most ~1 GiB
  const int64_t m_stride = (int64_t)n_out * n_in;
  int max_tr = 0;
  for (int i = 0; i < n_z; ++i) max_tr = std::max(max_tr, (int)tr_site[i].size());
  const int batch = (int)std::max<int64_t>(1, std::min<int64_t>(
      std::max(max_tr, 1), (int64_t)(1 << 30) / (m_stride * (int64_t)sizeof(float2))));
  if (!tc) EELS_CK(M.alloc((size_t)batch * m_stride, st));

  // tensor-core path: sites of a slice in batches of `sb` slots
  auto rup = [](int64_t v, int64_t m) { return (v + m - 1) / m * m; };
  const int kal = eels::tc_k_align(tc_prec);
  const int k1p = (int)rup(2 * (int64_t)w * w, kal), k2p = (int)rup(2 * (int64_t)n_in, kal);
  const int nr_cap = std::max(L.max_nr, 1);
  std::vector<std::vector<int>> slice_sites(n_z);
  for (int s = 0; s < S; ++s)
    if (L.xcnt[s] > 0 && L.ycnt[s] > 0) slice_sites[tr->slice[s]].push_back(s);
  // AUTO: measured once per shape (both groupings timed on the first occupied slice)
  const std::vector<int64_t> shape_key = {tc_prec, n, n_out, n_in, w, nr_cap, T};
  int chosen = ctx->assoc;
  // complex products of each grouping over the map's sites (Eq. SHn0 applied to the probes)
  double c_tr = 0, c_pr = 0;
  {
    const double P2 = (double)w * w;
    for (int s = 0; s < S; ++s) {
      const double nr = (double)L.xcnt[s] * L.ycnt[s];
      if (nr == 0) continue;
      c_tr += T * ((double)n_out * P2 * n_in + (double)n_out * n_in * nr);
      c_pr += nr * n_in * P2 + T * (double)n_out * P2 * nr;
    }
  }
  if (chosen == EELS_ASSOC_MODEL)   // the smaller one, with no timing: never load-dependent
    chosen = c_pr <= c_tr ? EELS_ASSOC_PROBE_FIRST : EELS_ASSOC_TRANSITION_FIRST;
  // tile widths: the narrow tile when it covers the GEMM's columns with at least 5 % fewer
  // padded columns (the rule when nothing is measured); per grouping, first and second GEMM
  auto padded = [](int64_t cols, int64_t wd) { return (cols + wd - 1) / wd * wd; };
  int narrow[2][2] = {};   // [grouping: 0 transition first, 1 probe first][GEMM 1st / 2nd]
  {
    int64_t cw = 0, cn = 0;   // second GEMM (GEMM 2 / GEMM-V): 2 n_R columns per transition
    for (int s = 0; s < S; ++s) {
      const int64_t nr = (int64_t)L.xcnt[s] * L.ycnt[s];
      if (nr == 0) continue;
      cw += T * padded(2 * nr, eels::tc_tile_width(0));
      cn += T * padded(2 * nr, eels::tc_tile_width(1));
    }
    const bool n2 = cn < 0.95 * cw;
    narrow[0][1] = narrow[1][1] = n2 ? 1 : 0;
    auto pick = [&](int64_t cols) {
      return padded(cols, eels::tc_tile_width(1)) < 0.95 * padded(cols, eels::tc_tile_width(0));
    };
    narrow[0][0] = pick(k2p) ? 1 : 0;   // GEMM 1: 2 n_in columns
    narrow[1][0] = pick(k1p) ? 1 : 0;   // GEMM-Y: 2 w^2 columns
    if (ctx->tile_width)                 // a width set by the caller wins
      for (auto& row : narrow) row[0] = row[1] = ctx->tile_width == 128 ? 1 : 0;
  }
  if (chosen == EELS_ASSOC_AUTO) {
    auto it = ctx->assoc_cache.find(shape_key);
    if (it != ctx->assoc_cache.end()) {
      chosen = it->second.assoc;
      const int gi = chosen == EELS_ASSOC_PROBE_FIRST ? 1 : 0;
      if (!ctx->tile_width) {
        narrow[gi][0] = it->second.narrow1;
        narrow[gi][1] = it->second.narrow2;
      }
    }
  }
  bool tune = tc && chosen == EELS_ASSOC_AUTO;
  const bool need_tr = tune || chosen == EELS_ASSOC_TRANSITION_FIRST;
  const bool need_pr = tune || chosen == EELS_ASSOC_PROBE_FIRST;
  const int vbytes = tc ? eels::tc_value_bytes(tc_prec) : 4;   // operand bytes per value
  const int vf = vbytes / 4;                                      // ... in floats
  const int64_t per_site =
      vbytes * ((int64_t)n_out * k1p +
           (need_pr ? (int64_t)nr_cap * k2p + (int64_t)k1p * k2p + (int64_t)T * 2 * nr_cap * k1p
                    : 0) +
           (need_tr ? (int64_t)T * 2 * n_in * k1p + (int64_t)T * n_out * k2p +
                          (int64_t)2 * nr_cap * k2p
                    : 0));
  int max_sites = 0;
  for (int i = 0; i < n_z; ++i) max_sites = std::max(max_sites, (int)slice_sites[i].size());
  int sb = (int)std::max<int64_t>(1, std::min<int64_t>(std::max(max_sites, 1),
                                                       ctx->operand_budget / per_site));
  if (ctx->batch_sites > 0) sb = std::min(sb, ctx->batch_sites);
  DevBuf<float> A1, B1, M1, B2, AY, BY, BV;
  DevBuf<int> dslot, dzs, dzt, dab1, dbb1, dnv1, dab2, dbb2, dnv2, dstatus, daby, dnvy, dnry;
  DevBuf<double> dscratch;
  std::vector<int> slot_all, zs_all, zt_all, nv2_all, nr_all, site_off(n_z + 1, 0);
  std::vector<int> pv_all[2], py_all[2];   // [0]: 256-column tiles, [1]: 128-column tiles
  DevBuf<int> dtile_v[2], dtile_y[2];
  if (tc) {
    for (int i = 0; i < n_z; ++i) {
      site_off[i] = (int)slot_all.size();
      for (int s : slice_sites[i]) {
        slot_all.push_back(s);
        nr_all.push_back(L.xcnt[s] * L.ycnt[s]);
        for (int m = 0; m < T; ++m) {
          zs_all.push_back(s);
          zt_all.push_back(m);
          nv2_all.push_back(2 * L.xcnt[s] * L.ycnt[s]);
        }
      }
    }
    site_off[n_z] = (int)slot_all.size();
    // prefix sums of the tiles with work, over all transitions (GEMM 2 / GEMM-V: column
    // tiles of 2 n_R x every row tile of n_out) and over all sites (GEMM-Y: row tiles of
    // n_R x every column tile of 2 w^2); a batch reads its slice of them
    // (for both tile widths: the autotuner may time both)
    const int64_t gy_v = (n_out + 127) / 128;
    for (int nw = 0; nw < 2; ++nw) {
      const int64_t wd = eels::tc_tile_width(nw), gx_y = (k1p + wd - 1) / wd;
      pv_all[nw].assign(nv2_all.size() + 1, 0);
      for (size_t z = 0; z < nv2_all.size(); ++z)
        pv_all[nw][z + 1] = pv_all[nw][z] + (int)(((int64_t)nv2_all[z] + wd - 1) / wd * gy_v);
      py_all[nw].assign(nr_all.size() + 1, 0);
      for (size_t q = 0; q < nr_all.size(); ++q)
        py_all[nw][q + 1] = py_all[nw][q] + (int)(((int64_t)nr_all[q] + 127) / 128 * gx_y);
    }
    std::vector<int> ab1(sb * T), bb1(sb * T), nv1(sb * T, k2p), ab2(sb * T), bb2(sb * T);
    for (int z = 0; z < sb * T; ++z) { ab1[z] = z / T; bb1[z] = z; ab2[z] = z; bb2[z] = z / T; }
    EELS_CK(dslot.upload(slot_all.data(), slot_all.size(), st));
    EELS_CK(dzs.upload(zs_all.data(), zs_all.size(), st));
    EELS_CK(dzt.upload(zt_all.data(), zt_all.size(), st));
    EELS_CK(dnv2.upload(nv2_all.data(), nv2_all.size(), st));
    for (int nw = 0; nw < 2; ++nw) {
      EELS_CK(dtile_v[nw].upload(pv_all[nw].data(), pv_all[nw].size(), st));
      EELS_CK(dtile_y[nw].upload(py_all[nw].data(), py_all[nw].size(), st));
    }
    EELS_CK(dab1.upload(ab1.data(), ab1.size(), st));
    EELS_CK(dbb1.upload(bb1.data(), bb1.size(), st));
    EELS_CK(dnv1.upload(nv1.data(), nv1.size(), st));
    EELS_CK(dab2.upload(ab2.data(), ab2.size(), st));
    EELS_CK(dbb2.upload(bb2.data(), bb2.size(), st));
    EELS_CK(dstatus.alloc(1, st));
    EELS_CK(cudaMemsetAsync(dstatus.p, 0, sizeof(int), st));
    EELS_CK(A1.alloc((size_t)vf * sb * n_out * k1p, st));
    if (need_pr) {
      std::vector<int> aby(sb), nvy(sb, k1p);
      for (int q = 0; q < sb; ++q) aby[q] = q;
      EELS_CK(daby.upload(aby.data(), aby.size(), st));
      EELS_CK(dnvy.upload(nvy.data(), nvy.size(), st));
      EELS_CK(dnry.upload(nr_all.data(), nr_all.size(), st));
      EELS_CK(AY.alloc((size_t)vf * sb * nr_cap * k2p, st));
      EELS_CK(BY.alloc((size_t)vf * sb * k1p * k2p, st));
      EELS_CK(BV.alloc((size_t)vf * sb * T * 2 * nr_cap * k1p, st));
    }
    if (need_tr) {
      EELS_CK(B1.alloc((size_t)vf * sb * T * 2 * n_in * k1p, st));
      EELS_CK(M1.alloc((size_t)vf * sb * T * n_out * k2p, st));
      EELS_CK(B2.alloc((size_t)vf * sb * 2 * nr_cap * k2p, st));
    }
    if (tune) EELS_CK(dscratch.alloc((size_t)n_map, st));
  }

  {
    Prof pr(ctx, "init_plane_waves", st);
    EELS_CK(eels::launch_init_plane_waves(W.p, n, n_out, dpx.p, dpy.p, damp.p, tw, st));
  }
  eels::WindowLists wl{dxoff.p, dxcnt.p, dxlist.p, dyoff.p, dycnt.p, dylist.p, L.max_nr};
  // tensor-core contraction of slice i with one grouping, accumulated into `map`
  // assoc: EELS_ASSOC_TRANSITION_FIRST or EELS_ASSOC_PROBE_FIRST; n1, n2: narrow tiles for
  // the first / second GEMM; timed (autotuner): event pairs around every GEMM launch,
  // [0] first GEMM, [1] second GEMM
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tev[2];
  auto timed_launch = [&](int which, bool timed, auto&& fn) -> cudaError_t {
    cudaEvent_t a = nullptr, b2 = nullptr;
    if (timed) {
      cudaEventCreate(&a);
      cudaEventCreate(&b2);
      cudaEventRecord(a, st);
    }
    const cudaError_t e = fn();
    if (timed) {
      cudaEventRecord(b2, st);
      tev[which].push_back({a, b2});
    }
    return e;
  };
  auto contract_slice = [&](const float2* Sin, int i, int assoc, int n1, int n2, double* map,
                            bool timed = false) -> eels_status {
    for (int q0 = site_off[i]; q0 < site_off[i + 1]; q0 += sb) {
      const int ns = std::min(sb, site_off[i + 1] - q0);
      eels::TcBatch b{};
      b.prec = tc_prec;
      b.Sout = Sout.p; b.Sin = Sin; b.nh = nh; b.n_out = n_out; b.n_in = n_in; b.w = w;
      b.n_types = T; b.H = H; b.h_mul = h_mul; b.wx = dwx.p; b.wy = dwy.p;
      b.slot_site = dslot.p + q0; b.z_site = dzs.p + (int64_t)q0 * T;
      b.z_type = dzt.p + (int64_t)q0 * T; b.n_sites = ns; b.slots_cap = sb;
      b.k1p = k1p; b.k2p = k2p; b.A1 = A1.p; b.B1 = B1.p; b.M1 = M1.p; b.B2 = B2.p;
      b.ax = ax.p; b.ay = ay.p; b.n_sx = win.nx; b.n_sy = win.ny;
      b.axT = axT.p; b.ayT = ayT.p;
      b.bn_first = eels::tc_tile_width(n1);
      b.bn_second = eels::tc_tile_width(n2);
      b.tiles_v = dtile_v[n2].p + (int64_t)q0 * T;
      b.n_tiles_v = pv_all[n2][(size_t)(q0 + ns) * T] - pv_all[n2][(size_t)q0 * T];
      b.tiles_y = dtile_y[n1].p + q0;
      b.n_tiles_y = py_all[n1][q0 + ns] - py_all[n1][q0];
      b.xoff = dxoff.p; b.xcnt = dxcnt.p; b.xlist = dxlist.p;
      b.yoff = dyoff.p; b.ycnt = dycnt.p; b.ylist = dylist.p; b.nr_cap = nr_cap;
      b.a_batch1 = dab1.p; b.b_batch1 = dbb1.p; b.n_valid1 = dnv1.p;
      b.a_batch2 = dab2.p; b.b_batch2 = dbb2.p; b.n_valid2 = dnv2.p + (int64_t)q0 * T;
      b.map = map; b.status = dstatus.p;
      b.wait_cycles = ctx->wait_test > 0 ? 1000LL * ctx->wait_test : 0;
      b.withhold = ctx->wait_test > 0 ? 1 : 0;
      b.AY = AY.p; b.BY = BY.p; b.BV = BV.p; b.a_batch_y = daby.p; b.n_valid_y = dnvy.p;
      b.m_valid_y = dnry.p ? dnry.p + q0 : nullptr;
      const bool bf = tc_prec == EELS_TC_BF16X3;
      if (assoc == EELS_ASSOC_PROBE_FIRST) {
        {
          Prof pr(ctx, "tc_gather_y", st);
          EELS_CK(eels::tc_gather_y(b, st));
        }
        {
          Prof pr(ctx, bf ? "gemm_y_bf16x3" : "gemm_y_tf32", st);
          EELS_CK(timed_launch(0, timed, [&] { return eels::tc_gemm_y(b, st); }));
        }
        {
          Prof pr(ctx, bf ? "gemm_v_abs2_bf16x3" : "gemm_v_abs2_tf32", st);
          EELS_CK(timed_launch(1, timed, [&] { return eels::tc_gemm_v(b, st); }));
        }
      } else {
        {
          Prof pr(ctx, "tc_gather", st);
          EELS_CK(eels::tc_gather(b, st));
        }
        {
          Prof pr(ctx, bf ? "gemm1_bf16x3" : "gemm1_tf32", st);
          EELS_CK(timed_launch(0, timed, [&] { return eels::tc_gemm1(b, st); }));
        }
        {
          Prof pr(ctx, bf ? "gemm2_abs2_bf16x3" : "gemm2_abs2_tf32", st);
          EELS_CK(timed_launch(1, timed, [&] { return eels::tc_gemm2(b, st); }));
        }
      }
    }
    return EELS_OK;
  };
  // contraction of depth i (S_out(i) in Sout) into the map
  auto contract_depth = [&](int i) -> eels_status {
    Range nvtx_depth("contract depth");
    const float2* Sin = sm->ckpt ? seg.p + (int64_t)(i % K) * n_in * plane
                                 : sm->s_in + (int64_t)i * n_in * plane;
    if (tc && site_off[i + 1] > site_off[i]) {
      eels_status r1 = EELS_OK;
      if (tune) {
        // Each grouping with both tile widths on this slice (scratch map, one warm-up run
        // each, then one timed run with events around every GEMM launch): per grouping
        // the faster width of each of its two GEMMs, then the grouping whose gathers and
        // GEMMs take least.  The slice then goes once into the map with that choice.
        const int groupings[2] = {EELS_ASSOC_TRANSITION_FIRST, EELS_ASSOC_PROBE_FIRST};
        float best_total = -1.f;
        int best_g = 0;
        for (int gi = 0; gi < 2; ++gi) {
          float tg[2][2] = {}, t_all[2] = {};   // [width][first, second GEMM]; whole slice
          const int nw0 = ctx->tile_width ? narrow[gi][0] : 0;
          const int nw1 = ctx->tile_width ? narrow[gi][0] : 1;
          for (int nw = nw0; nw <= nw1; ++nw) {
            if ((r1 = contract_slice(Sin, i, groupings[gi], nw, nw, dscratch.p)) != EELS_OK)
              return r1;
            cudaEvent_t e0, e1;
            EELS_CK(cudaEventCreate(&e0));
            EELS_CK(cudaEventCreate(&e1));
            EELS_CK(cudaEventRecord(e0, st));
            r1 = contract_slice(Sin, i, groupings[gi], nw, nw, dscratch.p, true);
            EELS_CK(cudaEventRecord(e1, st));
            EELS_CK(cudaEventSynchronize(e1));
            cudaEventElapsedTime(&t_all[nw], e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            for (int k = 0; k < 2; ++k) {
              for (auto& pr : tev[k]) {
                float t = 0.f;
                cudaEventElapsedTime(&t, pr.first, pr.second);
                tg[nw][k] += t;
                cudaEventDestroy(pr.first);
                cudaEventDestroy(pr.second);
              }
              tev[k].clear();
            }
            if (r1 != EELS_OK) return r1;
          }
          if (!ctx->tile_width) {
            narrow[gi][0] = tg[1][0] < tg[0][0] ? 1 : 0;
            narrow[gi][1] = tg[1][1] < tg[0][1] ? 1 : 0;
          }
          const float rest = t_all[nw0] - tg[nw0][0] - tg[nw0][1];   // gathers, launch gaps
          const float total = rest + tg[narrow[gi][0]][0] + tg[narrow[gi][1]][1];
          if (best_total < 0.f || total < best_total) {
            best_total = total;
            best_g = gi;
          }
        }
        chosen = groupings[best_g];
        ctx->assoc_cache[shape_key] = {chosen, narrow[best_g][0], narrow[best_g][1]};
        tune = false;
      }
      const int gi = chosen == EELS_ASSOC_PROBE_FIRST ? 1 : 0;
      if ((r1 = contract_slice(Sin, i, chosen, narrow[gi][0], narrow[gi][1], dmap.p)) !=
          EELS_OK)
        return r1;
    }
    for (int b0 = slice_off[i]; !tc && b0 < slice_off[i + 1]; b0 += batch) {
      eels::TransitionBatch tb{dts.p + b0, dtt.p + b0, std::min(batch, slice_off[i + 1] - b0)};
      {
        Prof pr(ctx, "gemm1_fp32", st);
        EELS_CK(eels::launch_gemm1_fp32(Sout.p, Sin, nh, n_out, n_in, w, H, T, h_mul, tb, dwx.p,
                                        dwy.p, M.p, m_stride, st));
      }
      {
        Prof pr(ctx, "gemm2_abs2_fp32", st);
        EELS_CK(eels::launch_gemm2_abs2_fp32(M.p, m_stride, n_out, n_in, ax.p, ay.p, win.nx,
                                             win.ny, tb, wl, dmap.p, st));
      }
    }
    return EELS_OK;
  };
  const auto t_of = [&](int i) { return sm->t + (int64_t)i * n * n; };
  const auto has_work = [&](int i) { return slice_off[i + 1] > slice_off[i]; };
  // some depth of the segment whose top depth is i holds transitions
  const auto has_work_to = [&](int i) {
    for (int j = i / K * K; j <= i; ++j)
      if (has_work(j)) return true;
    return false;
  };
  // one backward slice step of the detector waves in `from` (row-spectrum form):
  // conj(t_i), x-FFT, then y-FFT, conj(P), inverse y-FFT into `to`
  auto back_step = [&](float2* from, float2* tmp, int i) -> eels_status {
    {
      Prof pr(ctx, "row_pass_adjoint", st);
      EELS_CK(launch_row_pass(n, n_out, from, tmp, t_of(i), 1, 0, nullptr, 0, 0, 1, tw, st));
    }
    Prof pr(ctx, "col_pass_adjoint", st);
    EELS_CK(launch_col_pass(n, n_out, tmp, from, sm->ptab, 1, 0, nullptr, nullptr, nullptr, 0.0,
                            tw, st));
    return EELS_OK;
  };
  // S_out(i) = N Dec(wave) of the waves in `from`, nothing else
  auto store_sout = [&](const float2* from, int i) -> eels_status {
    Prof pr(ctx, "row_pass_store", st);
    EELS_CK(launch_row_pass(n, n_out, from, nullptr, t_of(i), 1, 2, Sout.p, n_out, plane, 0, tw,
                            st));
    return EELS_OK;
  };

  // checkpointed S-matrix: S_in(cK .. i) of the segment whose top depth is i, recomputed
  // from the checkpoint psi_j(cK) with the same row and column passes as the build
  auto recompute_segment = [&](int i) -> eels_status {
    Range nvtx_seg("S_in segment recompute");
    const int c0 = i / K * K;
    EELS_CK(cudaMemcpyAsync(Wf.p, sm->ckpt + (int64_t)(i / K) * n_in * n * nh,
                            sizeof(float2) * (size_t)n_in * n * nh, cudaMemcpyDeviceToDevice, st));
    for (int j = c0; j <= i; ++j) {
      {
        Prof pr(ctx, "row_pass_recompute", st);
        EELS_CK(launch_row_pass(n, n_in, Wf.p, Phif.p, t_of(j), 0, 1,
                                seg.p + (int64_t)(j - c0) * n_in * plane, n_in, plane,
                                j < i ? 1 : 0, tw, st));
      }
      if (j < i) {
        Prof pr(ctx, "col_pass_recompute", st);
        EELS_CK(launch_col_pass(n, n_in, Phif.p, Wf.p, sm->ptab, 0, 0, nullptr, nullptr, nullptr,
                                0.0, tw, st));
      }
    }
    return EELS_OK;
  };

  eels_status rs = EELS_OK;
  if (ctx->sout_scheme == EELS_SOUT_STREAM) {
    // S_out streamed backwards once (Alg. 2 with the slice loop run from the exit)
    for (int i = n_z - 1; i >= 0; --i) {
      if (sm->ckpt && (i == n_z - 1 || (i + 1) % K == 0) && has_work_to(i))
        if ((rs = recompute_segment(i)) != EELS_OK) return rs;
      // S_out(i) = N Dec beta(i), stored only where depth i holds transitions; then
      // conj(t_i) and the forward x-FFT for level i-1
      const int store = has_work(i) ? 2 : 0;
      if (store || i > 0) {
        Prof pr(ctx, "row_pass_adjoint", st);
        EELS_CK(launch_row_pass(n, n_out, W.p, Phi.p, t_of(i), 1, store, Sout.p, n_out, plane,
                                i > 0 ? 1 : 0, tw, st));
      }
      if ((rs = contract_depth(i)) != EELS_OK) return rs;
      if (i > 0) {
        Prof pr(ctx, "col_pass_adjoint", st);
        EELS_CK(launch_col_pass(n, n_out, Phi.p, W.p, sm->ptab, 1, 0, nullptr, nullptr, nullptr,
                                0.0, tw, st));
      }
      if (cancelled(ctx, 1, n_z - i, n_z)) return fail(ctx, EELS_ERR_CANCELLED, "cancelled");
    }
  } else if (ctx->sout_scheme == EELS_SOUT_RECOMPUTE) {
    // Alg. 2 as listed: S_2 recalculated from the exit surface for every depth
    for (int i = 0; i < n_z; ++i) {
      if (!has_work(i)) continue;
      {
        Prof pr(ctx, "init_plane_waves", st);
        EELS_CK(eels::launch_init_plane_waves(W.p, n, n_out, dpx.p, dpy.p, damp.p, tw, st));
      }
      for (int j = n_z - 1; j > i; --j)
        if ((rs = back_step(W.p, Phi.p, j)) != EELS_OK) return rs;
      if ((rs = store_sout(W.p, i)) != EELS_OK) return rs;
      if ((rs = contract_depth(i)) != EELS_OK) return rs;
      if (cancelled(ctx, 1, i + 1, n_z)) return fail(ctx, EELS_ERR_CANCELLED, "cancelled");
    }
  } else {
    // Sec. IV C: S_2 carried back to depth 0 once, then retreated one slice per depth
    // with the inverse step (P, then t_{i+1}) and projected onto the band
    // scales: a column pass multiplies by N x its table, a row pass by N; the retreat
    // starts from a wave at true scale, so col(P / N^2) -> 1/N, row -> 1, and the band
    // table carries 1/N to end at true scale again
    DevBuf<float2> mtab;
    EELS_CK(mtab.alloc((size_t)plane, st));
    EELS_CK(eels::launch_propagator_table(mtab.p, n, sm->cell, sm->lam, 0.0,
                                          (float)(1.0 / (double)n), st));
    float2* cur = W.p;
    float2* oth = Phi.p;
    for (int j = n_z - 1; j > 0; --j)
      if ((rs = back_step(cur, oth, j)) != EELS_OK) return rs;
    for (int i = 0; i < n_z; ++i) {
      if (has_work(i)) {
        if ((rs = store_sout(cur, i)) != EELS_OK) return rs;
        if ((rs = contract_depth(i)) != EELS_OK) return rs;
      }
      if (cancelled(ctx, 1, i + 1, n_z)) return fail(ctx, EELS_ERR_CANCELLED, "cancelled");
      if (i + 1 == n_z) break;
      {
        Prof pr(ctx, "col_pass_inverse", st);
        EELS_CK(launch_col_pass(n, n_out, cur, oth, sm->ptab, 0, 0, nullptr, nullptr, nullptr,
                                0.0, tw, st));
      }
      {
        Prof pr(ctx, "row_pass_inverse", st);
        EELS_CK(launch_row_pass(n, n_out, oth, cur, t_of(i + 1), 0, 0, nullptr, 0, 0, 1, tw, st));
      }
      {
        Prof pr(ctx, "col_pass_band", st);
        EELS_CK(launch_col_pass(n, n_out, cur, oth, mtab.p, 0, 0, nullptr, nullptr, nullptr, 0.0,
                                tw, st));
      }
      std::swap(cur, oth);
    }
  }
  // I = f^2 (f^2/n_in) (4/N^2)^2 sum |M_gpu a_gpu|^2: S-matrices are stored scaled
  // by N, S_out carries the factor 4 of the half-grid inner product, and the probe
  // coefficients carry c = f/sqrt(n_in).
  ctx->last_map_flops = 8.0 * ((tc && chosen == EELS_ASSOC_PROBE_FIRST) ? c_pr : c_tr);
  const double nn = (double)n * (double)n;
  const double scale = (double)f * f * ((double)f * f / n_in) * 16.0 / (nn * nn);
  // device status: bit 1 a bounded tensor-core wait timed out, bit 2 the map holds NaN or
  // Inf (the sentinel), bit 4 a check of the bounds-checked build failed; read once the
  // work is done
  if (!dstatus.p) {
    EELS_CK(dstatus.alloc(1, st));
    EELS_CK(cudaMemsetAsync(dstatus.p, 0, sizeof(int), st));
  }
  EELS_CK(eels::launch_scale_check(dmap.p, n_map, scale, dstatus.p, st));
  EELS_CK(collect_checks(dstatus.p, st));
  {
    int flag = 0;
    EELS_CK(cudaMemcpyAsync(&flag, dstatus.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    EELS_CK(cudaStreamSynchronize(st));
    if (flag & 4) return fail(ctx, EELS_ERR_BOUNDS, "a bounds check of the debug build failed");
    if (flag & 1) return fail(ctx, EELS_ERR_TIMEOUT, "tensor-core pipeline wait timed out");
    nonfinite = (flag & 2) != 0;
  }
  if (map_on_device) {
    EELS_CK(cudaMemcpyAsync(map_out, dmap.p, sizeof(double) * n_map, cudaMemcpyDeviceToDevice, st));
  } else {
    EELS_CK(cudaMemcpyAsync(map_out, dmap.p, sizeof(double) * n_map, cudaMemcpyDeviceToHost, st));
    EELS_CK(cudaStreamSynchronize(st));
  }
  if (nonfinite) return fail(ctx, EELS_ERR_NONFINITE, "the map holds NaN or Inf values");
  return EELS_OK;
}

eels_status check_map_args(eels_ctx* ctx, const eels_smatrix* sm, const eels_transitions* tr,
                           const eels_scan* sc, double beta, int precision) {
  eels_status r = check_transitions(ctx, tr, sc, sm->n, sm->n_z);
  if (r != EELS_OK) return r;
  if (precision != EELS_PREC_FP32 && precision != EELS_PREC_TF32 &&
      precision != EELS_PREC_BF16X3)
    return fail(ctx, EELS_ERR_UNSUPPORTED, "precision not built");
  if (!(beta > 0)) return fail(ctx, EELS_ERR_ARG, "bad beta");
  return EELS_OK;
}

}  // namespace

eels_status eels_inelastic_map(eels_ctx* ctx, const eels_smatrix* sm, const eels_transitions* tr,
                               const eels_scan* sc, double beta, int precision, double* map_out,
                               int map_on_device, void* stream) {
  if (!ctx || !sm || !map_out) return fail(ctx, EELS_ERR_ARG, "null argument");
  Range nvtx_range("eels_inelastic_map");
  eels_status r = check_map_args(ctx, sm, tr, sc, beta, precision);
  if (r != EELS_OK) return r;
  return map_window(ctx, sm, tr, sc, ScanWin{0, 0, sc->n_sx, sc->n_sy}, beta, precision, map_out,
                    map_on_device, stream);
}

eels_status eels_inelastic_map_tiles(eels_ctx* ctx, const eels_smatrix* sm,
                                     const eels_transitions* tr, const eels_scan* sc, double beta,
                                     int precision, int tile_nx, int tile_ny, double* map_out,
                                     uint8_t* tile_done, int max_tiles, int* remaining,
                                     void* stream) {
  if (!ctx || !sm || !map_out || !tile_done) return fail(ctx, EELS_ERR_ARG, "null argument");
  Range nvtx_range("eels_inelastic_map_tiles");
  eels_status r = check_map_args(ctx, sm, tr, sc, beta, precision);
  if (r != EELS_OK) return r;
  if (tile_nx < 1 || tile_ny < 1) return fail(ctx, EELS_ERR_ARG, "scan tiles need >= 1 position");
  const int gx = (sc->n_sx + tile_nx - 1) / tile_nx, gy = (sc->n_sy + tile_ny - 1) / tile_ny;
  const int T = tr->n_types;
  int todo = 0;
  for (int k = 0; k < gx * gy; ++k) todo += tile_done[k] ? 0 : 1;
  if (remaining) *remaining = todo;
  std::vector<double> part;
  int mapped = 0;
  for (int ty = 0; ty < gy; ++ty)
    for (int tx = 0; tx < gx; ++tx) {
      const int k = ty * gx + tx;
      if (tile_done[k]) continue;
      if (max_tiles > 0 && mapped >= max_tiles) return EELS_OK;
      const ScanWin win{tx * tile_nx, ty * tile_ny, std::min(tile_nx, sc->n_sx - tx * tile_nx),
                        std::min(tile_ny, sc->n_sy - ty * tile_ny)};
      part.assign((size_t)T * win.nx * win.ny, 0.0);
      r = map_window(ctx, sm, tr, sc, win, beta, precision, part.data(), 0, stream);
      if (r != EELS_OK) return r;   // finished tiles stay written and marked
      for (int m = 0; m < T; ++m)
        for (int y = 0; y < win.ny; ++y)
          std::memcpy(map_out + ((int64_t)m * sc->n_sy + win.iy0 + y) * sc->n_sx + win.ix0,
                      part.data() + ((int64_t)m * win.ny + y) * win.nx, sizeof(double) * win.nx);
      tile_done[k] = 1;
      ++mapped;
      if (remaining) --*remaining;
    }
  return EELS_OK;
}

// First pixel of the L/f cut around r on one axis of the N/2 grid: the in-rule pixel
// (same minimum-image rule as the site windows) whose cyclic predecessor is out of rule;
// -1 if the in-rule pixels are not one cyclic run.  Every pixel in rule (f = 1): 0.
static int cut_start(int nh, double cell, int f, double r) {
  std::vector<char> ok(nh);
  int count = 0;
  for (int p = 0; p < nh; ++p) {
    ok[p] = axis_in_window((double)p * (cell / nh), r, cell, f) ? 1 : 0;
    count += ok[p];
  }
  if (count == nh) return 0;
  int start = -1, runs = 0;
  for (int p = 0; p < nh; ++p)
    if (ok[p] && !ok[(p + nh - 1) % nh]) { start = p; ++runs; }
  return runs == 1 ? start : -1;
}

eels_status eels_elastic_images(eels_ctx* ctx, const eels_smatrix* sm, const eels_scan* sc,
                                const eels_detector* det, int n_det, double* out,
                                int out_on_device, void* stream) {
  if (!ctx || !sm || !sc || !det || !out) return fail(ctx, EELS_ERR_ARG, "null argument");
  if (!sm->s_exit)
    return fail(ctx, EELS_ERR_ARG, "S-matrix built without the exit plane (EELS_OPT_EXIT_PLANE)");
  if (n_det < 1 || n_det > eels::kMaxDetectors) return fail(ctx, EELS_ERR_ARG, "1..8 detectors");
  if (sc->n_sx <= 0 || sc->n_sy <= 0) return fail(ctx, EELS_ERR_ARG, "empty scan");
  const int n = sm->n, nh = n / 2, f = sm->f;
  if (nh % f) return fail(ctx, EELS_ERR_UNSUPPORTED, "the L/f cut needs N/2 divisible by f");
  const int m = nh / f;
  if (!eels::cut_supported(m))
    return fail(ctx, EELS_ERR_UNSUPPORTED, "cut size " + std::to_string(m) + " not built");
  for (int d = 0; d < n_det; ++d)
    if (!(det[d].inner >= 0) || det[d].outer != det[d].outer)
      return fail(ctx, EELS_ERR_ARG, "bad detector angles");
  EELS_CK(enter(ctx));
  cudaStream_t st = (cudaStream_t)stream;
  const int n_in = (int)sm->bp.size();
  const int64_t n_img = (int64_t)sc->n_sx * sc->n_sy;

  // cut origins per scan column / row
  std::vector<int> wx(sc->n_sx), wy(sc->n_sy);
  for (int i = 0; i < sc->n_sx; ++i)
    if ((wx[i] = cut_start(nh, sm->cell, f, sc->x0 + (double)i * sc->step_x)) < 0)
      return fail(ctx, EELS_ERR_ARG, "probe cut is not one run of pixels");
  for (int i = 0; i < sc->n_sy; ++i)
    if ((wy[i] = cut_start(nh, sm->cell, f, sc->y0 + (double)i * sc->step_y)) < 0)
      return fail(ctx, EELS_ERR_ARG, "probe cut is not one run of pixels");
  // detector bins of the cut's DFT lattice k = f (a, b) / L, inside the band limit
  std::vector<uint8_t> mask((size_t)m * m, 0);
  for (int b = 0; b < m; ++b)
    for (int a = 0; a < m; ++a) {
      const int sa = a < (m + 1) / 2 ? a : a - m, sb = b < (m + 1) / 2 ? b : b - m;
      const int64_t r2 = (int64_t)sa * sa + (int64_t)sb * sb;
      if (16 * (int64_t)f * f * r2 >= (int64_t)n * n) continue;
      const double k = f * std::sqrt((double)r2) / sm->cell;
      for (int d = 0; d < n_det; ++d) {
        bool in = sm->lam * k >= det[d].inner;
        if (det[d].outer > 0) in = in && sm->lam * k <= det[d].outer;
        if (in) mask[(size_t)b * m + a] |= (uint8_t)(1u << d);
      }
    }
  float2* tw = nullptr;
  eels_status r = twiddles(ctx, m, &tw);
  if (r != EELS_OK) return r;
  DevBuf<int> dwx, dwy, dbp, dbq;
  DevBuf<uint8_t> dmask;
  DevBuf<float2> ax, ay, cuts;
  DevBuf<double> dimg;
  EELS_CK(dwx.upload(wx.data(), wx.size(), st));
  EELS_CK(dwy.upload(wy.data(), wy.size(), st));
  EELS_CK(dmask.upload(mask.data(), mask.size(), st));
  EELS_CK(dbp.upload(sm->bp.data(), n_in, st));
  EELS_CK(dbq.upload(sm->bq.data(), n_in, st));
  EELS_CK(ax.alloc((size_t)n_in * sc->n_sx, st));
  EELS_CK(ay.alloc((size_t)n_in * sc->n_sy, st));
  EELS_CK(eels::launch_phase_table(ax.p, dbp.p, n_in, f, sm->cell, sc->x0, sc->step_x, sc->n_sx, st));
  EELS_CK(eels::launch_phase_table(ay.p, dbq.p, n_in, f, sm->cell, sc->y0, sc->step_y, sc->n_sy, st));
  EELS_CK(dimg.alloc((size_t)n_det * n_img, st));
  EELS_CK(cudaMemsetAsync(dimg.p, 0, sizeof(double) * n_det * n_img, st));
  // scan rows in batches whose cuts fit in ~1 GiB
  const int64_t per_row = (int64_t)sc->n_sx * m * m * (int64_t)sizeof(float2);
  const int rows_b = (int)std::max<int64_t>(1, std::min<int64_t>(sc->n_sy, ((int64_t)1 << 30) / per_row));
  EELS_CK(cuts.alloc((size_t)rows_b * sc->n_sx * m * m, st));
  for (int iy0 = 0; iy0 < sc->n_sy; iy0 += rows_b) {
    const int nr = std::min(rows_b, sc->n_sy - iy0);
    {
      Prof pr(ctx, "exit_cut", st);
      EELS_CK(eels::launch_exit_cut(sm->s_exit, n_in, nh, m, ax.p, ay.p, sc->n_sx, sc->n_sy,
                                    dwx.p, dwy.p, iy0, nr, cuts.p, st));
    }
    Prof pr(ctx, "cut_fft_detect", st);
    EELS_CK(eels::launch_cut_detect(m, cuts.p, nr * sc->n_sx, dmask.p, n_det, sc->n_sx, iy0,
                                    n_img, dimg.p, tw, st));
  }
  // I = (16 f^2 / N^2) (c^2 / N^2) sum |DFT|^2: S_exit carries N, the coefficients omit c
  const double nn = (double)n * (double)n;
  const double scale = (double)f * f * ((double)f * f / n_in) * 16.0 / (nn * nn);
  EELS_CK(eels::launch_scale(dimg.p, n_det * n_img, scale, st));
  if ((r = checked_status(ctx, st)) != EELS_OK) return r;
  if (out_on_device) {
    EELS_CK(cudaMemcpyAsync(out, dimg.p, sizeof(double) * n_det * n_img, cudaMemcpyDeviceToDevice, st));
  } else {
    EELS_CK(cudaMemcpyAsync(out, dimg.p, sizeof(double) * n_det * n_img, cudaMemcpyDeviceToHost, st));
    EELS_CK(cudaStreamSynchronize(st));
  }
  return EELS_OK;
}

eels_status eels_phonon_map(eels_ctx* ctx, const eels_specimen* specs,
                            const eels_transitions* trs, int n_configs, const eels_optics* optics,
                            const eels_scan* sc, double beta, int precision, double* map_out,
                            int map_on_device, void* stream) {
  if (!ctx || !specs || !trs || !optics || !sc || !map_out || n_configs < 1)
    return fail(ctx, EELS_ERR_ARG, "bad arguments");
  for (int c = 1; c < n_configs; ++c)
    if (specs[c].n != specs[0].n || trs[c].n_types != trs[0].n_types)
      return fail(ctx, EELS_ERR_ARG, "configurations differ in grid or channel count");
  EELS_CK(enter(ctx));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n_map = (int64_t)trs[0].n_types * sc->n_sx * sc->n_sy;
  DevBuf<double> acc, one;
  EELS_CK(acc.alloc((size_t)n_map, st));
  EELS_CK(one.alloc((size_t)n_map, st));
  EELS_CK(cudaMemsetAsync(acc.p, 0, sizeof(double) * n_map, st));
  for (int c = 0; c < n_configs; ++c) {
    eels_smatrix* sm = nullptr;
    eels_status r = eels_build_smatrix(ctx, &specs[c], optics, stream, &sm);
    if (r == EELS_OK) r = eels_inelastic_map(ctx, sm, &trs[c], sc, beta, precision, one.p, 1, stream);
    eels_smatrix_free(sm);
    if (r != EELS_OK) return r;
    EELS_CK(eels::launch_accumulate(acc.p, one.p, n_map, st));
  }
  EELS_CK(eels::launch_scale(acc.p, n_map, 1.0 / n_configs, st));
  if (map_on_device) {
    EELS_CK(cudaMemcpyAsync(map_out, acc.p, sizeof(double) * n_map, cudaMemcpyDeviceToDevice, st));
  } else {
    EELS_CK(cudaMemcpyAsync(map_out, acc.p, sizeof(double) * n_map, cudaMemcpyDeviceToHost, st));
    EELS_CK(cudaStreamSynchronize(st));
  }
  return EELS_OK;
}

eels_status eels_divide_map(eels_ctx* ctx, double* map, const double* bf, int n_types,
                            int64_t n_pix, int on_device, void* stream) {
  if (!ctx || !map || !bf || n_types < 0 || n_pix < 0) return fail(ctx, EELS_ERR_ARG, "bad arguments");
  EELS_CK(enter(ctx));
  cudaStream_t st = (cudaStream_t)stream;
  if (on_device) {
    EELS_CK(eels::launch_divide(map, bf, n_types, n_pix, st));
    return EELS_OK;
  }
  DevBuf<double> dm, db;
  EELS_CK(dm.upload(map, (size_t)n_types * n_pix, st));
  EELS_CK(db.upload(bf, (size_t)n_pix, st));
  EELS_CK(eels::launch_divide(dm.p, db.p, n_types, n_pix, st));
  EELS_CK(cudaMemcpyAsync(map, dm.p, sizeof(double) * n_types * n_pix, cudaMemcpyDeviceToHost, st));
  EELS_CK(cudaStreamSynchronize(st));
  return EELS_OK;
}

eels_status eels_quadratic_reference_map(eels_ctx* ctx, const eels_specimen* spec,
                                         const eels_optics* op, const eels_transitions* tr,
                                         const eels_scan* sc, double beta,
                                         const int32_t* positions, int n_pos, double* map_out,
                                         int map_on_device, void* stream, int64_t* steps) {
  if (!ctx || !map_out) return fail(ctx, EELS_ERR_ARG, "null argument");
  eels_status r = check_specimen(ctx, spec, op);
  if (r != EELS_OK) return r;
  if ((r = check_transitions(ctx, tr, sc, spec->n, spec->n_z)) != EELS_OK) return r;
  if (!(beta > 0)) return fail(ctx, EELS_ERR_ARG, "bad beta");
  EELS_CK(enter(ctx));
  cudaStream_t st = (cudaStream_t)stream;
  const int n = spec->n, nh = n / 2, n_z = spec->n_z, f = op->f;
  const int T = tr->n_types, w = tr->w, S = tr->n_sites;
  const int64_t plane = (int64_t)nh * nh;
  const int n_scan = sc->n_sx * sc->n_sy;
  const int64_t n_map = (int64_t)T * n_scan;

  std::vector<int> bp, bq, dp, dq;
  lattice_beams(n, spec->cell, op->lambda, f, op->alpha, bp, bq);
  lattice_beams(n, spec->cell, op->lambda, f, beta, dp, dq);
  if (bp.empty() || dp.empty()) return fail(ctx, EELS_ERR_ARG, "empty aperture");
  if (!inside_band(n, f, bp, bq) || !inside_band(n, f, dp, dq))
    return fail(ctx, EELS_ERR_ARG, "aperture extends beyond the band limit");
  float2* tw = nullptr;
  if ((r = twiddles(ctx, n, &tw)) != EELS_OK) return r;

  std::vector<std::pair<int, int>> pos;
  if (positions) {
    if (n_pos < 0) return fail(ctx, EELS_ERR_ARG, "bad n_pos");
    for (int k = 0; k < n_pos; ++k) {
      const int iy = positions[2 * k], ix = positions[2 * k + 1];
      if (iy < 0 || iy >= sc->n_sy || ix < 0 || ix >= sc->n_sx)
        return fail(ctx, EELS_ERR_ARG, "scan position out of range");
      pos.emplace_back(iy, ix);
    }
  } else {
    for (int iy = 0; iy < sc->n_sy; ++iy)
      for (int ix = 0; ix < sc->n_sx; ++ix) pos.emplace_back(iy, ix);
  }

  DevBuf<float2> t, ptab, dH;
  EELS_CK(t.alloc((size_t)n_z * n * n, st));
  EELS_CK(ptab.alloc((size_t)plane, st));
  if ((r = build_slices(ctx, spec, op, st, t.p, ptab.p)) != EELS_OK) return r;
  const float2* H = (const float2*)tr->H;
  if (!tr->on_device) {
    EELS_CK(dH.upload((const float2*)tr->H, (size_t)(tr->h_shared ? 1 : S) * T * w * w, st));
    H = dH.p;
  }
  DevBuf<int> dwx, dwy, dbp, dbq;
  EELS_CK(dwx.upload(tr->win_x0, S, st));
  EELS_CK(dwy.upload(tr->win_y0, S, st));
  EELS_CK(dbp.upload(bp.data(), bp.size(), st));
  EELS_CK(dbq.upload(bq.data(), bq.size(), st));
  // detector bins in box order [kx'][ky']
  std::vector<uint8_t> mask((size_t)plane, 0);
  for (size_t d = 0; d < dp.size(); ++d) {
    int kx = f * dp[d], ky = f * dq[d];
    kx = kx >= 0 ? kx : kx + nh;
    ky = ky >= 0 ? ky : ky + nh;
    mask[(size_t)kx * nh + ky] = 1;
  }
  DevBuf<uint8_t> dmask;
  EELS_CK(dmask.upload(mask.data(), mask.size(), st));
  DevBuf<double> dmap;
  EELS_CK(dmap.alloc((size_t)n_map, st));
  EELS_CK(cudaMemsetAsync(dmap.p, 0, sizeof(double) * n_map, st));

  // transitions each probe sees, per slice
  std::vector<std::vector<int>> by_slice(n_z);
  for (int s = 0; s < S; ++s) by_slice[tr->slice[s]].push_back(s);
  auto sees = [&](int s, int iy, int ix) {
    return axis_in_window(tr->x[s], sc->x0 + (double)ix * sc->step_x, spec->cell, f) &&
           axis_in_window(tr->y[s], sc->y0 + (double)iy * sc->step_y, spec->cell, f);
  };
  std::vector<int> waves_of(pos.size(), 1);
  int64_t total_steps = 0;
  for (size_t k = 0; k < pos.size(); ++k) {
    for (int i = 0; i < n_z; ++i)
      for (int s : by_slice[i])
        if (sees(s, pos[k].first, pos[k].second)) {
          waves_of[k] += T;
          total_steps += (int64_t)T * (n_z - i);
        }
    total_steps += n_z;
  }
  // probe batches: at most 65535 waves and about 32 GiB of work arrays
  const int64_t wave_bytes = 2 * (int64_t)n * nh * sizeof(float2);
  const int64_t max_waves = std::min<int64_t>(65535, ((int64_t)32 << 30) / wave_bytes);
  size_t k0 = 0;
  const double c = (double)f / std::sqrt((double)bp.size());
  while (k0 < pos.size()) {
    size_t k1 = k0;
    int64_t nw = 0;
    while (k1 < pos.size() && (k1 == k0 || nw + waves_of[k1] <= max_waves)) nw += waves_of[k1++];
    if (nw > 65535) return fail(ctx, EELS_ERR_UNSUPPORTED, "too many inelastic waves for one probe");
    const int B = (int)(k1 - k0);
    std::vector<double> rx(B), ry(B);
    for (int b = 0; b < B; ++b) {
      rx[b] = sc->x0 + (double)pos[k0 + b].second * sc->step_x;
      ry[b] = sc->y0 + (double)pos[k0 + b].first * sc->step_y;
    }
    // spawn lists per slice and the map index of every wave
    std::vector<int> wave_out((size_t)nw, -1), sp_src, sp_site, sp_type, sp_off(n_z + 1, 0);
    int next = B;
    for (int i = 0; i < n_z; ++i) {
      sp_off[i] = (int)sp_src.size();
      for (int b = 0; b < B; ++b)
        for (int s : by_slice[i])
          if (sees(s, pos[k0 + b].first, pos[k0 + b].second))
            for (int m = 0; m < T; ++m) {
              sp_src.push_back(b);
              sp_site.push_back(s);
              sp_type.push_back(m);
              wave_out[next++] = m * n_scan + pos[k0 + b].first * sc->n_sx + pos[k0 + b].second;
            }
    }
    sp_off[n_z] = (int)sp_src.size();
    DevBuf<double> drx, dry;
    DevBuf<int> dwo, dsrc, dsite, dtype;
    DevBuf<float2> W, Phi, D;
    EELS_CK(drx.upload(rx.data(), B, st));
    EELS_CK(dry.upload(ry.data(), B, st));
    EELS_CK(dwo.upload(wave_out.data(), wave_out.size(), st));
    EELS_CK(dsrc.upload(sp_src.data(), sp_src.size(), st));
    EELS_CK(dsite.upload(sp_site.data(), sp_site.size(), st));
    EELS_CK(dtype.upload(sp_type.data(), sp_type.size(), st));
    EELS_CK(W.alloc((size_t)nw * n * nh, st));
    EELS_CK(Phi.alloc((size_t)nw * n * nh, st));
    EELS_CK(D.alloc((size_t)B * plane, st));
    EELS_CK(eels::launch_probe_init(W.p, n, B, drx.p, dry.p, dbp.p, dbq.p, (int)bp.size(), f,
                                    spec->cell, c, tw, st));
    int active = B;
    for (int i = 0; i < n_z; ++i) {
      {
        Prof pr(ctx, "row_pass", st);
        EELS_CK(launch_row_pass(n, active, W.p, Phi.p, t.p + (int64_t)i * n * n, 0, 1, D.p, B,
                                plane, 1, tw, st));
      }
      eels::SpawnList sl{dsrc.p + sp_off[i], dsite.p + sp_off[i], dtype.p + sp_off[i],
                         sp_off[i + 1] - sp_off[i], active};
      {
        Prof pr(ctx, "spawn", st);
        EELS_CK(eels::launch_spawn(n, sl, D.p, H, T, tr->h_shared ? 0 : 1, w, dwx.p, dwy.p, Phi.p,
                                   tw, st));
      }
      active += sl.count;
      const bool last = (i == n_z - 1);
      {
        Prof pr(ctx, last ? "col_pass_detect" : "col_pass", st);
        EELS_CK(launch_col_pass(n, active, Phi.p, W.p, ptab.p, 0, last ? 1 : 0, dmask.p, dwo.p,
                                dmap.p, (double)f * f, tw, st));
      }
    }
    k0 = k1;
  }
  if (steps) *steps = total_steps;
  if ((r = checked_status(ctx, st)) != EELS_OK) return r;
  if (map_on_device) {
    EELS_CK(cudaMemcpyAsync(map_out, dmap.p, sizeof(double) * n_map, cudaMemcpyDeviceToDevice, st));
  } else {
    EELS_CK(cudaMemcpyAsync(map_out, dmap.p, sizeof(double) * n_map, cudaMemcpyDeviceToHost, st));
    EELS_CK(cudaStreamSynchronize(st));
  }
  return EELS_OK;
}

}  // extern "C"
