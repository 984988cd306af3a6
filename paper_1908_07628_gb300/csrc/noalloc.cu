// eels_build_smatrix_static: the S_in build for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: plug-ins living inside a host application
// that owns the device memory pool (or has reserved all of it), and real-time loops
// that must not pay for or risk an allocation failure mid-run.  For them this entry point produces exactly what
// eels_build_smatrix stores (S_in at every depth) in a buffer the caller passes,
// and keeps its own work arrays in one statically sized device array that the
// library reserves when it is loaded.  It calls no cudaMalloc/cudaFree and no
// allocating library routine.
//
// The work array is shared by every call on a device and keeps whatever the last
// call left in it; every region a call reads is written earlier in the same call,
// so nothing needs clearing.  Calls whose GPU work overlaps (two streams, two host
// threads) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"
#include "stem_eels.h"

namespace {

// 64 MiB, held by every GPU that loads the library until the process exits.
constexpr size_t kStaticBytes = (size_t)EELS_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

void set_err(char* err, int cap, const char* msg) {
  if (err && cap > 0) {
    std::strncpy(err, msg, (size_t)cap - 1);
    err[cap - 1] = 0;
  }
}

// Device address of g_scratch on the current device, looked up once per device (with
// that device current) and kept for the process; after cudaDeviceReset the kept
// address may be stale, which the header states.
cudaError_t scratch_ptr(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_ptr[dev]);
  return cudaSuccess;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" eels_status eels_build_smatrix_static(const eels_specimen* spec,
                                                 const eels_optics* op, float* s_in,
                                                 int64_t s_in_bytes, int* n_in_out,
                                                 void* stream, char* err, int err_cap) {
  set_err(err, err_cap, "");
  if (!spec || !op || !spec->vproj || !s_in) {
    set_err(err, err_cap, "null argument");
    return EELS_ERR_ARG;
  }
  const int n = spec->n, n_z = spec->n_z;
  if (!eels::grid_supported(n)) {
    set_err(err, err_cap, "grid size not built into this library");
    return EELS_ERR_UNSUPPORTED;
  }
  if (n_z <= 0 || !(spec->cell > 0) || op->f < 1 || !(op->lambda > 0) || !(op->dz > 0) ||
      !(op->alpha > 0)) {
    set_err(err, err_cap, "bad specimen or optics");
    return EELS_ERR_ARG;
  }
  // probe beams: f-lattice points with lambda |k| <= alpha, row-major (q, then p)
  std::vector<int> px, py;
  const int f = op->f;
  const int pmax = (int)std::ceil(op->alpha * spec->cell / (op->lambda * f)) + 1;
  for (int b = -pmax; b <= pmax; ++b)
    for (int a = -pmax; a <= pmax; ++a)
      if (op->lambda * f * std::sqrt((double)(a * a + b * b)) / spec->cell <= op->alpha) {
        px.push_back(f * a);
        py.push_back(f * b);
      }
  const int n_in = (int)px.size();
  if (n_in == 0) {
    set_err(err, err_cap, "no probe beam inside the aperture");
    return EELS_ERR_ARG;
  }
  for (int j = 0; j < n_in; ++j)
    if (16 * ((int64_t)px[j] * px[j] + (int64_t)py[j] * py[j]) >= (int64_t)n * n) {
      set_err(err, err_cap, "probe aperture extends beyond the band limit");
      return EELS_ERR_ARG;
    }
  const int nh = n / 2;
  const int64_t plane = (int64_t)nh * nh;
  const int64_t need_out = (int64_t)n_z * n_in * plane * 8;
  if (s_in_bytes < need_out) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "output buffer holds %lld bytes, S_in needs %lld",
                  (long long)s_in_bytes, (long long)need_out);
    set_err(err, err_cap, msg);
    return EELS_ERR_ARG;
  }

  // carve the static array: twiddles | propagator | one transmission slice |
  // one potential slice | beam lists | W | Phi (waves processed in chunks)
  size_t off = 0;
  const size_t o_tw = off;   off = align256(off + sizeof(float2) * eels::twiddle_table_size(n));
  const size_t o_p = off;    off = align256(off + sizeof(float2) * plane);
  const size_t o_t = off;    off = align256(off + sizeof(float2) * (size_t)n * n);
  const size_t o_v = off;    off = align256(off + sizeof(float) * (size_t)n * n);
  const size_t o_px = off;   off = align256(off + sizeof(int) * n_in);
  const size_t o_py = off;   off = align256(off + sizeof(int) * n_in);
  const size_t o_amp = off;  off = align256(off + sizeof(float2) * n_in);
  const size_t wave_bytes = sizeof(float2) * (size_t)n * nh;
  if (off >= kStaticBytes || (kStaticBytes - off) / (2 * wave_bytes) < 1) {
    char msg[200];
    std::snprintf(msg, sizeof msg,
                  "problem too large for the %zu-byte static work array (N = %d, %d beams)",
                  kStaticBytes, n, n_in);
    set_err(err, err_cap, msg);
    return EELS_ERR_ARG;
  }
  const int chunk = (int)std::min<size_t>((size_t)n_in, (kStaticBytes - off) / (2 * wave_bytes));
  if (n_in_out) *n_in_out = n_in;   // written only once every check has passed
  const size_t o_w = off;
  const size_t o_phi = align256(o_w + wave_bytes * chunk);

  unsigned char* base = nullptr;
  (void)cudaGetLastError();   // drop a non-sticky error left by unrelated earlier calls
  cudaError_t e = scratch_ptr(&base);
  if (e != cudaSuccess) {
    set_err(err, err_cap, cudaGetErrorString(e));
    return EELS_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  float2* tw = reinterpret_cast<float2*>(base + o_tw);
  float2* ptab = reinterpret_cast<float2*>(base + o_p);
  float2* tsl = reinterpret_cast<float2*>(base + o_t);
  float* vsl = reinterpret_cast<float*>(base + o_v);
  int* dpx = reinterpret_cast<int*>(base + o_px);
  int* dpy = reinterpret_cast<int*>(base + o_py);
  float2* damp = reinterpret_cast<float2*>(base + o_amp);
  float2* W = reinterpret_cast<float2*>(base + o_w);
  float2* Phi = reinterpret_cast<float2*>(base + o_phi);

  // host-computed tables, copied into the static array
  std::vector<float2> htw(eels::twiddle_table_size(n)), hamp(n_in, make_float2(1.f, 0.f));
  eels::fill_twiddle_tables(n, htw.data());
#define EELS_SCK(call)                                      \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) {                                \
      set_err(err, err_cap, cudaGetErrorString(e_));        \
      return EELS_ERR_CUDA;                                 \
    }                                                       \
  } while (0)
  EELS_SCK(cudaMemcpyAsync(tw, htw.data(), sizeof(float2) * htw.size(), cudaMemcpyHostToDevice,
                           st));
  EELS_SCK(cudaMemcpyAsync(dpx, px.data(), sizeof(int) * n_in, cudaMemcpyHostToDevice, st));
  EELS_SCK(cudaMemcpyAsync(dpy, py.data(), sizeof(int) * n_in, cudaMemcpyHostToDevice, st));
  EELS_SCK(cudaMemcpyAsync(damp, hamp.data(), sizeof(float2) * n_in, cudaMemcpyHostToDevice, st));
  EELS_SCK(eels::launch_propagator_table(ptab, n, spec->cell, op->lambda, op->dz,
                                         (float)(1.0 / ((double)n * n)), st));
  float2* out = reinterpret_cast<float2*>(s_in);
  for (int j0 = 0; j0 < n_in; j0 += chunk) {
    const int nb = std::min(chunk, n_in - j0);
    EELS_SCK(eels::launch_init_plane_waves(W, n, nb, dpx + j0, dpy + j0, damp + j0, tw, st));
    for (int i = 0; i < n_z; ++i) {
      const float* v = spec->vproj + (int64_t)i * n * n;
      if (!spec->vproj_on_device) {
        EELS_SCK(cudaMemcpyAsync(vsl, v, sizeof(float) * (size_t)n * n, cudaMemcpyHostToDevice,
                                 st));
        v = vsl;
      }
      EELS_SCK(eels::launch_transmission(v, op->sigma, tsl, (int64_t)n * n, st));
      const bool last = (i == n_z - 1);
      EELS_SCK(eels::launch_row_pass(n, nb, W, Phi, tsl, 0, 1,
                                     out + ((int64_t)i * n_in + j0) * plane, nb, plane,
                                     last ? 0 : 1, tw, st));
      if (!last)
        EELS_SCK(eels::launch_col_pass(n, nb, Phi, W, ptab, 0, 0, nullptr, nullptr, nullptr, 0.0,
                                       tw, st));
    }
  }
#undef EELS_SCK
  return EELS_OK;
}
