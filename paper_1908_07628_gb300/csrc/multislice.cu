// Band-limited plane-wave multislice on the GPU (Eqs. 3, 4, MSop, MSTop).
//
// A slice step psi -> F^-1[P F[t psi]] is split into two passes over a batch of
// waves.  Between the passes every wave is kept in "row-spectrum" form: an
// array [y][kx'] of N rows by N/2 columns holding the x-DFT of the wave restricted
// to the band box |kx| < N/4 (column kx' < N/4 is frequency kx', otherwise
// kx' - N/2).  Because the propagator limits every wave to p^2 + q^2 < (N/4)^2,
// nothing outside the box is ever needed.
//
//   row pass    (one warp per row y):  zero-pad kx to N, inverse FFT_x, multiply
//                by t (or conj t), optionally store the even samples (the N/2
//                representation used by the S-matrices), forward FFT_x, keep the box.
//   column pass (one warp per column kx'): FFT_y, keep the box, multiply by the
//                propagator table (or its conjugate), zero-pad, inverse FFT_y.
//
// Scale convention: W holds the true row spectrum; the row pass produces N times
// the true real-space wave and N times the true row spectrum, and the propagator
// table carries the 1/N^2 that restores W after the column pass.
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace eels {

namespace {

constexpr int kRowWarps = 4;   // warps per CTA in the row pass (ROWS rows each)
constexpr int kColCB = 8;      // columns per CTA in the column pass (one warp each)

template <int N>
__device__ __forceinline__ void row_pass_body(const float2* __restrict__ W, float2* __restrict__ Phi,
                                              const float2* __restrict__ t_slice, int conj_t,
                                              int store_mode, float2* __restrict__ S, int s_waves,
                                              int64_t s_stride, int fft_out,
                                              const float2* __restrict__ tw) {
  constexpr int NH = N / 2, NQ = N / 4;
  constexpr int ROWS = RegFFT<N>::ROWS;
  constexpr int LDR = spad_len(N);
  using PI = Plan<N, true>;    // inverse transform: reversed radix plan
  using PF = Plan<N, false>;   // forward transform
  constexpr int E = RegFFT<N>::E;
  extern __shared__ float2 smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* sbuf = smem + warp * ROWS * LDR;
  const int y0 = (blockIdx.x * kRowWarps + warp) * ROWS;   // rows y0 .. y0 + ROWS - 1
  const int64_t wave = blockIdx.y;
  float2 v[E];

  // inputs of the inverse x-FFT: the band box, zero-padded to N
  {
    constexpr int R0 = PI::R(0), NB0 = N / R0, PER0 = PI::per(0);
#pragma unroll
    for (int t = 0; t < PER0; ++t) {
      const int u = lane + 32 * t;
      const bool live = (ROWS * NB0) % 32 == 0 || u < ROWS * NB0;
      const int b = u % NB0;
      const float2* src = W + (wave * N + y0 + u / NB0) * NH;
#pragma unroll
      for (int q = 0; q < R0; ++q) {
        const int pos = b + q * NB0;
        float2 x = make_float2(0.f, 0.f);
        if (live && (q * NB0 < NQ || q * NB0 >= N - NQ)) x = src[pos < NQ ? pos : pos - NH];
        v[t * R0 + q] = x;
      }
    }
  }
  reg_fft<N, true, true>(v, sbuf, LDR, tw, lane, band_mask(PI::R(0)));

  // real space: slot u holds N psi(x = u%NBL + q N/RL, y0 + u/NBL)
  {
    constexpr int RL = PF::R(0), NBL = N / RL, PERL = PF::per(0);
#pragma unroll
    for (int t = 0; t < PERL; ++t) {
      const int u = lane + 32 * t;
      if ((ROWS * NBL) % 32 == 0 || u < ROWS * NBL) {
        const int y = y0 + u / NBL, b = u % NBL;
        const float2* trow = t_slice + (int64_t)y * N;
        const bool store = store_mode != 0 && (y & 1) == 0 && wave < s_waves;
        float2* srow = store ? S + wave * s_stride + (int64_t)(y >> 1) * NH : nullptr;
#pragma unroll
        for (int q = 0; q < RL; ++q) {
          const int x = b + q * NBL;
          float2 val = v[t * RL + q];
          if (store && store_mode == 2 && !(x & 1)) srow[x >> 1] = val;
          const float2 tt = trow[x];
          val = conj_t ? cmulc(val, tt) : cmul(val, tt);
          if (store && store_mode == 1 && !(x & 1)) srow[x >> 1] = val;
          v[t * RL + q] = val;
        }
      }
    }
  }
  if (!fft_out) return;
  __syncwarp();
  reg_fft<N, false, false>(v, sbuf, LDR, tw, lane);
  {
    constexpr int RF = PF::R(PF::NS - 1), NBF = N / RF, PERF = PF::per(PF::NS - 1);
#pragma unroll
    for (int t = 0; t < PERF; ++t) {
      const int u = lane + 32 * t;
      if ((ROWS * NBF) % 32 == 0 || u < ROWS * NBF) {
        const int b = u % NBF;
        float2* dst = Phi + (wave * N + y0 + u / NBF) * NH;
#pragma unroll
        for (int q = 0; q < RF; ++q) {
          if (q * NBF < NQ || q * NBF >= N - NQ) {
            const int pos = b + q * NBF;
            dst[pos < NQ ? pos : pos - NH] = v[t * RF + q];
          }
        }
      }
    }
  }
}

template <int N>
__global__ void __launch_bounds__(kRowWarps * 32)
k_row_pass(const float2* __restrict__ W, float2* __restrict__ Phi,
           const float2* __restrict__ t_slice, int conj_t, int store_mode,
           float2* __restrict__ S, int s_waves, int64_t s_stride, int fft_out,
           const float2* __restrict__ tw) {
  row_pass_body<N>(W, Phi, t_slice, conj_t, store_mode, S, s_waves, s_stride, fft_out, tw);
}

// The 768 plan (radix 24 then 32) would take 132 registers, leaving an SM fewer than 16
// warps; this form caps it at 128 registers (16 warps per SM) without spills.
template <int N>
__global__ void __launch_bounds__(kRowWarps * 32, 16 / kRowWarps)
k_row_pass_capped(const float2* __restrict__ W, float2* __restrict__ Phi,
                const float2* __restrict__ t_slice, int conj_t, int store_mode,
                float2* __restrict__ S, int s_waves, int64_t s_stride, int fft_out,
                const float2* __restrict__ tw) {
  row_pass_body<N>(W, Phi, t_slice, conj_t, store_mode, S, s_waves, s_stride, fft_out, tw);
}

// Padding period of the column tile: the forward transform's first stage reads
// x[b + q N/R0] from it and the inverse transform's last stage writes the same form.
template <int N>
__host__ __device__ constexpr int tile_pad() {
  return plan2_radix(N, 0) > 0 ? N / plan_radix(N, 0) : 8;
}

template <int N>
__host__ __device__ constexpr int col_ld() {
  // tile column stride: the cooperative tile load / store touches 8*ROWS columns of
  // one row per half-warp; an odd number of float2 words per column keeps it
  // conflict-free for 16 columns, 2 mod 16 for 8
  return spad_len(N) + (rows_per_warp(N) == 2 ? 1 : 2);
}

template <int N>
__global__ void __launch_bounds__(kColCB * 32)
k_col_pass(const float2* __restrict__ Phi, float2* __restrict__ W,
           const float2* __restrict__ ptab, int conj_p, int mode,
           const uint8_t* __restrict__ det_mask, const int* __restrict__ wave_out,
           double* __restrict__ det_acc, double det_scale, const float2* __restrict__ tw) {
  constexpr int NH = N / 2, NQ = N / 4;
  constexpr int ROWS = RegFFT<N>::ROWS;
  constexpr int CB = kColCB * ROWS;          // columns per CTA
  constexpr int LD = col_ld<N>();
  constexpr int TP = tile_pad<N>();
  using PI = Plan<N, true>;
  using PF = Plan<N, false>;
  constexpr int E = RegFFT<N>::E;
  extern __shared__ float2 smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kx0 = blockIdx.x * CB;
  const int64_t wave = blockIdx.y;
  const float2* src = Phi + wave * (int64_t)N * NH;
  {
    // all N / (256 / CB) loads of a thread in flight at once
    const int c = threadIdx.x % CB;
    constexpr int STEP = (kColCB * 32) / CB, NL = N / STEP;
    float2 tmp[NL];
#pragma unroll
    for (int i = 0; i < NL; ++i) tmp[i] = src[(int64_t)(threadIdx.x / CB + i * STEP) * NH + kx0 + c];
#pragma unroll
    for (int i = 0; i < NL; ++i) smem[c * LD + spad<TP>(threadIdx.x / CB + i * STEP)] = tmp[i];
  }
  __syncthreads();
  float2* sbuf = smem + warp * ROWS * LD;    // this warp's ROWS columns
  float2 v[E];
  {
    constexpr int R0 = PF::R(0), NB0 = N / R0, PER0 = PF::per(0);
#pragma unroll
    for (int t = 0; t < PER0; ++t) {
      const int u = lane + 32 * t;
      if ((ROWS * NB0) % 32 == 0 || u < ROWS * NB0) {
        const int b = u % NB0;
        const float2* col = sbuf + (u / NB0) * LD;
#pragma unroll
        for (int q = 0; q < R0; ++q) v[t * R0 + q] = col[spad<TP>(b + q * NB0)];
      }
    }
  }
  __syncwarp();
  // the column pass is bound by wavefronts as much as by arithmetic
  reg_fft<N, false, false, table_twiddles_cheap<N, false>()>(v, sbuf, LD, tw, lane);
  // y-spectrum: slot u holds ky = u%NBF + q N/RF of column kx0 + warp*ROWS + u/NBF
  constexpr int RF = PF::R(PF::NS - 1), NBF = N / RF, PERF = PF::per(PF::NS - 1);
  if (mode == 0) {
#pragma unroll
    for (int t = 0; t < PERF; ++t) {
      const int u = lane + 32 * t;
      const bool live = (ROWS * NBF) % 32 == 0 || u < ROWS * NBF;
      const int b = u % NBF;
      const float2* prow = ptab + (int64_t)(kx0 + warp * ROWS + u / NBF) * NH;
#pragma unroll
      for (int q = 0; q < RF; ++q) {
        float2 val = make_float2(0.f, 0.f);
        if (live && (q * NBF < NQ || q * NBF >= N - NQ)) {
          const int pos = b + q * NBF;
          const float2 p = prow[pos < NQ ? pos : pos - NH];
          val = conj_p ? cmulc(v[t * RF + q], p) : cmul(v[t * RF + q], p);
        }
        v[t * RF + q] = val;
      }
    }
    __syncwarp();
    reg_fft<N, true, true, table_twiddles_cheap<N, true>()>(v, sbuf, LD, tw, lane,
                                                           band_mask(PI::R(0)));
    {
      constexpr int RL = PI::R(PI::NS - 1), NBL = N / RL, PERL = PI::per(PI::NS - 1);
#pragma unroll
      for (int t = 0; t < PERL; ++t) {
        const int u = lane + 32 * t;
        if ((ROWS * NBL) % 32 == 0 || u < ROWS * NBL) {
          const int b = u % NBL;
          float2* col = sbuf + (u / NBL) * LD;
#pragma unroll
          for (int q = 0; q < RL; ++q) col[spad<TP>(b + q * NBL)] = v[t * RL + q];
        }
      }
    }
    __syncthreads();
    float2* dst = W + wave * (int64_t)N * NH;
    const int c = threadIdx.x % CB;
    constexpr int STEP = (kColCB * 32) / CB, NL = N / STEP;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
      const int r = threadIdx.x / CB + i * STEP;
      dst[(int64_t)r * NH + kx0 + c] = smem[c * LD + spad<TP>(r)];
    }
  } else {
    const int out = wave_out[wave];
    if (out < 0) return;
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < PERF; ++t) {
      const int u = lane + 32 * t;
      const bool live = (ROWS * NBF) % 32 == 0 || u < ROWS * NBF;
      const int b = u % NBF;
      const int kx = kx0 + warp * ROWS + u / NBF;
      const float2* prow = ptab + (int64_t)kx * NH;
      const uint8_t* mrow = det_mask + (int64_t)kx * NH;
#pragma unroll
      for (int q = 0; q < RF; ++q) {
        if (live && (q * NBF < NQ || q * NBF >= N - NQ)) {
          const int pos = b + q * NBF;
          const int ky = pos < NQ ? pos : pos - NH;
          if (mrow[ky]) {
            const float2 val = conj_p ? cmulc(v[t * RF + q], prow[ky]) : cmul(v[t * RF + q], prow[ky]);
            acc = fmaf(val.x, val.x, fmaf(val.y, val.y, acc));
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc != 0.f) atomicAdd(det_acc + out, det_scale * (double)acc);
  }
}

__global__ void k_transmission(const float* __restrict__ v, double sigma, float2* __restrict__ t,
                               int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    sincos(sigma * (double)v[i], &s, &c);
    t[i] = make_float2((float)c, (float)s);
  }
}

__global__ void k_propagator_table(float2* __restrict__ ptab, int n, double cell, double lam,
                                   double dz, float scale) {
  const int nh = n / 2, nq = n / 4;
  const int total = nh * nh;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int a = i / nh, b = i % nh;             // [kx'][ky']
    const int kx = a < nq ? a : a - nh;
    const int ky = b < nq ? b : b - nh;
    const int64_t k2 = (int64_t)kx * kx + (int64_t)ky * ky;
    float2 p = make_float2(0.f, 0.f);
    if (16 * k2 < (int64_t)n * n) {
      // phase = -pi * lam * dz * |k|^2, argument (in units of pi) reduced mod 2 in FP64
      double arg = lam * dz * (double)k2 / (cell * cell);
      arg -= 2.0 * floor(0.5 * arg);
      float s, c;
      sincospif(-(float)arg, &s, &c);
      p = make_float2(c * scale, s * scale);
    }
    ptab[i] = p;
  }
}

// One block writes kInitRows rows of one wave as float4 pairs of row-spectrum values
// (N/2 is even, so every row starts on a 16-byte boundary); only the thread holding
// column box(px) computes a nonzero value.
constexpr int kInitRows = 16;

__global__ void k_init_plane_waves(float2* __restrict__ W, int n, const int* __restrict__ px,
                                   const int* __restrict__ py, const float2* __restrict__ amp,
                                   const float2* __restrict__ tw) {
  const int nh = n / 2, npair = nh / 2;
  const int64_t wave = blockIdx.y;
  if (!STEM_REQUIRE(px[wave] >= -nh && px[wave] < nh)) return;   // beam column on the grid
  const int col = px[wave] >= 0 ? px[wave] : px[wave] + nh;
  const float2 a = amp[wave];
  const int q = py[wave];
  float4* base = reinterpret_cast<float4*>(W + wave * (int64_t)n * nh);
  const int y0 = blockIdx.x * kInitRows;
  for (int r = 0; r < kInitRows && y0 + r < n; ++r) {
    const int y = y0 + r;
    float4* row = base + (int64_t)y * npair;
    for (int k2 = threadIdx.x; k2 < npair; k2 += blockDim.x) {
      float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k2 == (col >> 1)) {
        int m = (int)(((int64_t)q * y) % n);
        if (m < 0) m += n;
        const float2 v = cmul(a, cconj(tw[m]));   // exp(+2 pi i q y / N)
        if (col & 1) {
          o.z = v.x;
          o.w = v.y;
        } else {
          o.x = v.x;
          o.y = v.y;
        }
      }
      row[k2] = o;
    }
  }
}

__global__ void k_probe_init(float2* __restrict__ W, int n, const double* __restrict__ rx,
                             const double* __restrict__ ry, const int* __restrict__ bp,
                             const int* __restrict__ bq, int n_beams, int f, double cell,
                             double c, const float2* __restrict__ tw) {
  extern __shared__ float2 coef[];   // [n_beams]
  const int nh = n / 2, nq = n / 4;
  const int64_t wave = blockIdx.y;
  for (int j = threadIdx.x; j < n_beams; j += blockDim.x) {
    // a_j = c exp(-2 pi i f (p Rx + q Ry) / L), phase in cycles reduced in FP64
    double cyc = (double)f * ((double)bp[j] * rx[wave] + (double)bq[j] * ry[wave]) / cell;
    cyc -= floor(cyc);
    double s, co;
    sincospi(-2.0 * cyc, &s, &co);
    coef[j] = make_float2((float)(c * co), (float)(c * s));
  }
  __syncthreads();
  const int64_t per = (int64_t)n * nh;
  float2* dst = W + wave * per;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / nh), k = (int)(i % nh);
    const int kx = k < nq ? k : k - nh;
    float2 v = make_float2(0.f, 0.f);
    for (int j = 0; j < n_beams; ++j) {
      if (f * bp[j] != kx) continue;
      int m = (int)(((int64_t)f * bq[j] * y) % n);
      if (m < 0) m += n;
      v = cadd(v, cmul(coef[j], cconj(tw[m])));
    }
    dst[i] = v;
  }
}

// One CTA per (output row y, spawn).  Writes the row-pass output form of the
// inelastic wave Interp(H . D) of Eq. Hn0Psi: only even rows y = 2m carry the
// N/2-grid row spectrum 4 * sum_u x(m,u) exp(-2 pi i kx u/(N/2)), odd rows are
// zero; the column pass only looks at the band box of the y-spectrum, where this
// equals the spectrum of the Fourier-interpolated wave.
__global__ void k_spawn(int n, const int* __restrict__ src, const int* __restrict__ site,
                        const int* __restrict__ type, int first_wave, const float2* __restrict__ D,
                        const float2* __restrict__ H, int n_types, int h_mul, int w,
                        const int* __restrict__ win_x0, const int* __restrict__ win_y0,
                        float2* __restrict__ Phi, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  float2* xrow = sm;                 // [w] x(m, u) = H * D
  int* gcol = (int*)(sm + w);        // [w] grid column of u
  const int nh = n / 2, nq = n / 4;
  const int y = blockIdx.x;
  const int k = blockIdx.y;
  const int s = site[k];
  if (!STEM_REQUIRE(s >= 0 && src[k] >= 0 && type[k] >= 0 && type[k] < n_types &&
                    window_ok(win_x0[s], win_y0[s], w, nh)))
    return;   // the whole block, before any barrier
  const int64_t wave = first_wave + k;
  float2* dst = Phi + (wave * n + y) * nh;
  int v = -1;
  if ((y & 1) == 0) {
    v = (y / 2 - win_y0[s]) % nh;
    if (v < 0) v += nh;
    if (v >= w) v = -1;
  }
  if (v < 0) {
    for (int i = threadIdx.x; i < nh; i += blockDim.x) dst[i] = make_float2(0.f, 0.f);
    return;
  }
  const float2* drow = D + (int64_t)src[k] * nh * nh + (int64_t)(y / 2) * nh;
  const float2* hrow = H + (((int64_t)s * h_mul * n_types + type[k]) * w + v) * w;
  for (int u = threadIdx.x; u < w; u += blockDim.x) {
    const int g = (win_x0[s] + u) % nh;
    gcol[u] = g;
    xrow[u] = cmul(hrow[u], drow[g]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nh; i += blockDim.x) {
    const int kx = i < nq ? i : i - nh;
    float2 acc = make_float2(0.f, 0.f);
    for (int u = 0; u < w; ++u) {
      int m = (int)(((int64_t)2 * kx * gcol[u]) % n);
      if (m < 0) m += n;
      acc = cadd(acc, cmul(xrow[u], tw[m]));   // exp(-2 pi i kx g / (N/2))
    }
    dst[i] = cscale(acc, 4.f);
  }
}

template <int N>
cudaError_t row_pass_n(int n_waves, const float2* W, float2* Phi, const float2* t, int conj_t,
                       int store_mode, float2* S, int s_waves, int64_t s_stride, int fft_out,
                       const float2* tw, cudaStream_t s) {
  constexpr int ROWS = RegFFT<N>::ROWS;
  const size_t smem = (size_t)kRowWarps * ROWS * spad_len(N) * sizeof(float2);
  auto kern = [] {
    if constexpr (N == 768) return k_row_pass_capped<N>;
    else return k_row_pass<N>;
  }();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(N / (kRowWarps * ROWS), n_waves);
  kern<<<grid, kRowWarps * 32, smem, s>>>(W, Phi, t, conj_t, store_mode, S, s_waves, s_stride,
                                          fft_out, tw);
  return cudaGetLastError();
}

template <int N>
cudaError_t col_pass_n(int n_waves, const float2* Phi, float2* W, const float2* ptab, int conj_p,
                       int mode, const uint8_t* det_mask, const int* wave_out, double* det_acc,
                       double det_scale, const float2* tw, cudaStream_t s) {
  constexpr int ROWS = RegFFT<N>::ROWS;
  const size_t smem = (size_t)kColCB * ROWS * col_ld<N>() * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_col_pass<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(N / 2 / (kColCB * ROWS), n_waves);
  k_col_pass<N><<<grid, kColCB * 32, smem, s>>>(Phi, W, ptab, conj_p, mode, det_mask, wave_out,
                                                det_acc, det_scale, tw);
  return cudaGetLastError();
}

}  // namespace

#define EELS_FOR_EACH_N(X) X(64) X(128) X(256) X(384) X(512) X(768) X(1024)

bool grid_supported(int n) {
#define EELS_CASE(NN) if (n == NN) return true;
  EELS_FOR_EACH_N(EELS_CASE)
#undef EELS_CASE
  return false;
}

int twiddle_table_size(int n) { return twiddle_table_len(n); }

void fill_twiddle_tables(int n, float2* h) {
  auto root = [n](int64_t e) {
    const double a = 2.0 * 3.14159265358979323846 * (double)(e % n) / (double)n;
    return make_float2((float)std::cos(a), (float)-std::sin(a));
  };
  for (int k = 0; k < n; ++k) h[k] = root(k);
  for (int k = n; k < twiddle_table_len(n); ++k) h[k] = make_float2(0.f, 0.f);
  if (plan_len(n) != 2) return;
  for (int rev = 0; rev < 2; ++rev) {
    // stage 1 of the plan: radix r1 after a first stage of radix r0 (r0 r1 = n)
    const int r0 = plan_radix(n, rev ? 1 : 0), r1 = plan_radix(n, rev ? 0 : 1);
    float2* t = h + twiddle_table_offset(n, rev != 0);
    for (int q = 0; q < r1; ++q)
      for (int k = 0; k < r0; ++k) t[q * r0 + k] = root((int64_t)q * k);
  }
}

cudaError_t launch_row_pass(int n, int n_waves, const float2* W, float2* Phi, const float2* t,
                            int conj_t, int store_mode, float2* S, int s_waves, int64_t s_stride,
                            int fft_out, const float2* tw, cudaStream_t s) {
  if (n_waves <= 0) return cudaSuccess;
#define EELS_CASE(NN) \
  if (n == NN) return row_pass_n<NN>(n_waves, W, Phi, t, conj_t, store_mode, S, s_waves, s_stride, fft_out, tw, s);
  EELS_FOR_EACH_N(EELS_CASE)
#undef EELS_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_col_pass(int n, int n_waves, const float2* Phi, float2* W, const float2* ptab,
                            int conj_p, int mode, const uint8_t* det_mask, const int* wave_out,
                            double* det_acc, double det_scale, const float2* tw, cudaStream_t s) {
  if (n_waves <= 0) return cudaSuccess;
#define EELS_CASE(NN) \
  if (n == NN) return col_pass_n<NN>(n_waves, Phi, W, ptab, conj_p, mode, det_mask, wave_out, det_acc, det_scale, tw, s);
  EELS_FOR_EACH_N(EELS_CASE)
#undef EELS_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_transmission(const float* v, double sigma, float2* t, int64_t count,
                                cudaStream_t s) {
  k_transmission<<<1184, 256, 0, s>>>(v, sigma, t, count);
  return cudaGetLastError();
}

cudaError_t launch_propagator_table(float2* ptab, int n, double cell, double lam, double dz,
                                    float scale, cudaStream_t s) {
  const int total = (n / 2) * (n / 2);
  k_propagator_table<<<(total + 255) / 256, 256, 0, s>>>(ptab, n, cell, lam, dz, scale);
  return cudaGetLastError();
}

cudaError_t launch_init_plane_waves(float2* W, int n, int n_waves, const int* px, const int* py,
                                    const float2* amp, const float2* tw, cudaStream_t s) {
  if (n_waves <= 0) return cudaSuccess;
  dim3 grid((unsigned)((n + kInitRows - 1) / kInitRows), n_waves);
  k_init_plane_waves<<<grid, 128, 0, s>>>(W, n, px, py, amp, tw);
  return cudaGetLastError();
}

cudaError_t launch_probe_init(float2* W, int n, int n_probes, const double* rx, const double* ry,
                              const int* bp, const int* bq, int n_beams, int f, double cell,
                              double c, const float2* tw, cudaStream_t s) {
  if (n_probes <= 0) return cudaSuccess;
  const int64_t per = (int64_t)n * (n / 2);
  dim3 grid((unsigned)((per + 255) / 256), n_probes);
  k_probe_init<<<grid, 256, n_beams * sizeof(float2), s>>>(W, n, rx, ry, bp, bq, n_beams, f, cell,
                                                           c, tw);
  return cudaGetLastError();
}

cudaError_t launch_spawn(int n, const SpawnList& sp, const float2* D, const float2* H, int n_types,
                         int h_mul, int w, const int* win_x0, const int* win_y0, float2* Phi,
                         const float2* tw, cudaStream_t s) {
  if (sp.count <= 0) return cudaSuccess;
  dim3 grid(n, sp.count);
  const size_t smem = (size_t)w * (sizeof(float2) + sizeof(int));
  k_spawn<<<grid, 256, smem, s>>>(n, sp.src, sp.site, sp.type, sp.first_wave, D, H, n_types,
                                  h_mul, w, win_x0, win_y0, Phi, tw);
  return cudaGetLastError();
}

EELS_CHECK_COLLECTOR(collect_checks_ms)

}  // namespace eels
