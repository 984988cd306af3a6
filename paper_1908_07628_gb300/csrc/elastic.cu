// Elastic STEM images (ADF, incoherent bright field) from the exit-surface S-matrix
// (Sec. IV D), in three passes over a batch of scan rows:
//
//   cut pass:     psi_R on its L/f cut, psi_R[y'][x'] = sum_j ax_j(Rx) ay_j(Ry)
//                 S_exit[j][(y0(R) + y') % (N/2)][(x0(R) + x') % (N/2)]; the S-matrix
//                 beams are combined with the probe coefficients of Eq. illum (Sec. III).
//   row pass:     forward DFT of every cut row (register-resident FFT).
//   column pass:  forward DFT of every cut column, then |.|^2 summed over the bins of
//                 each detector (FP64 accumulation per probe and detector).
//
// Scale: S_exit is stored N times the true decimated exit wave and the probe
// coefficients carry no c = f/sqrt(n_in); the caller applies the constant.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace eels {

namespace {

constexpr int kCutProbes = 16;    // probes of one scan row per CTA of the cut pass
constexpr int kCutThreads = 256;
constexpr int kBeamChunk = 32;    // beams whose coefficients are staged at a time
constexpr int kFftWarps = 8;

// One CTA: up to 16 consecutive probes ix0.. of scan row iy, one cut row y'.  Every
// S_exit element of the group's column span is loaded once and used by all probes
// whose cut contains it.
__global__ void __launch_bounds__(kCutThreads)
k_exit_cut(const float2* __restrict__ S, int n_in, int nh, int m,
           const float2* __restrict__ ax, const float2* __restrict__ ay, int n_sx, int n_sy,
           const int* __restrict__ wx, const int* __restrict__ wy, int iy0,
           float2* __restrict__ out) {
  __shared__ __align__(16) float2 coef[kBeamChunk][kCutProbes];
  __shared__ int dx[kCutProbes];
  const int ix0 = blockIdx.x * kCutProbes;
  const int np = min(kCutProbes, n_sx - ix0);
  const int yp = blockIdx.y;
  const int iyl = blockIdx.z;
  const int iy = iy0 + iyl;
  // window origins on the grid (the block's row origin and first column origin decide
  // for the whole block; a bad later column origin is replaced by the first)
  if (!STEM_REQUIRE(wy[iy] >= 0 && wy[iy] < nh && wx[ix0] >= 0 && wx[ix0] < nh)) return;
  const int y = (wy[iy] + yp) % nh;
  const int xa = wx[ix0];
  if (threadIdx.x < kCutProbes) {
    int xg = threadIdx.x < np ? wx[ix0 + threadIdx.x] : xa;
    if (!STEM_REQUIRE(xg >= 0 && xg < nh)) xg = xa;
    dx[threadIdx.x] = (xg - xa + nh) % nh;
  }
  __syncthreads();
  int span = 0;
  for (int g = 0; g < np; ++g) span = max(span, dx[g]);
  const int U = min(span + m, nh);   // columns xa .. xa + U - 1 (cyclic)
  const int64_t plane = (int64_t)nh * nh;
  const float2* Srow = S + (int64_t)y * nh;

  for (int u0 = 0; u0 < U; u0 += kCutThreads) {
    const int u = u0 + threadIdx.x;
    const bool active = u < U;
    const int x = (xa + (active ? u : 0)) % nh;
    float2 acc[kCutProbes];
#pragma unroll
    for (int g = 0; g < kCutProbes; ++g) acc[g] = make_float2(0.f, 0.f);
    for (int j0 = 0; j0 < n_in; j0 += kBeamChunk) {
      const int jc = min(kBeamChunk, n_in - j0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < kBeamChunk * kCutProbes; idx += kCutThreads) {
        const int jj = idx / kCutProbes, g = idx % kCutProbes;
        float2 c = make_float2(0.f, 0.f);
        if (jj < jc && g < np)
          c = cmul(ax[(int64_t)(j0 + jj) * n_sx + ix0 + g], ay[(int64_t)(j0 + jj) * n_sy + iy]);
        coef[jj][g] = c;
      }
      __syncthreads();
      if (active) {
        for (int jj = 0; jj < jc; ++jj) {
          const float2 s = __ldg(Srow + (int64_t)(j0 + jj) * plane + x);
          const float4* c4 = reinterpret_cast<const float4*>(&coef[jj][0]);
#pragma unroll
          for (int g2 = 0; g2 < kCutProbes / 2; ++g2) {
            const float4 c = c4[g2];
            acc[2 * g2] = cadd(acc[2 * g2], cmul(make_float2(c.x, c.y), s));
            acc[2 * g2 + 1] = cadd(acc[2 * g2 + 1], cmul(make_float2(c.z, c.w), s));
          }
        }
      }
    }
    if (active) {
#pragma unroll
      for (int g = 0; g < kCutProbes; ++g) {
        if (g < np) {
          const int xp = (u - dx[g] + nh) % nh;
          if (xp < m)
            out[(((int64_t)iyl * n_sx + ix0 + g) * m + yp) * m + xp] = acc[g];
        }
      }
    }
  }
}

// In-place forward DFT of `rows` rows of length M (ROWS rows per warp).
template <int M>
__global__ void __launch_bounds__(kFftWarps * 32)
k_cut_rows(float2* __restrict__ X, int64_t rows, const float2* __restrict__ tw) {
  constexpr int ROWS = RegFFT<M>::ROWS;
  constexpr int LDR = spad_len(M);
  constexpr int E = RegFFT<M>::E;
  using PF = Plan<M, false>;
  extern __shared__ float2 smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* sbuf = smem + warp * ROWS * LDR;
  const int64_t r0 = ((int64_t)blockIdx.x * kFftWarps + warp) * ROWS;
  if (r0 >= rows) return;
  float2 v[E];
  {
    constexpr int R0 = PF::R(0), NB0 = M / R0, PER0 = PF::per(0);
#pragma unroll
    for (int t = 0; t < PER0; ++t) {
      const int u = lane + 32 * t;
      const bool live = ((ROWS * NB0) % 32 == 0 || u < ROWS * NB0) && r0 + u / NB0 < rows;
      const float2* src = X + (r0 + u / NB0) * M;
#pragma unroll
      for (int q = 0; q < R0; ++q)
        v[t * R0 + q] = live ? src[u % NB0 + q * NB0] : make_float2(0.f, 0.f);
    }
  }
  reg_fft<M, false, false>(v, sbuf, LDR, tw, lane);
  {
    constexpr int RF = PF::R(PF::NS - 1), NBF = M / RF, PERF = PF::per(PF::NS - 1);
#pragma unroll
    for (int t = 0; t < PERF; ++t) {
      const int u = lane + 32 * t;
      if (((ROWS * NBF) % 32 == 0 || u < ROWS * NBF) && r0 + u / NBF < rows) {
        float2* dst = X + (r0 + u / NBF) * M;
#pragma unroll
        for (int q = 0; q < RF; ++q) dst[u % NBF + q * NBF] = v[t * RF + q];
      }
    }
  }
}

// Forward DFT of every column of cut blockIdx.y (ROWS columns per warp), then
// sum |X|^2 over each detector's bins (bit d of mask[ky][kx]) into img[d][probe].
template <int M>
__global__ void __launch_bounds__(kFftWarps * 32)
k_cut_cols_detect(const float2* __restrict__ X, const uint8_t* __restrict__ mask, int n_det,
                  int n_sx, int iy0, int64_t img_stride, double* __restrict__ img,
                  const float2* __restrict__ tw) {
  constexpr int ROWS = RegFFT<M>::ROWS;
  constexpr int LDR = spad_len(M);
  constexpr int E = RegFFT<M>::E;
  using PF = Plan<M, false>;
  extern __shared__ float2 smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* sbuf = smem + warp * ROWS * LDR;
  const int c0 = (blockIdx.x * kFftWarps + warp) * ROWS;
  if (c0 >= M) return;
  const float2* cut = X + (int64_t)blockIdx.y * M * M;
  float2 v[E];
  {
    constexpr int R0 = PF::R(0), NB0 = M / R0, PER0 = PF::per(0);
#pragma unroll
    for (int t = 0; t < PER0; ++t) {
      const int u = lane + 32 * t;
      const int col = c0 + u / NB0;
      const bool live = ((ROWS * NB0) % 32 == 0 || u < ROWS * NB0) && col < M;
#pragma unroll
      for (int q = 0; q < R0; ++q)
        v[t * R0 + q] = live ? cut[(int64_t)(u % NB0 + q * NB0) * M + col] : make_float2(0.f, 0.f);
    }
  }
  reg_fft<M, false, false>(v, sbuf, LDR, tw, lane);
  float acc[kMaxDetectors];
#pragma unroll
  for (int d = 0; d < kMaxDetectors; ++d) acc[d] = 0.f;
  {
    constexpr int RF = PF::R(PF::NS - 1), NBF = M / RF, PERF = PF::per(PF::NS - 1);
#pragma unroll
    for (int t = 0; t < PERF; ++t) {
      const int u = lane + 32 * t;
      const int col = c0 + u / NBF;
      if (((ROWS * NBF) % 32 == 0 || u < ROWS * NBF) && col < M) {
#pragma unroll
        for (int q = 0; q < RF; ++q) {
          const int ky = u % NBF + q * NBF;
          const unsigned bits = mask[ky * M + col];
          if (bits) {
            const float2 z = v[t * RF + q];
            const float p = fmaf(z.x, z.x, z.y * z.y);
#pragma unroll
            for (int d = 0; d < kMaxDetectors; ++d)
              if (bits & (1u << d)) acc[d] += p;
          }
        }
      }
    }
  }
  const int cutg = blockIdx.y;
  const int64_t probe = (int64_t)iy0 * n_sx + cutg;
  for (int d = 0; d < n_det; ++d) {
    float a = acc[d];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0 && a != 0.f) atomicAdd(img + d * img_stride + probe, (double)a);
  }
}

template <int M>
cudaError_t cut_fft_detect(float2* X, int n_cut, const uint8_t* mask, int n_det, int n_sx,
                           int iy0, int64_t img_stride, double* img, const float2* tw,
                           cudaStream_t s) {
  constexpr int ROWS = RegFFT<M>::ROWS;
  const size_t smem = (size_t)kFftWarps * ROWS * spad_len(M) * sizeof(float2);
  static std::atomic<uint64_t> rows_attr{0}, cols_attr{0};
  cudaError_t e0 = smem_attr_once(k_cut_rows<M>, smem, rows_attr);
  if (e0 != cudaSuccess) return e0;
  e0 = smem_attr_once(k_cut_cols_detect<M>, smem, cols_attr);
  if (e0 != cudaSuccess) return e0;
  const int64_t rows = (int64_t)n_cut * M;
  const int64_t per_cta = (int64_t)kFftWarps * ROWS;
  k_cut_rows<M><<<(unsigned)((rows + per_cta - 1) / per_cta), kFftWarps * 32, smem, s>>>(X, rows, tw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 g((unsigned)((M + per_cta - 1) / per_cta), (unsigned)n_cut);
  k_cut_cols_detect<M><<<g, kFftWarps * 32, smem, s>>>(X, mask, n_det, n_sx, iy0, img_stride, img, tw);
  return cudaGetLastError();
}

__global__ void k_divide(double* __restrict__ map, const double* __restrict__ bf, int n_types,
                         int64_t n_pix) {
  const int64_t total = (int64_t)n_types * n_pix;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    map[i] = map[i] / bf[i % n_pix];
}

}  // namespace

cudaError_t launch_divide(double* map, const double* bf, int n_types, int64_t n_pix,
                          cudaStream_t s) {
  if (n_types <= 0 || n_pix <= 0) return cudaSuccess;
  const int64_t total = (int64_t)n_types * n_pix;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
  k_divide<<<blocks, 256, 0, s>>>(map, bf, n_types, n_pix);
  return cudaGetLastError();
}

bool cut_supported(int m) {
  switch (m) {
    case 16: case 32: case 48: case 64: case 96: case 128: case 192: case 256: case 384: case 512:
      return true;
    default:
      return false;
  }
}

cudaError_t launch_exit_cut(const float2* S, int n_in, int nh, int m, const float2* ax,
                            const float2* ay, int n_sx, int n_sy, const int* wx, const int* wy,
                            int iy0, int n_rows, float2* out, cudaStream_t s) {
  if (n_rows <= 0) return cudaSuccess;
  dim3 g((unsigned)((n_sx + kCutProbes - 1) / kCutProbes), (unsigned)m, (unsigned)n_rows);
  k_exit_cut<<<g, kCutThreads, 0, s>>>(S, n_in, nh, m, ax, ay, n_sx, n_sy, wx, wy, iy0, out);
  return cudaGetLastError();
}

cudaError_t launch_cut_detect(int m, float2* X, int n_cut, const uint8_t* mask, int n_det,
                              int n_sx, int iy0, int64_t img_stride, double* img,
                              const float2* tw, cudaStream_t s) {
  if (n_cut <= 0) return cudaSuccess;
  switch (m) {
#define EELS_CUT_CASE(MM) \
    case MM: return cut_fft_detect<MM>(X, n_cut, mask, n_det, n_sx, iy0, img_stride, img, tw, s);
    EELS_CUT_CASE(16) EELS_CUT_CASE(32) EELS_CUT_CASE(48) EELS_CUT_CASE(64) EELS_CUT_CASE(96)
    EELS_CUT_CASE(128) EELS_CUT_CASE(192) EELS_CUT_CASE(256) EELS_CUT_CASE(384)
    EELS_CUT_CASE(512)
#undef EELS_CUT_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

EELS_CHECK_COLLECTOR(collect_checks_elastic)

}  // namespace eels
