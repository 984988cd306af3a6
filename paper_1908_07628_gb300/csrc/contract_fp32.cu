// Inelastic contraction on CUDA cores in FP32 (Eq. SHn0 and the |.|^2 scan sum of
// the second algorithm listing of Sec. III).
//
//   GEMM 1   M_t[d][j] = sum_{p in W_s} conj(Sout[d][p]) H_t[p] Sin[j][p]
//   GEMM 2   V[d][R]   = sum_j M_t[d][j] a_j(R),  a_j(R) = ax[j][ix(R)] ay[j][iy(R)]
//            map[type_t][R] += sum_d |V[d][R]|^2        (FP64 atomics)
//
// Sin / Sout are depth planes [beam][N/2][N/2]; the window W_s of a site is the
// periodic w x w block at (win_x0, win_y0).  R runs over the scan positions whose
// PRISM window contains the site: a product of a column list and a row list.
#include "common.cuh"
#include "internal.h"

namespace eels {

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__device__ __forceinline__ void cfma_conj(float2& acc, float2 a, float2 b) {
  // acc += conj(a) * b
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

__global__ void __launch_bounds__(256)
k_gemm1(const float2* __restrict__ Sout, const float2* __restrict__ Sin, int nh, int n_out,
        int n_in, int w, const float2* __restrict__ H, int n_types, int h_mul,
        const int* __restrict__ tr_site,
        const int* __restrict__ tr_type, const int* __restrict__ win_x0,
        const int* __restrict__ win_y0, float2* __restrict__ M, int64_t m_stride) {
  __shared__ float2 As[TK][TM + 1];
  __shared__ float2 Bs[TK][TN + 1];
  __shared__ int pix[TK];
  __shared__ float2 hk[TK];
  const int t = blockIdx.z;
  const int s = tr_site[t];
  if (!STEM_REQUIRE(s >= 0 && tr_type[t] >= 0 && tr_type[t] < n_types &&
                    window_ok(win_x0[s], win_y0[s], w, nh)))
    return;   // the whole block, before any barrier
  const float2* Ht = H + ((int64_t)s * h_mul * n_types + tr_type[t]) * w * w;
  const int x0 = win_x0[s], y0 = win_y0[s];
  const int d0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t plane = (int64_t)nh * nh;
  const int P = w * w;
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);

  for (int kc = 0; kc < P; kc += TK) {
    if (threadIdx.x < TK) {
      const int p = kc + threadIdx.x;
      if (p < P) {
        const int v = p / w, u = p % w;
        const int gy = (y0 + v) % nh, gx = (x0 + u) % nh;
        pix[threadIdx.x] = gy * nh + gx;
        hk[threadIdx.x] = Ht[p];
      } else {
        pix[threadIdx.x] = -1;
        hk[threadIdx.x] = make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
    {
      const int k = threadIdx.x & (TK - 1);
      const int r0 = threadIdx.x >> 4;   // 0..15
      const int pk = pix[k];
      const float2 h = hk[k];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = r0 + 16 * i;
        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
        if (pk >= 0) {
          if (d0 + r < n_out) a = Sout[(int64_t)(d0 + r) * plane + pk];
          if (j0 + r < n_in) b = cmul(h, Sin[(int64_t)(j0 + r) * plane + pk]);
        }
        As[k][r] = a;
        Bs[k][r] = b;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int i = 0; i < 4; ++i) b[i] = Bs[k][tx + 16 * i];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) cfma_conj(acc[i][jj], a[i], b[jj]);
    }
    __syncthreads();
  }
  float2* Mt = M + (int64_t)t * m_stride;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int d = d0 + ty + 16 * i;
    if (d >= n_out) continue;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int j = j0 + tx + 16 * jj;
      if (j < n_in) Mt[(int64_t)d * n_in + j] = acc[i][jj];
    }
  }
}

__global__ void __launch_bounds__(256)
k_gemm2_abs2(const float2* __restrict__ M, int64_t m_stride, int n_out, int n_in,
             const float2* __restrict__ ax, const float2* __restrict__ ay, int n_sx, int n_sy,
             const int* __restrict__ tr_site, const int* __restrict__ tr_type,
             const int* __restrict__ xoff, const int* __restrict__ xcnt,
             const int* __restrict__ xlist, const int* __restrict__ yoff,
             const int* __restrict__ ycnt, const int* __restrict__ ylist,
             double* __restrict__ map) {
  __shared__ float2 As[TK][TM + 1];
  __shared__ float2 Bs[TK][TN + 1];
  __shared__ float red[16][TN];
  __shared__ int rix[TN], riy[TN];
  const int t = blockIdx.z;
  const int s = tr_site[t];
  const int nx = xcnt[s], ny = ycnt[s];
  const int nr = nx * ny;
  const int r0 = blockIdx.x * TN;
  if (r0 >= nr) return;
  const int d0 = blockIdx.y * TM;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (threadIdx.x < TN) {
    const int r = r0 + threadIdx.x;
    if (r < nr) {
      rix[threadIdx.x] = xlist[xoff[s] + r % nx];
      riy[threadIdx.x] = ylist[yoff[s] + r / nx];
      if (!STEM_REQUIRE(rix[threadIdx.x] >= 0 && rix[threadIdx.x] < n_sx &&
                        riy[threadIdx.x] >= 0 && riy[threadIdx.x] < n_sy && tr_type[t] >= 0))
        rix[threadIdx.x] = riy[threadIdx.x] = -1;   // skipped below
    } else {
      rix[threadIdx.x] = -1;
      riy[threadIdx.x] = -1;
    }
  }
  const float2* Mt = M + (int64_t)t * m_stride;
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int kc = 0; kc < n_in; kc += TK) {
    {
      const int k = threadIdx.x & (TK - 1);
      const int rr = threadIdx.x >> 4;
      const int j = kc + k;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = rr + 16 * i;
        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
        if (j < n_in) {
          if (d0 + r < n_out) a = Mt[(int64_t)(d0 + r) * n_in + j];
          if (rix[r] >= 0) b = cmul(ax[(int64_t)j * n_sx + rix[r]], ay[(int64_t)j * n_sy + riy[r]]);
        }
        As[k][r] = a;
        Bs[k][r] = b;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int i = 0; i < 4; ++i) b[i] = Bs[k][tx + 16 * i];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) cfma(acc[i][jj], a[i], b[jj]);
    }
    __syncthreads();
  }
  // |V|^2 summed over this tile's d rows, per scan position
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) sum = fmaf(acc[i][jj].x, acc[i][jj].x, fmaf(acc[i][jj].y, acc[i][jj].y, sum));
    red[ty][tx + 16 * jj] = sum;
  }
  __syncthreads();
  if (threadIdx.x < TN && rix[threadIdx.x] >= 0) {
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) sum += red[i][threadIdx.x];
    const int64_t idx = ((int64_t)tr_type[t] * n_sy + riy[threadIdx.x]) * n_sx + rix[threadIdx.x];
    atomicAdd(map + idx, (double)sum);
  }
}

__global__ void k_phase_table(float2* __restrict__ out, const int* __restrict__ bidx, int n_beams,
                              int f, double cell, double r0, double step, int n_pos,
                              int transposed, int r_first) {
  const int total = n_beams * n_pos;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int j = transposed ? i % n_beams : i / n_pos;
    const int r = transposed ? i / n_beams : i % n_pos;
    const double R = __dadd_rn(r0, __dmul_rn((double)(r_first + r), step));
    double cyc = (double)f * (double)bidx[j] * R / cell;   // exp(-2 pi i cyc)
    cyc -= floor(cyc);
    double s, c;
    sincospi(-2.0 * cyc, &s, &c);
    out[i] = make_float2((float)c, (float)s);
  }
}

__global__ void k_accumulate(double* __restrict__ acc, const double* __restrict__ x,
                             int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    acc[i] += x[i];
}

__global__ void k_scale(double* a, int64_t count, double scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] *= scale;
}

// a *= scale, and bit 2 of *flag set if any scaled value is not finite (NaN or Inf)
__global__ void k_scale_check(double* a, int64_t count, double scale, int* flag) {
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = a[i] * scale;
    a[i] = v;
    bad |= !isfinite(v);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 2);
}

}  // namespace

cudaError_t launch_gemm1_fp32(const float2* Sout, const float2* Sin, int nh, int n_out, int n_in,
                              int w, const float2* H, int n_types, int h_mul,
                              const TransitionBatch& tb, const int* win_x0, const int* win_y0,
                              float2* M, int64_t m_stride, cudaStream_t s) {
  if (tb.count <= 0) return cudaSuccess;
  dim3 grid((n_in + TN - 1) / TN, (n_out + TM - 1) / TM, tb.count);
  k_gemm1<<<grid, 256, 0, s>>>(Sout, Sin, nh, n_out, n_in, w, H, n_types, h_mul, tb.site, tb.type,
                               win_x0, win_y0, M, m_stride);
  return cudaGetLastError();
}

cudaError_t launch_gemm2_abs2_fp32(const float2* M, int64_t m_stride, int n_out, int n_in,
                                   const float2* ax, const float2* ay, int n_sx, int n_sy,
                                   const TransitionBatch& tb, const WindowLists& wl, double* map,
                                   cudaStream_t s) {
  if (tb.count <= 0 || wl.max_nr <= 0) return cudaSuccess;
  dim3 grid((wl.max_nr + TN - 1) / TN, (n_out + TM - 1) / TM, tb.count);
  k_gemm2_abs2<<<grid, 256, 0, s>>>(M, m_stride, n_out, n_in, ax, ay, n_sx, n_sy, tb.site, tb.type,
                                    wl.xoff, wl.xcnt, wl.xlist, wl.yoff, wl.ycnt, wl.ylist, map);
  return cudaGetLastError();
}

cudaError_t launch_phase_table(float2* out, const int* bidx, int n_beams, int f, double cell,
                               double r0, double step, int n_pos, cudaStream_t s, int transposed,
                               int r_first) {
  const int total = n_beams * n_pos;
  if (total <= 0) return cudaSuccess;
  k_phase_table<<<(total + 255) / 256, 256, 0, s>>>(out, bidx, n_beams, f, cell, r0, step, n_pos,
                                                    transposed, r_first);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(double* acc, const double* x, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_accumulate<<<256, 256, 0, s>>>(acc, x, count);
  return cudaGetLastError();
}

cudaError_t launch_scale_check(double* a, int64_t count, double scale, int* flag,
                               cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_scale_check<<<256, 256, 0, s>>>(a, count, scale, flag);
  return cudaGetLastError();
}

cudaError_t launch_scale(double* a, int64_t count, double scale, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_scale<<<256, 256, 0, s>>>(a, count, scale);
  return cudaGetLastError();
}

EELS_CHECK_COLLECTOR(collect_checks_fp32)

}  // namespace eels
