// Device helpers shared by the STEM-EELS kernels: complex float2 arithmetic and a
// warp-synchronous mixed-radix Stockham FFT operating on one row in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace eels {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by +i (s = +1) or -i (s = -1)
template <int S>
__device__ __forceinline__ float2 mul_i(float2 a) {
  return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// Radix plan: N = 3^a 2^b.  Radix-3 stages first, then radix-8 stages, and the
// remaining factor of the power of two as 4, 4x4 or 2.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int plan_len(int n) {
  int c = 0;
  while (n % 3 == 0) { ++c; n /= 3; }
  int b = 0;
  while (n > 1) { ++b; n /= 2; }
  if (b % 3 == 0) return c + b / 3;
  if (b % 3 == 1) return b >= 4 ? c + (b - 4) / 3 + 2 : c + 1;
  return c + (b - 2) / 3 + 1;
}

__host__ __device__ constexpr int plan_radix(int n, int s) {
  int c = 0;
  int m = n;
  while (m % 3 == 0) { ++c; m /= 3; }
  if (s < c) return 3;
  int b = 0;
  while (m > 1) { ++b; m /= 2; }
  int k = s - c;
  int n8 = 0, tail0 = 0, tail1 = 0;
  if (b % 3 == 0) { n8 = b / 3; tail0 = 0; tail1 = 0; }
  else if (b % 3 == 1) {
    if (b >= 4) { n8 = (b - 4) / 3; tail0 = 4; tail1 = 4; }
    else { n8 = 0; tail0 = 2; tail1 = 0; }
  } else { n8 = (b - 2) / 3; tail0 = 4; tail1 = 0; }
  if (k < n8) return 8;
  if (k == n8) return tail0;
  if (k == n8 + 1) return tail1;
  return 0;
}

// In-register DFT of length R.  INV = false: X_q = sum_n x_n exp(-2 pi i n q / R);
// INV = true: the + sign.  Unnormalised.
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* u);

template <>
__device__ __forceinline__ void dft<2, false>(float2* u) { float2 a = u[0]; u[0] = cadd(a, u[1]); u[1] = csub(a, u[1]); }
template <>
__device__ __forceinline__ void dft<2, true>(float2* u) { float2 a = u[0]; u[0] = cadd(a, u[1]); u[1] = csub(a, u[1]); }

template <bool INV>
__device__ __forceinline__ void dft4(float2& u0, float2& u1, float2& u2, float2& u3) {
  constexpr int S = INV ? 1 : -1;
  float2 t0 = cadd(u0, u2), t1 = csub(u0, u2);
  float2 t2 = cadd(u1, u3), t3 = mul_i<S>(csub(u1, u3));
  u0 = cadd(t0, t2);
  u2 = csub(t0, t2);
  u1 = cadd(t1, t3);
  u3 = csub(t1, t3);
}

template <>
__device__ __forceinline__ void dft<4, false>(float2* u) { dft4<false>(u[0], u[1], u[2], u[3]); }
template <>
__device__ __forceinline__ void dft<4, true>(float2* u) { dft4<true>(u[0], u[1], u[2], u[3]); }

template <bool INV>
__device__ __forceinline__ void dft8(float2* u) {
  constexpr int S = INV ? 1 : -1;
  constexpr float H = 0.70710678118654752440f;   // 1/sqrt(2)
  float2 e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6];
  float2 o0 = u[1], o1 = u[3], o2 = u[5], o3 = u[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // o_q *= w8^q, w8 = exp(S 2 pi i / 8)
  o1 = make_float2(H * (o1.x - S * o1.y), H * (o1.y + S * o1.x));
  o2 = mul_i<S>(o2);
  o3 = make_float2(H * (-o3.x - S * o3.y), H * (-o3.y + S * o3.x));
  u[0] = cadd(e0, o0); u[4] = csub(e0, o0);
  u[1] = cadd(e1, o1); u[5] = csub(e1, o1);
  u[2] = cadd(e2, o2); u[6] = csub(e2, o2);
  u[3] = cadd(e3, o3); u[7] = csub(e3, o3);
}
template <>
__device__ __forceinline__ void dft<8, false>(float2* u) { dft8<false>(u); }
template <>
__device__ __forceinline__ void dft<8, true>(float2* u) { dft8<true>(u); }

template <bool INV>
__device__ __forceinline__ void dft3(float2* u) {
  constexpr float S3 = (INV ? 1.0f : -1.0f) * 0.86602540378443864676f;   // sign * sqrt(3)/2
  float2 t1 = cadd(u[1], u[2]);
  float2 t2 = csub(u[1], u[2]);
  float2 m = make_float2(u[0].x - 0.5f * t1.x, u[0].y - 0.5f * t1.y);
  float2 r = make_float2(-S3 * t2.y, S3 * t2.x);   // i * S3 * t2
  u[0] = cadd(u[0], t1);
  u[1] = cadd(m, r);
  u[2] = csub(m, r);
}
template <>
__device__ __forceinline__ void dft<3, false>(float2* u) { dft3<false>(u); }
template <>
__device__ __forceinline__ void dft<3, true>(float2* u) { dft3<true>(u); }

// ---------------------------------------------------------------------------
// Register-resident warp FFT.
//
// A length-N sequence is spread over the 32 lanes of a warp.  For a stage of
// radix R the lane holds x[b + q N/R] for its butterflies b = lane + 32 t
// (t < ceil(N/R/32)) in v[t R + q].  Between stages the outputs are exchanged
// through the warp's padded shared-memory buffer (Stockham order); the first
// stage reads and the last stage leaves its data in registers.  The last stage of
// a Stockham pass writes x[b + q N/R], the same layout the first stage of a pass
// with the same radix reads, so an inverse transform run with the reversed radix
// plan feeds a forward transform (and vice versa) without any exchange.
// ---------------------------------------------------------------------------
template <int N, bool REV>
struct Plan {
  static constexpr int NS = plan_len(N);
  __host__ __device__ static constexpr int R(int s) {
    return REV ? plan_radix(N, NS - 1 - s) : plan_radix(N, s);
  }
  __host__ __device__ static constexpr int P(int s) {
    int p = 1;
    for (int i = 0; i < s; ++i) p *= R(i);
    return p;
  }
  __host__ __device__ static constexpr int elems(int s) {
    return ((N / R(s) + 31) / 32) * R(s);
  }
  __host__ __device__ static constexpr int max_elems() {
    int m = 0;
    for (int i = 0; i < NS; ++i) m = elems(i) > m ? elems(i) : m;
    return m;
  }
};

template <int N>
struct RegFFT {
  static constexpr int E = Plan<N, false>::max_elems() > Plan<N, true>::max_elems()
                               ? Plan<N, false>::max_elems()
                               : Plan<N, true>::max_elems();
};

// padded shared-memory index: one spare slot every 8 elements
__device__ __forceinline__ int spad(int j) { return j + (j >> 3); }
__host__ __device__ constexpr int spad_len(int n) { return n + n / 8; }

template <int N, bool INV, bool REV, int S>
__device__ __forceinline__ void reg_fft_stage(float2* v, float2* sbuf,
                                              const float2* __restrict__ tw, int lane) {
  using PL = Plan<N, REV>;
  constexpr int R = PL::R(S), P = PL::P(S), NB = N / R, PER = (NB + 31) / 32;
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int b = lane + 32 * t;
    if (NB % 32 == 0 || b < NB) {
      if constexpr (P > 1) {
        const int k = b % P;
#pragma unroll
        for (int q = 1; q < R; ++q) {
          float2 w = __ldg(tw + q * k * (N / (P * R)));
          if (INV) w.y = -w.y;
          v[t * R + q] = cmul(v[t * R + q], w);
        }
      }
      dft<R, INV>(v + t * R);
    }
  }
  if constexpr (S + 1 < PL::NS) {
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int b = lane + 32 * t;
      if (NB % 32 == 0 || b < NB) {
        const int k = b % P;
        const int j0 = (b - k) * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) sbuf[spad(j0 + q * P)] = v[t * R + q];
      }
    }
    __syncwarp();
    constexpr int R2 = PL::R(S + 1), NB2 = N / R2, PER2 = (NB2 + 31) / 32;
#pragma unroll
    for (int t = 0; t < PER2; ++t) {
      const int b = lane + 32 * t;
      if (NB2 % 32 == 0 || b < NB2) {
#pragma unroll
        for (int q = 0; q < R2; ++q) v[t * R2 + q] = sbuf[spad(b + q * NB2)];
      }
    }
    __syncwarp();
    reg_fft_stage<N, INV, REV, S + 1>(v, sbuf, tw, lane);
  }
}

// Transform the warp-held sequence.  On entry v holds x[b + q N/R0] (R0 = first
// radix of the plan), on exit X[b + q N/RL] (RL = last radix).  tw[n] = exp(-2 pi i n/N).
template <int N, bool INV, bool REV>
__device__ __forceinline__ void reg_fft(float2* v, float2* sbuf, const float2* __restrict__ tw,
                                        int lane) {
  reg_fft_stage<N, INV, REV, 0>(v, sbuf, tw, lane);
}

// One warp transforms buf[0..N) in place (Stockham autosort, natural order in
// and out).  tw[n] = exp(-2 pi i n / N) for n in [0, N).  Stage s with radix R
// and P = product of the earlier radices: butterfly b reads buf[b + q N/R],
// multiplies by exp(-+2 pi i q (b mod P) / (P R)), does a radix-R DFT and writes
// buf[(b - b mod P) R + b mod P + q P].
template <int N, bool INV, int STAGE = 0, int P = 1>
__device__ __forceinline__ void warp_fft(float2* buf, const float2* __restrict__ tw, int lane) {
  constexpr int R = plan_radix(N, STAGE);
  if constexpr (R != 0) {
    constexpr int NB = N / R;
    constexpr int PER = (NB + 31) / 32;
    float2 u[PER][R];
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int b = lane + 32 * t;
      if (NB % 32 == 0 || b < NB) {
#pragma unroll
        for (int q = 0; q < R; ++q) u[t][q] = buf[b + q * NB];
      }
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int b = lane + 32 * t;
      if (NB % 32 == 0 || b < NB) {
        const int k = b % P;
        if constexpr (P > 1) {
#pragma unroll
          for (int q = 1; q < R; ++q) {
            float2 w = tw[q * k * (N / (P * R))];
            if (INV) w.y = -w.y;
            u[t][q] = cmul(u[t][q], w);
          }
        }
        dft<R, INV>(u[t]);
        const int j = (b - k) * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) buf[j + q * P] = u[t][q];
      }
    }
    __syncwarp();
    warp_fft<N, INV, STAGE + 1, P * R>(buf, tw, lane);
  }
}

}  // namespace eels
