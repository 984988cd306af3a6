// Helpers shared by the STEM-EELS kernels: complex float2 arithmetic, small
// in-register DFTs, a register-resident mixed-radix Stockham FFT run by one warp, and a
// host helper that sets launch attributes once per device.
#pragma once

#include <atomic>
#include <cstdint>

#include <cuda_runtime.h>
#include <stdint.h>

namespace eels {

// Raises a kernel's dynamic shared-memory limit once per device.  `done` holds one bit
// per device ordinal that already has it; safe to call from several host threads (the
// map server's workers launch concurrently).
template <typename K>
inline cudaError_t smem_attr_once(K* kernel, size_t bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
  return e;
}

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
// Radix plans.  Two-stage plans with in-register radix-16/24/32 butterflies for the
// common grids 256, 512, 768, 1024 (one shared-memory exchange per transform).
__host__ __device__ constexpr int plan2_radix(int n, int s) {
  return n == 256 ? (s < 2 ? 16 : 0)
       : n == 512 ? (s == 0 ? 16 : s == 1 ? 32 : 0)
       : n == 768 ? (s == 0 ? 24 : s == 1 ? 32 : 0)
       : n == 1024 ? (s < 2 ? 32 : 0)
       : -1;
}

__host__ __device__ constexpr int plan_len_generic(int n);
__host__ __device__ constexpr int plan_radix_generic(int n, int s);

__host__ __device__ constexpr int plan_len(int n) {
  return plan2_radix(n, 0) > 0 ? 2 : plan_len_generic(n);
}
__host__ __device__ constexpr int plan_radix(int n, int s) {
  return plan2_radix(n, 0) > 0 ? plan2_radix(n, s) : plan_radix_generic(n, s);
}

// Sequences per warp: two where a single sequence would leave lanes idle in a stage.
__host__ __device__ constexpr int rows_per_warp(int n) { return (n == 256 || n == 512) ? 2 : 1; }

// Generic plan for N = 3^a 2^b: radix-3 stages first, then radix-8 stages, and the
// remaining factor of the power of two as 4, 4x4 or 2.
__host__ __device__ constexpr int plan_len_generic(int n) {
  int c = 0;
  while (n % 3 == 0) { ++c; n /= 3; }
  int b = 0;
  while (n > 1) { ++b; n /= 2; }
  if (b % 3 == 0) return c + b / 3;
  if (b % 3 == 1) return b >= 4 ? c + (b - 4) / 3 + 2 : c + 1;
  return c + (b - 2) / 3 + 1;
}

__host__ __device__ constexpr int plan_radix_generic(int n, int s) {
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
// `nz`: inputs that may be nonzero (see the input masks below); all by default.
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* u, unsigned nz = ~0u);

template <>
__device__ __forceinline__ void dft<2, false>(float2* u, unsigned) { float2 a = u[0]; u[0] = cadd(a, u[1]); u[1] = csub(a, u[1]); }
template <>
__device__ __forceinline__ void dft<2, true>(float2* u, unsigned) { float2 a = u[0]; u[0] = cadd(a, u[1]); u[1] = csub(a, u[1]); }

// Input masks.  The DFTs below take a bit mask `nz` of the inputs that may be nonzero
// (bit q for input q); inputs outside it must hold zero and the sums and differences
// with them are skipped.  The masks are compile-time constants once the fully unrolled
// transforms are inlined, so a pruned butterfly costs nothing at run time.  The first
// stage of an inverse transform of a band-limited sequence sees half its inputs zero.
//
// a + b and a - b where na / nb say whether a / b may be nonzero
__device__ __forceinline__ float2 cadd_nz(float2 a, float2 b, bool na, bool nb) {
  return na ? (nb ? cadd(a, b) : a) : (nb ? b : make_float2(0.f, 0.f));
}
__device__ __forceinline__ float2 csub_nz(float2 a, float2 b, bool na, bool nb) {
  return na ? (nb ? csub(a, b) : a) : (nb ? make_float2(-b.x, -b.y) : make_float2(0.f, 0.f));
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& u0, float2& u1, float2& u2, float2& u3,
                                     unsigned nz = 0xFu) {
  constexpr int S = INV ? 1 : -1;
  const bool n0 = nz & 1u, n1 = nz & 2u, n2 = nz & 4u, n3 = nz & 8u;
  float2 t0 = cadd_nz(u0, u2, n0, n2), t1 = csub_nz(u0, u2, n0, n2);
  float2 t2 = cadd_nz(u1, u3, n1, n3), t3 = mul_i<S>(csub_nz(u1, u3, n1, n3));
  const bool a = n0 || n2, b = n1 || n3;
  u0 = cadd_nz(t0, t2, a, b);
  u2 = csub_nz(t0, t2, a, b);
  u1 = cadd_nz(t1, t3, a, b);
  u3 = csub_nz(t1, t3, a, b);
}

template <>
__device__ __forceinline__ void dft<4, false>(float2* u, unsigned nz) { dft4<false>(u[0], u[1], u[2], u[3], nz); }
template <>
__device__ __forceinline__ void dft<4, true>(float2* u, unsigned nz) { dft4<true>(u[0], u[1], u[2], u[3], nz); }

template <bool INV>
__device__ __forceinline__ void dft8(float2* u, unsigned nz = 0xFFu) {
  constexpr int S = INV ? 1 : -1;
  constexpr float H = 0.70710678118654752440f;   // 1/sqrt(2)
  // masks of the even (u0, u2, u4, u6) and odd (u1, u3, u5, u7) inputs
  const unsigned me = (nz & 1u) | (nz >> 1 & 2u) | (nz >> 2 & 4u) | (nz >> 3 & 8u);
  const unsigned mo = (nz >> 1 & 1u) | (nz >> 2 & 2u) | (nz >> 3 & 4u) | (nz >> 4 & 8u);
  float2 e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6];
  float2 o0 = u[1], o1 = u[3], o2 = u[5], o3 = u[7];
  dft4<INV>(e0, e1, e2, e3, me);
  dft4<INV>(o0, o1, o2, o3, mo);
  // o_q *= w8^q, w8 = exp(S 2 pi i / 8)
  o1 = make_float2(H * (o1.x - S * o1.y), H * (o1.y + S * o1.x));
  o2 = mul_i<S>(o2);
  o3 = make_float2(H * (-o3.x - S * o3.y), H * (-o3.y + S * o3.x));
  const bool he = me != 0u, ho = mo != 0u;
  u[0] = cadd_nz(e0, o0, he, ho); u[4] = csub_nz(e0, o0, he, ho);
  u[1] = cadd_nz(e1, o1, he, ho); u[5] = csub_nz(e1, o1, he, ho);
  u[2] = cadd_nz(e2, o2, he, ho); u[6] = csub_nz(e2, o2, he, ho);
  u[3] = cadd_nz(e3, o3, he, ho); u[7] = csub_nz(e3, o3, he, ho);
}
template <>
__device__ __forceinline__ void dft<8, false>(float2* u, unsigned nz) { dft8<false>(u, nz); }
template <>
__device__ __forceinline__ void dft<8, true>(float2* u, unsigned nz) { dft8<true>(u, nz); }

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
__device__ __forceinline__ void dft<3, false>(float2* u, unsigned) { dft3<false>(u); }
template <>
__device__ __forceinline__ void dft<3, true>(float2* u, unsigned) { dft3<true>(u); }

// exp(2 pi i m / 32) components, FP64-rounded to FP32
__host__ __device__ constexpr float cos32(int m) {
  constexpr float c[32] = {1.0f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f,
                           7.071067812e-01f, 5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f,
                           0.0f, -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f,
                           -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f,
                           -1.0f, -9.807852804e-01f, -9.238795325e-01f, -8.314696123e-01f,
                           -7.071067812e-01f, -5.555702330e-01f, -3.826834324e-01f, -1.950903220e-01f,
                           0.0f, 1.950903220e-01f, 3.826834324e-01f, 5.555702330e-01f,
                           7.071067812e-01f, 8.314696123e-01f, 9.238795325e-01f, 9.807852804e-01f};
  return c[m & 31];
}
__host__ __device__ constexpr float sin32(int m) { return cos32(m - 8); }

// exp(2 pi i m / 24) components (multiples of 15 degrees)
__host__ __device__ constexpr float cos24(int m) {
  constexpr float c[24] = {1.0f, 9.659258263e-01f, 8.660254038e-01f, 7.071067812e-01f, 0.5f,
                           2.588190451e-01f, 0.0f, -2.588190451e-01f, -0.5f, -7.071067812e-01f,
                           -8.660254038e-01f, -9.659258263e-01f, -1.0f, -9.659258263e-01f,
                           -8.660254038e-01f, -7.071067812e-01f, -0.5f, -2.588190451e-01f, 0.0f,
                           2.588190451e-01f, 0.5f, 7.071067812e-01f, 8.660254038e-01f,
                           9.659258263e-01f};
  return c[((m % 24) + 24) % 24];
}
__host__ __device__ constexpr float sin24(int m) { return cos24(m - 6); }

// exp(sg 2 pi i m / R) for R dividing 32 or 24
template <int R>
__device__ __forceinline__ float2 croot(int m, float sg) {
  if constexpr (32 % R == 0) {
    return make_float2(cos32(m * (32 / R)), sg * sin32(m * (32 / R)));
  } else {
    static_assert(24 % R == 0, "composite radix must divide 32 or 24");
    return make_float2(cos24(m * (24 / R)), sg * sin24(m * (24 / R)));
  }
}

// a exp(+-2 pi i m / R) (+ for INV); quarter turns are exact sign swaps, not products
template <int R, bool INV>
__device__ __forceinline__ float2 rotate(float2 a, int m) {
  constexpr int S = INV ? 1 : -1;
  if ((4 * m) % R == 0) {
    const int quarter = (4 * m / R) % 4;
    return quarter == 0 ? a
         : quarter == 2 ? make_float2(-a.x, -a.y)
         : quarter == 1 ? mul_i<S>(a)
                        : mul_i<-S>(a);
  }
  return cmul(a, croot<R>(m, (float)S));
}

// In-register DFT of length R = R1 R2: n = R2 n1 + n2, k = k1 + R1 k2;
// DFT_R1 over n1, twiddle exp(+-2 pi i n2 k1 / R), DFT_R2 over n2.
template <int R1, int R2, bool INV>
__device__ __forceinline__ void dft_composite(float2* x, unsigned nz) {
  constexpr int R = R1 * R2;
  float2 y[R];
  unsigned live = 0u;   // n2 whose length-R1 transform has a nonzero input
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    float2 t[R1];
    unsigned sub = 0u;
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      t[n1] = x[R2 * n1 + n2];
      if (nz >> (R2 * n1 + n2) & 1u) sub |= 1u << n1;
    }
    if (sub) live |= 1u << n2;
    dft<R1, INV>(t, sub);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) y[n2 * R1 + k1] = rotate<R, INV>(t[k1], (n2 * k1) % R);
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    float2 t[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) t[n2] = y[n2 * R1 + k1];
    dft<R2, INV>(t, live);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = t[k2];
  }
}
template <>
__device__ __forceinline__ void dft<16, false>(float2* u, unsigned nz) { dft_composite<4, 4, false>(u, nz); }
template <>
__device__ __forceinline__ void dft<16, true>(float2* u, unsigned nz) { dft_composite<4, 4, true>(u, nz); }
template <>
__device__ __forceinline__ void dft<24, false>(float2* u, unsigned nz) { dft_composite<8, 3, false>(u, nz); }
template <>
__device__ __forceinline__ void dft<24, true>(float2* u, unsigned nz) { dft_composite<8, 3, true>(u, nz); }
template <>
__device__ __forceinline__ void dft<32, false>(float2* u, unsigned nz) { dft_composite<8, 4, false>(u, nz); }
template <>
__device__ __forceinline__ void dft<32, true>(float2* u, unsigned nz) { dft_composite<8, 4, true>(u, nz); }

// First-stage input mask of an inverse transform whose input is band-limited to
// |frequency| < N/4: for radix R (a multiple of 4) input q holds frequency b + q N/R with
// b < N/R, inside the band iff q < R/4 or q >= 3R/4.
__host__ __device__ constexpr unsigned band_mask(int r) {
  unsigned m = 0u;
  for (int q = 0; q < r; ++q)
    if (4 * q < r || 4 * q >= 3 * r) m |= 1u << q;
  return m;
}

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
  static constexpr int ROWS = rows_per_warp(N);
  __host__ __device__ static constexpr int R(int s) {
    return REV ? plan_radix(N, NS - 1 - s) : plan_radix(N, s);
  }
  __host__ __device__ static constexpr int P(int s) {
    int p = 1;
    for (int i = 0; i < s; ++i) p *= R(i);
    return p;
  }
  // butterflies of all ROWS sequences of a stage, spread over the 32 lanes
  __host__ __device__ static constexpr int per(int s) { return (ROWS * (N / R(s)) + 31) / 32; }
  __host__ __device__ static constexpr int elems(int s) { return per(s) * R(s); }
  __host__ __device__ static constexpr int max_elems() {
    int m = 0;
    for (int i = 0; i < NS; ++i) m = elems(i) > m ? elems(i) : m;
    return m;
  }
};

template <int N>
struct RegFFT {
  static constexpr int ROWS = rows_per_warp(N);
  static constexpr int E = Plan<N, false>::max_elems() > Plan<N, true>::max_elems()
                               ? Plan<N, false>::max_elems()
                               : Plan<N, true>::max_elems();
};

// Padded shared-memory index: one spare slot every PAD elements.  A first stage of
// radix R writes x[R b + q] and the next stage of a two-stage plan reads
// x[b + R q]; with PAD = R both map a half-warp onto distinct banks.
template <int PAD>
__device__ __forceinline__ int spad(int j) { return j + j / PAD; }
__host__ __device__ constexpr int spad_len(int n) { return n + n / 8; }   // largest padding used

// Exchange padding of a transform: its first radix for two-stage plans, 8 otherwise.
template <int N, bool REV>
__host__ __device__ constexpr int pad_of() {
  return plan2_radix(N, 0) > 0 ? (REV ? plan_radix(N, plan_len(N) - 1) : plan_radix(N, 0)) : 8;
}

// Twiddle tables.  A table for length N holds 3N float2 values:
//   [0, N)    exp(-2 pi i n / N);
//   [N, 2N)   for a two-stage plan (radices R0, R1; R0 R1 = N), the second stage's
//             factors exp(-2 pi i q k / N) at N + q R0 + k (q < R1, k < R0);
//   [2N, 3N)  the same for the reversed plan (radices R1, R0), at 2N + q R1 + k.
// The last two ranges are unused (zero) for plans of more than two stages.
__host__ __device__ constexpr int twiddle_table_offset(int n, bool rev) { return rev ? 2 * n : n; }
__host__ __device__ constexpr int twiddle_table_len(int n) { return 3 * n; }

// Twiddles exp(-+2 pi i q k s / N) for q = 1..R-1 of one butterfly: one or two table
// loads and products (at most six roundings) instead of R - 1 loads.
template <int N, int R, bool INV>
__device__ __forceinline__ void twiddles(float2* w, int ks, const float2* __restrict__ tw) {
  if constexpr (R <= 4) {
#pragma unroll
    for (int q = 1; q < R; ++q) {
      w[q] = __ldg(tw + q * ks);
      if (INV) w[q].y = -w[q].y;
    }
  } else {
    w[1] = __ldg(tw + ks);
    if (INV) w[1].y = -w[1].y;
    w[2] = cmul(w[1], w[1]);
    w[3] = cmul(w[2], w[1]);
    w[4] = cmul(w[2], w[2]);
    if constexpr (R > 4) {
#pragma unroll
      for (int q = 5; q < (R < 8 ? R : 8); ++q) w[q] = cmul(w[4], w[q - 4]);
    }
    if constexpr (R > 8) {
      float2 w8 = __ldg(tw + ((8 * ks) % N));
      if (INV) w8.y = -w8.y;
      float2 hi = w8;
#pragma unroll
      for (int a = 1; a < R / 8; ++a) {
        w[8 * a] = hi;
#pragma unroll
        for (int q = 1; q < 8; ++q) w[8 * a + q] = cmul(hi, w[q]);
        hi = cmul(hi, w8);
      }
    }
  }
}

// Butterfly slot u = lane + 32 t of a stage with NB butterflies per sequence
// belongs to sequence u / NB, butterfly u % NB.  Sequence r lives at
// sbuf + r * ld in the warp's shared buffer.
template <int N, bool INV, bool REV, int S, bool TAB>
__device__ __forceinline__ void reg_fft_stage(float2* v, float2* sbuf, int ld,
                                              const float2* __restrict__ tw, int lane,
                                              unsigned nz) {
  using PL = Plan<N, REV>;
  constexpr int ROWS = PL::ROWS;
  constexpr int PAD = pad_of<N, REV>();
  constexpr int R = PL::R(S), P = PL::P(S), NB = N / R, PER = PL::per(S);
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int u = lane + 32 * t;
    if ((ROWS * NB) % 32 == 0 || u < ROWS * NB) {
      const int b = u % NB;
      if constexpr (TAB && P > 1 && PL::NS == 2) {
        // second stage of a two-stage plan (P R = N): one table load per twiddle
        // exp(-2 pi i q k / N), stored at q P + k so that a warp reads a contiguous run
        const float2* __restrict__ tab = tw + twiddle_table_offset(N, REV) + b % P;
#pragma unroll
        for (int q = 1; q < R; ++q) {
          const float2 w = __ldg(tab + q * P);
          v[t * R + q] = INV ? cmulc(v[t * R + q], w) : cmul(v[t * R + q], w);
        }
      } else if constexpr (P > 1) {
        const int k = b % P;
        float2 w[R];
        twiddles<N, R, INV>(w, k * (N / (P * R)), tw);
#pragma unroll
        for (int q = 1; q < R; ++q) v[t * R + q] = cmul(v[t * R + q], w[q]);
      }
      dft<R, INV>(v + t * R, S == 0 ? nz : ~0u);
    }
  }
  if constexpr (S + 1 < PL::NS) {
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int u = lane + 32 * t;
      if ((ROWS * NB) % 32 == 0 || u < ROWS * NB) {
        const int b = u % NB;
        const int k = b % P;
        const int j0 = (b - k) * R + k;
        float2* row = sbuf + (u / NB) * ld;
#pragma unroll
        for (int q = 0; q < R; ++q) row[spad<PAD>(j0 + q * P)] = v[t * R + q];
      }
    }
    __syncwarp();
    constexpr int R2 = PL::R(S + 1), NB2 = N / R2, PER2 = PL::per(S + 1);
#pragma unroll
    for (int t = 0; t < PER2; ++t) {
      const int u = lane + 32 * t;
      if ((ROWS * NB2) % 32 == 0 || u < ROWS * NB2) {
        const int b = u % NB2;
        const float2* row = sbuf + (u / NB2) * ld;
#pragma unroll
        for (int q = 0; q < R2; ++q) v[t * R2 + q] = row[spad<PAD>(b + q * NB2)];
      }
    }
    __syncwarp();
    reg_fft_stage<N, INV, REV, S + 1, TAB>(v, sbuf, ld, tw, lane, ~0u);
  }
}

// Transform the ROWS warp-held sequences.  On entry slot u of v holds
// x_{u/NB0}[u%NB0 + q N/R0] (R0 = first radix), on exit X in the same form for the
// last radix.  `tw` is a table built by fill_twiddle_tables for this N.  `nz0` masks
// the first stage's inputs q that may be nonzero (band_mask for a band-limited input).
// TAB: a two-stage plan reads its second-stage twiddles from the table (one L1 load
// each) instead of forming them by products from two loads (about one complex product
// each); the first suits kernels bound by arithmetic issue, the second kernels bound by
// L1 / shared-memory wavefronts.
template <int N, bool INV, bool REV, bool TAB = true>
__device__ __forceinline__ void reg_fft(float2* v, float2* sbuf, int ld,
                                        const float2* __restrict__ tw, int lane,
                                        unsigned nz0 = ~0u) {
  reg_fft_stage<N, INV, REV, 0, TAB>(v, sbuf, ld, tw, lane, nz0);
}

// Table twiddles for a transform in a wavefront-bound kernel: only where a warp's reads
// of one factor index take a single wavefront (at most 16 distinct entries) or serve
// two sequences at once.
template <int N, bool REV>
__host__ __device__ constexpr bool table_twiddles_cheap() {
  using PL = Plan<N, REV>;
  return PL::NS == 2 && (PL::R(0) <= 16 || PL::per(1) > 1);
}

// ---------------------------------------------------------------------------
// Bounds-checked debug build (-DSTEM_CHECK).  STEM_REQUIRE(c) evaluates c there: a false c
// sets the check flag of this translation unit and the caller skips the access that c
// guards.  In the normal build it is the constant true and c is not evaluated.  Without
// relocatable device code every translation unit has its own flag; EELS_CHECK_COLLECTOR(fn)
// defines fn(status, stream), which moves the unit's flag into bit 4 of a status word.
#ifdef STEM_CHECK
namespace {
__device__ int g_check_flag;
}
__device__ __forceinline__ bool stem_require(bool ok) {
  if (!ok) atomicOr(&g_check_flag, 1);
  return ok;
}
#define STEM_REQUIRE(c) (::eels::stem_require(c))
#define EELS_CHECK_COLLECTOR(fn)                                                 \
  namespace {                                                                    \
  __global__ void fn##_kernel(int* status) {                                     \
    if (atomicExch(&g_check_flag, 0)) atomicOr(status, 4);                       \
  }                                                                              \
  }                                                                              \
  cudaError_t fn(int* status, cudaStream_t s) {                                  \
    fn##_kernel<<<1, 1, 0, s>>>(status);                                         \
    return cudaGetLastError();                                                   \
  }
#else
#define STEM_REQUIRE(c) true
#define EELS_CHECK_COLLECTOR(fn) \
  cudaError_t fn(int*, cudaStream_t) { return cudaSuccess; }
#endif

// A periodic window of w x w pixels with origin (x0, y0) on the nh x nh grid: the walks
// wrap once, so the origin must lie on the grid and the window must fit in it.
__device__ __forceinline__ bool window_ok(int x0, int y0, int w, int nh) {
  return x0 >= 0 && x0 < nh && y0 >= 0 && y0 < nh && w >= 1 && w <= nh;
}

}  // namespace eels
