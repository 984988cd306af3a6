// Inelastic contraction on the tcgen05 tensor cores with FP32 accumulation in
// TMEM, Eq. SHn0 and the |.|^2 scan sum of Sec. III.
//
// Both complex products are run as real GEMMs with K-major operands whose K
// axis interleaves (re, im):
//   GEMM 1  C1[d][2j+c] = sum_k A1[d][k] B1[2j+c][k]
//           A1[d]    = Sout[d][window]            (complex, interleaved)
//           B1[2j]   = H . Sin[j][window]         -> C1[d][2j]   = Re M[d][j]
//           B1[2j+1] = -i H . Sin[j][window]      -> C1[d][2j+1] = Im M[d][j]
//   GEMM 2  C2[d][2r+c] = sum_k M[d][k] B2[2r+c][k]
//           B2[2r]   = conj(a_r),  B2[2r+1] = i conj(a_r)  -> C2 = (Re, Im) of V[d][r]
//           map[type][R_r] += sum_d C2[d][2r]^2 + C2[d][2r+1]^2     (fused epilogue)
//
// Two operand precisions, both a hi + lo split of every operand x into two planes,
// each product being lo*hi + hi*lo + hi*hi into the same FP32 accumulator (the lo*lo
// term is below the resolution the split keeps):
//   TF32    hi = tf32(x), lo = tf32(x - hi), kind::tf32 MMAs (about 21 significant bits);
//   BF16x3  hi = bf16(x), lo = bf16(x - hi), kind::f16 MMAs (about 16 significant bits).
// Operands are gathered into K-padded buffers [batch][plane][rows][K] and streamed
// by TMA (128-byte swizzle) through an mbarrier pipeline.  Every GEMM runs one persistent,
// warp-specialised kernel with a double-buffered TMEM accumulator (k_tc_gemm_ws).
#include <algorithm>

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "internal.h"

#include "tc_ptx.cuh"

namespace eels {

namespace {

constexpr int BM = 128;
// tile widths (columns of the output tile): the widest is the default, 128 suits problems
// whose column count leaves most of a 256-wide tile empty; the autotuner picks per GEMM
constexpr int BN_WIDE = 256, BN_NARROW = 128;

template <int PREC>
struct Prec;
template <>
struct Prec<EELS_TC_TF32> {
  using T = float;
  static constexpr int BK = 32;         // 128 bytes of K per row
  static constexpr int PLANES = 2;      // hi, lo
  static constexpr CUtensorMapDataType DT = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  __host__ __device__ static constexpr uint32_t idesc(int bn) { return tc::idesc_tf32(BM, bn); }
};
template <>
struct Prec<EELS_TC_BF16X3> {
  using T = __nv_bfloat16;
  static constexpr int BK = 64;
  static constexpr int PLANES = 2;      // hi, lo
  static constexpr CUtensorMapDataType DT = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  __host__ __device__ static constexpr uint32_t idesc(int bn) { return tc::idesc_bf16(BM, bn); }
};

template <int PREC, int BN>
struct Tile {
  using P = Prec<PREC>;
  static constexpr int A_BYTES = BM * P::BK * (int)sizeof(typename P::T);   // one plane
  static constexpr int B_BYTES = BN * P::BK * (int)sizeof(typename P::T);
  static constexpr int STAGE_BYTES = P::PLANES * (A_BYTES + B_BYTES);
};

// plane pl of the TF32 hi + lo split of x (0: hi = x rounded; 1: lo = x - hi rounded)
__device__ __forceinline__ float tf32_part(float x, int pl) {
  const float h = tc::to_tf32(x);
  return pl == 0 ? h : tc::to_tf32(x - h);
}

// store the pair (a, b) at element e of a row, in every plane of the precision
template <int PREC>
__device__ __forceinline__ void put2(void* base, int64_t plane_stride, int64_t e, float a, float b) {
  if constexpr (PREC == EELS_TC_TF32) {
    float* p = static_cast<float*>(base);
    const float ah = tc::to_tf32(a), bh = tc::to_tf32(b);
    reinterpret_cast<float2*>(p + e)[0] = make_float2(ah, bh);
    reinterpret_cast<float2*>(p + plane_stride + e)[0] =
        make_float2(tc::to_tf32(a - ah), tc::to_tf32(b - bh));
  } else {
    __nv_bfloat16* p = static_cast<__nv_bfloat16*>(base);
    const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
    const __nv_bfloat16 al = __float2bfloat16_rn(a - __bfloat162float(ah));
    const __nv_bfloat16 bl = __float2bfloat16_rn(b - __bfloat162float(bh));
    reinterpret_cast<__nv_bfloat162*>(p + e)[0] = __halves2bfloat162(ah, bh);
    reinterpret_cast<__nv_bfloat162*>(p + plane_stride + e)[0] = __halves2bfloat162(al, bl);
  }
}

// plane pl of the BF16 hi + lo split of x (0: hi = x rounded; 1: lo = x - hi rounded)
__device__ __forceinline__ __nv_bfloat16 bf16_part(float x, int pl) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  return pl == 0 ? h : __float2bfloat16_rn(x - __bfloat162float(h));
}
// two BF16 values as one 32-bit word, lo first in memory
__device__ __forceinline__ uint32_t bf16_pair(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// store 16 consecutive values of a row (element e, a multiple of 16) in every plane
template <int PREC>
__device__ __forceinline__ void put16(void* base, int64_t plane_stride, int64_t e, const float* v) {
  if constexpr (PREC == EELS_TC_TF32) {
    float* p = static_cast<float*>(base);
    float4* dh = reinterpret_cast<float4*>(p + e);
    float4* dl = reinterpret_cast<float4*>(p + plane_stride + e);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 h = make_float4(tc::to_tf32(v[4 * q]), tc::to_tf32(v[4 * q + 1]),
                                   tc::to_tf32(v[4 * q + 2]), tc::to_tf32(v[4 * q + 3]));
      dh[q] = h;
      dl[q] = make_float4(tc::to_tf32(v[4 * q] - h.x), tc::to_tf32(v[4 * q + 1] - h.y),
                          tc::to_tf32(v[4 * q + 2] - h.z), tc::to_tf32(v[4 * q + 3] - h.w));
    }
  } else {
    __align__(16) __nv_bfloat16 hi[16], lo[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      hi[q] = __float2bfloat16_rn(v[q]);
      lo[q] = __float2bfloat16_rn(v[q] - __bfloat162float(hi[q]));
    }
    __nv_bfloat16* p = static_cast<__nv_bfloat16*>(base);
    uint4* dh = reinterpret_cast<uint4*>(p + e);
    uint4* dl = reinterpret_cast<uint4*>(p + plane_stride + e);
    dh[0] = reinterpret_cast<uint4*>(hi)[0];
    dh[1] = reinterpret_cast<uint4*>(hi)[1];
    dl[0] = reinterpret_cast<uint4*>(lo)[0];
    dl[1] = reinterpret_cast<uint4*>(lo)[1];
  }
}

struct EpiStore {
  void* out;
  int64_t z_stride;      // elements between problems
  int64_t plane_stride;  // elements between hi and lo planes
  int64_t row_pitch;
  int rows;
  int cols;
};

// |.|^2 epilogue (GEMM 2, GEMM-V): map[type][R] += sum over rows of C[row][2R]^2 +
// C[row][2R+1]^2.
struct EpiAbs2 {
  const int* z_site;
  const int* z_type;
  const int* xoff;
  const int* xcnt;
  const int* xlist;
  const int* yoff;
  const int* ylist;
  int n_sx, n_sy;
  double* map;
  int rows;
  int n_types;           // map planes (checked in the bounds-checked build)
};

// GEMM-Y epilogue: C[r][2p + c] = Y[r][p] of one site; for every channel t write
// BV[site*T + t][2r] = H_t[p] Y[r][p] and BV[site*T + t][2r + 1] = -i H_t[p] Y[r][p]
// (interleaved over p), the B operand of the per-channel GEMM-V.
struct EpiSpread {
  void* bv;
  int64_t z_stride;      // elements between transitions
  int64_t plane_stride;
  int64_t row_pitch;     // k1p
  int rows;              // nr_cap
  int P;                 // window pixels w*w
  int n_types;
  const float2* H;       // [S][T][w][w], or [T][w][w] shared by all sites (h_mul = 0)
  int h_mul;
  const int* slot_site;
};

// ---------------------------------------------------------------------------
// Persistent, warp-specialised kernel of the three GEMMs (both precisions).  Tile
// BM x BN = 128 x 256 or 128 x 128, K blocks of 128 bytes per row.  One CTA per SM walks
// the tiles blockIdx.x, blockIdx.x + gridDim.x, ...; warp 0 issues the TMA loads, warp 1
// the MMAs, warps 2-9 run the epilogue (two per TMEM lane quarter, each pair splitting
// the BN columns).  The accumulator is double-buffered in TMEM (2 x BN columns), so
// the MMAs of the next tile overlap the epilogue of this one.  Every wait is bounded; a
// failed wait stops every role (the four epilogue warps of a column half decide together
// after their named barrier), and before returning the CTA waits, again bounded, for its
// MMAs and its loads in flight, then frees its TMEM.
// ---------------------------------------------------------------------------
namespace ws {
constexpr int EPI_WARPS = 8;                    // two per TMEM lane quarter, one per column half
constexpr int THREADS = 64 + 32 * EPI_WARPS;
// GEMM-Y stages one plane of a chunk of columns at a time: 256 rows x 64 bytes (16 TF32
// or 32 BF16 values), 64-byte swizzled, 16 KB per column half.
constexpr int STG_ROW = 64;
constexpr int TILE_STG = 2 * BM * STG_ROW;
// Stages hold both planes of a 128-byte K block of A and B: 96 KB for 256-wide tiles (two
// stages), 64 KB for 128-wide tiles (three), also beside the GEMM-Y staging (2 x 16 KB).
template <int MODE, int PREC, int BN>
__host__ __device__ constexpr int stages() {
  return BN == BN_WIDE ? 2 : 3;
}
template <int MODE, int PREC, int BN>
__host__ __device__ constexpr size_t staging_half() {
  return MODE != 2 ? 0 : (size_t)TILE_STG;
}
template <int MODE, int PREC, int BN>
__host__ __device__ constexpr size_t smem() {
  return (size_t)stages<MODE, PREC, BN>() * Tile<PREC, BN>::STAGE_BYTES +
         2 * staging_half<MODE, PREC, BN>() + 1024 + 256;
}
template <int PREC, int BN>
constexpr bool fits() {
  return smem<2, PREC, BN>() + (BN / 2) * 4 + 16 <= 232448 &&
         smem<1, PREC, BN>() + 4 * (BN / 2) * 4 + 16 <= 232448 &&
         smem<0, PREC, BN>() + 16 <= 232448;
}
static_assert(fits<EELS_TC_BF16X3, BN_WIDE>() && fits<EELS_TC_TF32, BN_WIDE>() &&
                  fits<EELS_TC_BF16X3, BN_NARROW>() && fits<EELS_TC_TF32, BN_NARROW>(),
              "GEMM stages, staging and partial sums exceed the shared memory of a CTA");
}  // namespace ws

// named barrier of the four epilogue warps of one column half (ids 1 and 2)
__device__ __forceinline__ void epi_sync(int half) {
  asm volatile("bar.sync %0, 128;" ::"r"(1 + half) : "memory");
}

template <int MODE, int PREC, int BN>
__global__ void __launch_bounds__(ws::THREADS, 1)
k_tc_gemm_ws(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
             const __grid_constant__ CUtensorMap tv, int kblocks, int gx, int gy, int gz, const int* __restrict__ tile_prefix,
             const int* __restrict__ a_batch, const int* __restrict__ b_batch,
             const int* __restrict__ n_valid, const int* __restrict__ m_valid, EpiStore es,
             EpiAbs2 ea, EpiSpread ey, int* __restrict__ status, long long wait_cycles,
             int withhold) {
  using P = Prec<PREC>;
  using TL = Tile<PREC, BN>;
  constexpr int S = ws::stages<MODE, PREC, BN>(), BK = P::BK, PL = P::PLANES;
  constexpr uint32_t IDESC = P::idesc(BN);
  extern __shared__ uint8_t smem_raw[];
  // |.|^2 partial sums of the column pairs, one row per TMEM lane quarter; summed in a
  // fixed order so that a map does not depend on warp scheduling
  __shared__ float red[MODE == 1 ? 4 : 1][BN / 2];   // only the |.|^2 epilogue uses it
  __shared__ int abort_flag;
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* stg = sm + S * TL::STAGE_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(stg + 2 * ws::staging_half<MODE, PREC, BN>());
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(full + s, 1);
      tc::mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(acc_full + b, 1);
      tc::mbar_init(acc_empty + b, ws::EPI_WARPS);   // one arrival per epilogue warp
    }
    tc::mbar_init(drain, 1);
    abort_flag = 0;
    tc::fence_barrier_init();
    tc::tma_prefetch(&ta);
    tc::tma_prefetch(&tb);
  }
  if (warp == 1) tc::tmem_alloc(tmem_holder, 2 * BN);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  bool ok = true;

  // Work list.  With tile_prefix, problem z owns the tiles tile_prefix[z] - tile_prefix[0]
  // .. tile_prefix[z + 1] - tile_prefix[0] (exclusive), a rectangle of nx column tiles
  // (column tile fastest) by its row tiles; only tiles with work are listed, so the
  // round-robin below gives every CTA the same amount of work.  Without it every tile
  // of the gx x gy x gz grid is listed.
  const int base = tile_prefix ? tile_prefix[0] : 0;
  const int tiles = tile_prefix ? tile_prefix[gz] - base : gx * gy * gz;
  auto decode = [&](int t, int& z, int& n0, int& m0) {
    if (!tile_prefix) {
      z = t / (gx * gy);
      m0 = ((t / gx) % gy) * BM;
      n0 = (t % gx) * BN;
    } else {
      int lo = 0, hi = gz - 1;            // last z with tile_prefix[z] - base <= t
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile_prefix[mid] - base <= t) lo = mid; else hi = mid - 1;
      }
      z = lo;
      const int local = t - (tile_prefix[z] - base);
      const int count = tile_prefix[z + 1] - tile_prefix[z];
      // a problem's tiles form a rectangle of whole rows of the tile grid
      if (!STEM_REQUIRE(count > 0 && count % (MODE == 2 ? gx : gy) == 0 && count <= gx * gy &&
                        local >= 0 && local < count))
        return false;
      const int nx = MODE == 2 ? gx : count / gy;
      n0 = (local % nx) * BN;
      m0 = (local / nx) * BM;
    }
    return !(n0 >= n_valid[z] || (m_valid && m0 >= m_valid[z]));
  };

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      // withhold (failure-detection test): issue no load at all, so that the consumers'
      // bounded waits run out while nothing is in flight
      for (int t = blockIdx.x; t < tiles && ok && !withhold; t += gridDim.x) {
        int z, n0, m0;
        if (!decode(t, z, n0, m0)) continue;
        const int ab = a_batch[z], bb = b_batch[z];
        (void)STEM_REQUIRE(ab >= 0 && bb >= 0);   // TMA box coordinates of the problem
        for (int kb = 0; kb < kblocks; ++kb, ++it) {
          const int s = it % S;
          if (it >= S && !(ok = tc::mbar_wait(empty + s, ((it / S) - 1) & 1, wait_cycles))) break;
          uint8_t* st = sm + s * TL::STAGE_BYTES;
          tc::mbar_arrive_expect_tx(full + s, TL::STAGE_BYTES);
#pragma unroll
          for (int pl = 0; pl < PL; ++pl) {
            tc::tma_load_4d(st + pl * TL::A_BYTES, &ta, full + s, kb * BK, m0, pl, ab);
            tc::tma_load_4d(st + PL * TL::A_BYTES + pl * TL::B_BYTES, &tb, full + s, kb * BK, n0,
                            pl, bb);
          }
        }
      }
      // the last load of every stage has landed before the CTA may leave
      for (int j = max(0, it - S); j < it; ++j) ok &= tc::mbar_wait(full + j % S, (j / S) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0, i = 0;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        int z, n0, m0;
        if (!decode(t, z, n0, m0)) continue;
        const int b = i & 1;
        if (i >= 2 && !(ok = tc::mbar_wait(acc_empty + b, ((i >> 1) - 1) & 1, wait_cycles))) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(b * BN);
        for (int kb = 0; kb < kblocks; ++kb, ++it) {
          const int s = it % S;
          if (!(ok = tc::mbar_wait(full + s, (it / S) & 1, wait_cycles))) break;
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(sm + s * TL::STAGE_BYTES);
          const uint32_t sb = sa + PL * TL::A_BYTES;
          // each MMA consumes 32 bytes of K: 8 TF32 or 16 BF16 elements; the small
          // products first (lo*hi, hi*lo), then hi*hi
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t acc = (kb | kk) != 0 ? 1u : 0u;
            const uint32_t ah = sa + kk * 32, al = sa + TL::A_BYTES + kk * 32;
            const uint32_t bh = sb + kk * 32, bl = sb + TL::B_BYTES + kk * 32;
            if constexpr (PREC == EELS_TC_TF32) {
              tc::mma_tf32(d, tc::desc_sw128(al), tc::desc_sw128(bh), IDESC, acc);
              tc::mma_tf32(d, tc::desc_sw128(ah), tc::desc_sw128(bl), IDESC, 1u);
              tc::mma_tf32(d, tc::desc_sw128(ah), tc::desc_sw128(bh), IDESC, 1u);
            } else {
              tc::mma_f16(d, tc::desc_sw128(al), tc::desc_sw128(bh), IDESC, acc);
              tc::mma_f16(d, tc::desc_sw128(ah), tc::desc_sw128(bl), IDESC, 1u);
              tc::mma_f16(d, tc::desc_sw128(ah), tc::desc_sw128(bh), IDESC, 1u);
            }
          }
          tc::mma_commit(empty + s);
        }
        if (!ok) break;
        tc::mma_commit(acc_full + b);
        ++i;
      }
      // every MMA issued has completed before the TMEM is freed
      tc::mma_commit(drain);
      ok &= tc::mbar_wait(drain, 0);
    }
  } else {
    const int q4 = warp & 3;                  // TMEM lane quarter this warp may read
    const int half = (warp - 2) >> 2;         // column half of the tile
    const int te = threadIdx.x - 64 - 128 * half;   // 0 .. 127 within the half
    const int c_lo = half * (BN / 2), c_hi = c_lo + BN / 2;
    uint8_t* stg_h = stg + (size_t)half * ws::staging_half<MODE, PREC, BN>();
    int i = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      int z, n0, m0;
      if (!decode(t, z, n0, m0)) continue;
      const int b = i & 1;
      if (!tc::mbar_wait(acc_full + b, (i >> 1) & 1, wait_cycles)) atomicOr(&abort_flag, 1);
      epi_sync(half);
      if (abort_flag) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t trow = tmem + (uint32_t)(b * BN) + ((uint32_t)(q4 * 32) << 16);
      const int row = m0 + q4 * 32 + lane;
      if constexpr (MODE == 0) {
        const int64_t rbase = (int64_t)z * es.z_stride + (int64_t)row * es.row_pitch;
        for (int c = c_lo; c < c_hi; c += 16) {
          float v[16];
          tc::tmem_ld16(trow + c, v);
          const int col = n0 + c;
          if (row < es.rows && col < es.cols)
            put16<PREC>(es.out, es.plane_stride, rbase + col, v);
        }
      } else if constexpr (MODE == 2) {
        // chunks of CC columns (CC / 2 pixels; 64 bytes of one plane per operand row): each
        // thread forms its two rows (H_t Y and -i H_t Y) and writes them, hi plane then lo
        // plane, into the half's staging tile (64-byte rows, 64-byte swizzle); one thread of
        // the half stores each plane with one TMA box, and the tile is rewritten only after
        // that store has read it
        constexpr int CC = ws::STG_ROW / (int)sizeof(typename P::T);   // 16 TF32, 32 BF16
        constexpr int PX = CC / 2;
        const int site = ey.slot_site[z];
        if (!STEM_REQUIRE(site >= 0)) {   // skip the tile, keeping the TMEM handshake below
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(acc_empty + b);
          ++i;
          continue;
        }
        const int rr = 2 * (q4 * 32 + lane);
        for (int c = c_lo; c < c_hi && n0 + c < es.cols; c += CC) {
          for (int t0 = 0; t0 < ey.n_types; ++t0) {
            float v[CC];
            tc::tmem_ld16(trow + c, v);
            if constexpr (CC == 32) tc::tmem_ld16(trow + c + 16, v + 16);
            const float2* Ht = ey.H + ((int64_t)site * ey.h_mul * ey.n_types + t0) * ey.P;
            float2 y[PX];
#pragma unroll
            for (int k = 0; k < PX; ++k) {
              const int pp = (n0 + c) / 2 + k;
              const float2 h = pp < ey.P ? __ldg(Ht + pp) : make_float2(0.f, 0.f);
              y[k] = cmul(h, make_float2(v[2 * k], v[2 * k + 1]));
            }
            for (int pl = 0; pl < 2; ++pl) {
              if (te == 0) tc::bulk_wait_read();
              epi_sync(half);
              uint8_t* r0 = stg_h + (size_t)rr * ws::STG_ROW;
              uint8_t* r1 = r0 + ws::STG_ROW;
#pragma unroll
              for (int q = 0; q < 4; ++q) {   // 16-byte chunk q of the 64-byte row
                uint4 a, b;
                if constexpr (PREC == EELS_TC_TF32) {   // pixels 2q, 2q + 1
                  const float2 u0 = y[2 * q], u1 = y[2 * q + 1];
                  a = make_uint4(__float_as_uint(tf32_part(u0.x, pl)),
                                 __float_as_uint(tf32_part(u0.y, pl)),
                                 __float_as_uint(tf32_part(u1.x, pl)),
                                 __float_as_uint(tf32_part(u1.y, pl)));
                  b = make_uint4(__float_as_uint(tf32_part(u0.y, pl)),
                                 __float_as_uint(tf32_part(-u0.x, pl)),
                                 __float_as_uint(tf32_part(u1.y, pl)),
                                 __float_as_uint(tf32_part(-u1.x, pl)));
                } else {                                 // pixels 4q .. 4q + 3
                  uint32_t wa[4], wb[4];
#pragma unroll
                  for (int e = 0; e < 4; ++e) {
                    const float2 u = y[4 * q + e];
                    wa[e] = bf16_pair(bf16_part(u.x, pl), bf16_part(u.y, pl));
                    wb[e] = bf16_pair(bf16_part(u.y, pl), bf16_part(-u.x, pl));
                  }
                  a = make_uint4(wa[0], wa[1], wa[2], wa[3]);
                  b = make_uint4(wb[0], wb[1], wb[2], wb[3]);
                }
                // chunk q of 64-byte row r sits at chunk q ^ ((r >> 1) & 3) (64-byte swizzle)
                *reinterpret_cast<uint4*>(r0 + ((q ^ ((rr >> 1) & 3)) << 4)) = a;
                *reinterpret_cast<uint4*>(r1 + ((q ^ (((rr + 1) >> 1) & 3)) << 4)) = b;
              }
              tc::fence_async_shared();
              epi_sync(half);
              // a store box starts at non-negative coordinates, x on a 16-byte boundary
              if (te == 0 && STEM_REQUIRE(n0 + c >= 0 && ((n0 + c) * (int)sizeof(typename P::T)) % 16 == 0 &&
                                          m0 >= 0 && z * ey.n_types + t0 >= 0)) {
                tc::tma_store_4d(&tv, stg_h, n0 + c, 2 * m0, pl, z * ey.n_types + t0);
                tc::bulk_commit();
              }
            }
          }
        }
      } else {
        // this half owns red[*][c_lo / 2 .. c_hi / 2); every entry is written once below
        const bool live = row < ea.rows;
        for (int c = c_lo; c < c_hi; c += 16) {
          float v[16];
          tc::tmem_ld16(trow + c, v);
          float p[8];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            p[q] = live ? fmaf(v[2 * q], v[2 * q], v[2 * q + 1] * v[2 * q + 1]) : 0.f;
          const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
          float r4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float send = b4 ? p[q] : p[q + 4];
            r4[q] = (b4 ? p[q + 4] : p[q]) + __shfl_xor_sync(0xffffffffu, send, 16);
          }
          float r2[2];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const float send = b3 ? r4[q] : r4[q + 2];
            r2[q] = (b3 ? r4[q + 2] : r4[q]) + __shfl_xor_sync(0xffffffffu, send, 8);
          }
          float r1 = (b2 ? r2[1] : r2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? r2[0] : r2[1], 4);
          r1 += __shfl_xor_sync(0xffffffffu, r1, 2);
          r1 += __shfl_xor_sync(0xffffffffu, r1, 1);
          if ((lane & 3) == 0) red[q4][c / 2 + (b4 ? 4 : 0) + (b3 ? 2 : 0) + (b2 ? 1 : 0)] = r1;
        }
        epi_sync(half);
        const int s = ea.z_site[z];
        const int nx = ea.xcnt[s];
        const int nv = n_valid[z];
        for (int k = c_lo / 2 + te; k < c_hi / 2; k += 128) {
          const int r = n0 / 2 + k;
          if (2 * r < nv && STEM_REQUIRE(s >= 0 && nx > 0)) {
            const int ix = ea.xlist[ea.xoff[s] + r % nx];
            const int iy = ea.ylist[ea.yoff[s] + r / nx];
            const int ty = ea.z_type[z];
            if (!STEM_REQUIRE(ix >= 0 && ix < ea.n_sx && iy >= 0 && iy < ea.n_sy && ty >= 0 &&
                              ty < ea.n_types))
              continue;
            const int64_t idx = ((int64_t)ty * ea.n_sy + iy) * ea.n_sx + ix;
            atomicAdd(ea.map + idx, (double)(((red[0][k] + red[1][k]) + red[2][k]) + red[3][k]));
          }
        }
        epi_sync(half);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(acc_empty + b);
      ++i;
    }
    if constexpr (MODE == 2) {
      if (te == 0) tc::bulk_wait();   // the CTA's TMA stores are complete before it leaves
    }
  }
  __syncwarp();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, 2 * BN);
  if (!ok && status) atomicExch(status, 1);
}

// Window gathers: consecutive threads take consecutive window pixels (coalesced).  A
// thread's pixels p0, p0 + blockDim.x, ... are visited by an incremental walk (the window
// row and column advance by fixed steps, no division), and each batch of kGatherBatch
// loads is issued before any of its stores so that the loads overlap.
constexpr int kGatherBatch = 4;

struct WindowWalk {
  int x0, y0, w, nh, dx, dy, xx, yy;
  __device__ WindowWalk(int x0_, int y0_, int w_, int nh_)
      : x0(x0_), y0(y0_), w(w_), nh(nh_), dx(blockDim.x % w_), dy(blockDim.x / w_),
        xx(threadIdx.x % w_), yy(threadIdx.x / w_) {}
  // off[u] = plane offset of pixel p0 + u blockDim.x of the periodic window, -1 past P
  __device__ __forceinline__ void offsets(int p0, int P, int* off) {
#pragma unroll
    for (int u = 0; u < kGatherBatch; ++u) {
      off[u] = -1;
      if (p0 + u * (int)blockDim.x < P) {
        int gy = y0 + yy, gx = x0 + xx;
        if (gy >= nh) gy -= nh;
        if (gx >= nh) gx -= nh;
        off[u] = gy * nh + gx;
        xx += dx;
        yy += dy;
        if (xx >= w) {
          xx -= w;
          ++yy;
        }
      }
    }
  }
  // v[u] = plane[pixel p0 + u blockDim.x of the window], zero past P
  __device__ __forceinline__ void load(const float2* __restrict__ plane, int p0, int P,
                                       float2* v) {
    int off[kGatherBatch];
    offsets(p0, P, off);
#pragma unroll
    for (int u = 0; u < kGatherBatch; ++u)
      v[u] = off[u] >= 0 ? plane[off[u]] : make_float2(0.f, 0.f);
  }
};

// Beams of S_out per block of the S_out gather, and probe rows per block of the
// probe-row gather: enough loads per thread to cover the memory latency.
constexpr int kSoutBeams = 4;
constexpr int kArowRows = 16;

// A1[slot][plane][d][2p + c] = Sout[d][pixel p of the window of site slot_site[slot]];
// a block takes kSoutBeams beams d of one site.
template <int PREC>
__global__ void k_gather_sout(const float2* __restrict__ Sout, int nh, int n_out, int w,
                              const int* __restrict__ slot_site, const int* __restrict__ wx,
                              const int* __restrict__ wy, void* __restrict__ A1, int k1p) {
  constexpr int PL = Prec<PREC>::PLANES;
  const int d0 = blockIdx.x * kSoutBeams, slot = blockIdx.y;
  const int s = slot_site[slot];
  if (!STEM_REQUIRE(s >= 0 && window_ok(wx[s], wy[s], w, nh))) return;   // whole block
  const int64_t plane = (int64_t)nh * nh;
  const int64_t pstride = (int64_t)n_out * k1p;
  const int64_t rbase = (int64_t)slot * PL * pstride + (int64_t)d0 * k1p;
  const float2* src = Sout + (int64_t)d0 * plane;
  const int nb = min(kSoutBeams, n_out - d0);
  const int P = w * w;
  WindowWalk walk(wx[s], wy[s], w, nh);
  for (int p0 = threadIdx.x; p0 < P; p0 += kGatherBatch * blockDim.x) {
    int off[kGatherBatch];
    walk.offsets(p0, P, off);
    float2 v[kSoutBeams][kGatherBatch];
#pragma unroll
    for (int b = 0; b < kSoutBeams; ++b)
#pragma unroll
      for (int u = 0; u < kGatherBatch; ++u)
        v[b][u] = (b < nb && off[u] >= 0) ? src[b * plane + off[u]] : make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < kSoutBeams; ++b)
#pragma unroll
      for (int u = 0; u < kGatherBatch; ++u)
        if (b < nb && off[u] >= 0)
          put2<PREC>(A1, pstride, rbase + (int64_t)b * k1p + 2 * (p0 + u * (int)blockDim.x),
                     v[b][u].x, v[b][u].y);
  }
  for (int b = 0; b < nb; ++b)
    for (int p = P + threadIdx.x; p < k1p / 2; p += blockDim.x)   // K padding
      put2<PREC>(A1, pstride, rbase + (int64_t)b * k1p + 2 * p, 0.f, 0.f);
}

// B1[z][plane][2j][2p + c] = H_z[p] Sin[j][p],  B1[z][plane][2j+1] = -i H_z[p] Sin[j][p]
template <int PREC>
__global__ void k_gather_sin_h(const float2* __restrict__ Sin, int nh, int n_in, int w,
                               const int* __restrict__ z_site, const int* __restrict__ z_type,
                               const float2* __restrict__ H, int n_types, int h_mul,
                               const int* __restrict__ wx, const int* __restrict__ wy,
                               void* __restrict__ B1, int k1p) {
  constexpr int PL = Prec<PREC>::PLANES;
  const int j = blockIdx.x, z = blockIdx.y;
  const int s = z_site[z];
  if (!STEM_REQUIRE(s >= 0 && z_type[z] >= 0 && z_type[z] < n_types &&
                    window_ok(wx[s], wy[s], w, nh)))
    return;   // the whole block
  const int64_t plane = (int64_t)nh * nh;
  const int64_t pstride = (int64_t)2 * n_in * k1p;
  const int64_t r0 = (int64_t)z * PL * pstride + (int64_t)(2 * j) * k1p;
  const int64_t r1 = r0 + k1p;
  const float2* Hz = H + ((int64_t)s * h_mul * n_types + z_type[z]) * w * w;
  const float2* src = Sin + (int64_t)j * plane;
  const int P = w * w;
  WindowWalk walk(wx[s], wy[s], w, nh);
  for (int p0 = threadIdx.x; p0 < P; p0 += kGatherBatch * blockDim.x) {
    float2 v[kGatherBatch];
    walk.load(src, p0, P, v);
#pragma unroll
    for (int u = 0; u < kGatherBatch; ++u) {
      const int p = p0 + u * blockDim.x;
      if (p < P) {
        const float2 h = cmul(Hz[p], v[u]);
        put2<PREC>(B1, pstride, r0 + 2 * p, h.x, h.y);
        put2<PREC>(B1, pstride, r1 + 2 * p, h.y, -h.x);
      }
    }
  }
  for (int p = P + threadIdx.x; p < k1p / 2; p += blockDim.x) {   // K padding
    put2<PREC>(B1, pstride, r0 + 2 * p, 0.f, 0.f);
    put2<PREC>(B1, pstride, r1 + 2 * p, 0.f, 0.f);
  }
}

// B2[slot][plane][2r] = conj(a_r), B2[slot][plane][2r+1] = i conj(a_r),
// a_r[j] = ax[j][ix(r)] ay[j][iy(r)]
template <int PREC>
__global__ void k_gather_probe(const float2* __restrict__ axT, const float2* __restrict__ ayT,
                               int n_in, int n_sx, int n_sy, const int* __restrict__ slot_site,
                               const int* __restrict__ xoff, const int* __restrict__ xcnt,
                               const int* __restrict__ xlist, const int* __restrict__ yoff,
                               const int* __restrict__ ycnt, const int* __restrict__ ylist,
                               int nr_cap, void* __restrict__ B2, int k2p) {
  constexpr int PL = Prec<PREC>::PLANES;
  const int r = blockIdx.x, slot = blockIdx.y;
  const int s = slot_site[slot];
  const int nx = xcnt[s], nr = nx * ycnt[s];
  // rows of N tiles GEMM 2 skips (the widest tile: a narrower one reads no more rows)
  if (2 * r >= (2 * nr + BN_WIDE - 1) / BN_WIDE * BN_WIDE) return;
  const int64_t pstride = (int64_t)2 * nr_cap * k2p;
  const int64_t r0 = (int64_t)slot * PL * pstride + (int64_t)(2 * r) * k2p;
  const int64_t r1 = r0 + k2p;
  int ix = 0, iy = 0;
  if (r < nr) {
    ix = xlist[xoff[s] + r % nx];
    iy = ylist[yoff[s] + r / nx];
    if (!STEM_REQUIRE(ix >= 0 && ix < n_sx && iy >= 0 && iy < n_sy)) ix = iy = 0;
  }
  const float2* axr = axT + (int64_t)ix * n_in;
  const float2* ayr = ayT + (int64_t)iy * n_in;
  for (int j = threadIdx.x; j < k2p / 2; j += blockDim.x) {
    float2 a = make_float2(0.f, 0.f);
    if (r < nr && j < n_in) a = cmul(axr[j], ayr[j]);
    put2<PREC>(B2, pstride, r0 + 2 * j, a.x, -a.y);
    put2<PREC>(B2, pstride, r1 + 2 * j, a.y, a.x);
  }
}

// AY[slot][plane][r][2j + c] = a_r[j] (interleaved), a_r[j] = axT[ix(r)][j] ayT[iy(r)][j];
// a block takes kArowRows rows r of one site (their phase-table rows are looked up once,
// by the first kArowRows threads) and writes them four at a time.
template <int PREC>
__global__ void k_gather_arows(const float2* __restrict__ axT, const float2* __restrict__ ayT,
                               int n_in, int n_sx, int n_sy, const int* __restrict__ slot_site,
                               const int* __restrict__ xoff, const int* __restrict__ xcnt,
                               const int* __restrict__ xlist, const int* __restrict__ yoff,
                               const int* __restrict__ ycnt, const int* __restrict__ ylist,
                               int nr_cap, void* __restrict__ AY, int k2p) {
  constexpr int PL = Prec<PREC>::PLANES;
  __shared__ int s_ix[kArowRows], s_iy[kArowRows];
  const int rb = blockIdx.x * kArowRows, slot = blockIdx.y;
  const int s = slot_site[slot];
  const int nx = xcnt[s], nr = nx * ycnt[s];
  const int r_end = min((nr + BM - 1) / BM * BM, nr_cap);   // rows of M tiles GEMM-Y reads
  if (rb >= r_end) return;                                   // the same for the whole block
  if (threadIdx.x < kArowRows) {
    const int r = rb + threadIdx.x;
    s_ix[threadIdx.x] = r < nr ? xlist[xoff[s] + r % nx] : -1;   // -1: a zero row
    s_iy[threadIdx.x] = r < nr ? ylist[yoff[s] + r / nx] : -1;
    if (r < nr && !STEM_REQUIRE(s_ix[threadIdx.x] >= 0 && s_ix[threadIdx.x] < n_sx &&
                                s_iy[threadIdx.x] >= 0 && s_iy[threadIdx.x] < n_sy))
      s_ix[threadIdx.x] = s_iy[threadIdx.x] = -1;
  }
  __syncthreads();
  const int rows = min(kArowRows, r_end - rb);
  const int64_t pstride = (int64_t)nr_cap * k2p;
  const int64_t base = (int64_t)slot * PL * pstride + (int64_t)rb * k2p;
  for (int i0 = 0; i0 < rows; i0 += 4) {
    for (int j = threadIdx.x; j < k2p / 2; j += blockDim.x) {
      float2 a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u;
        const int ix = i < rows ? s_ix[i] : -1, iy = i < rows ? s_iy[i] : -1;
        a[u] = (ix >= 0 && j < n_in)
                   ? cmul(axT[(int64_t)ix * n_in + j], ayT[(int64_t)iy * n_in + j])
                   : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u < rows)
          put2<PREC>(AY, pstride, base + (int64_t)(i0 + u) * k2p + 2 * j, a[u].x, a[u].y);
    }
  }
}

// BY[slot][plane][2p][2j + c] = conj(Sin[j][p]), BY[slot][plane][2p + 1] = i conj(Sin[j][p])
// over the window pixels p; a 32 x 32 (p, j) tile is transposed through shared memory.
template <int PREC>
__global__ void k_gather_sin_t(const float2* __restrict__ Sin, int nh, int n_in, int w,
                               const int* __restrict__ slot_site, const int* __restrict__ wx,
                               const int* __restrict__ wy, void* __restrict__ BY, int k1p,
                               int k2p) {
  constexpr int PL = Prec<PREC>::PLANES;
  __shared__ float2 tile[32][33];
  const int p0 = blockIdx.x * 32, j0 = blockIdx.y * 32, slot = blockIdx.z;
  const int s = slot_site[slot];
  if (!STEM_REQUIRE(s >= 0 && window_ok(wx[s], wy[s], w, nh))) return;   // before any barrier
  const int P = w * w;
  const int64_t plane = (int64_t)nh * nh;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  int64_t pix = -1;                                         // window pixel of column tx
  if (p0 + tx < P) {
    const int p = p0 + tx;
    const int gy = (wy[s] + p / w) % nh, gx = (wx[s] + p % w) % nh;
    pix = (int64_t)gy * nh + gx;
  }
  // the four loads of a thread in flight together
  float2 got[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = j0 + ty + 8 * u;
    got[u] = (j < n_in && pix >= 0) ? Sin[(int64_t)j * plane + pix] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) tile[ty + 8 * u][tx] = got[u];
  __syncthreads();
  const int64_t pstride = (int64_t)k1p * k2p;
  for (int pp = ty; pp < 32; pp += 8) {
    const int p = p0 + pp, j = j0 + tx;
    if (2 * p >= k1p || 2 * j >= k2p) continue;
    const float2 v = tile[tx][pp];
    const int64_t r0 = (int64_t)slot * PL * pstride + (int64_t)(2 * p) * k2p;
    put2<PREC>(BY, pstride, r0 + 2 * j, v.x, -v.y);
    put2<PREC>(BY, pstride, r0 + k2p + 2 * j, v.y, v.x);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 4D tensor map (k, rows, plane, batch) over a K-major buffer; box (BK, box_rows, 1, 1),
// 128-byte swizzle; out-of-range rows read as zero.
template <int PREC>
cudaError_t make_map(CUtensorMap* map, void* base, int k, int rows, int batch, int box_rows,
                     int box_k = 0, CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_128B) {
  using P = Prec<PREC>;
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t es = sizeof(typename P::T);
  cuuint64_t dims[4] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)P::PLANES, (cuuint64_t)batch};
  cuuint64_t strides[3] = {(cuuint64_t)k * es, (cuuint64_t)k * es * rows,
                           (cuuint64_t)k * es * rows * P::PLANES};
  cuuint32_t box[4] = {(cuuint32_t)(box_k > 0 ? box_k : P::BK), (cuuint32_t)box_rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(map, P::DT, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int PREC>
cudaError_t gather_impl(const TcBatch& b, cudaStream_t st) {
  const int nz = b.n_sites * b.n_types;
  cudaError_t e;
  k_gather_sout<PREC><<<dim3((b.n_out + kSoutBeams - 1) / kSoutBeams, b.n_sites), 256, 0, st>>>(
      b.Sout, b.nh, b.n_out, b.w, b.slot_site, b.wx, b.wy, b.A1, b.k1p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_gather_sin_h<PREC><<<dim3(b.n_in, nz), 256, 0, st>>>(b.Sin, b.nh, b.n_in, b.w, b.z_site,
                                                          b.z_type, b.H, b.n_types, b.h_mul, b.wx,
                                                          b.wy, b.B1, b.k1p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_gather_probe<PREC><<<dim3(b.nr_cap, b.n_sites), 256, 0, st>>>(
      b.axT, b.ayT, b.n_in, b.n_sx, b.n_sy, b.slot_site, b.xoff, b.xcnt, b.xlist, b.yoff, b.ycnt, b.ylist,
      b.nr_cap, b.B2, b.k2p);
  return cudaGetLastError();
}

int sm_count() {
  static std::atomic<int> count[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  int c = count[dev].load(std::memory_order_relaxed);
  if (c == 0) {
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0)
      c = 148;
    count[dev].store(c, std::memory_order_relaxed);
  }
  return c;
}

// Launch of one GEMM over a (gx, gy, gz) tile grid (or its listed tiles): the persistent
// warp-specialised kernel, one CTA per SM at most.
template <int MODE, int PREC, int BN>
cudaError_t launch_gemm(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tv,
                        int kblocks, int gx, int gy,
                        int gz, const int* tile_prefix, const int* a_batch, const int* b_batch,
                        const int* n_valid, const int* m_valid, const EpiStore& es,
                        const EpiAbs2& ea, const EpiSpread& ey, int* status, cudaStream_t st,
                        int valid_tiles, long long wait_cycles, int withhold) {
  if (gx <= 0 || gy <= 0 || gz <= 0) return cudaSuccess;
  static std::atomic<uint64_t> attr{0};
  cudaError_t e =
      smem_attr_once(k_tc_gemm_ws<MODE, PREC, BN>, ws::smem<MODE, PREC, BN>(), attr);
  if (e != cudaSuccess) return e;
  const int tiles = tile_prefix ? valid_tiles : gx * gy * gz;
  if (tiles <= 0) return cudaSuccess;
  const int grid = std::min(tiles, sm_count());
  if (wait_cycles <= 0) wait_cycles = tc::kWaitCycles;   // 0: the default limit
  k_tc_gemm_ws<MODE, PREC, BN><<<grid, ws::THREADS, ws::smem<MODE, PREC, BN>(), st>>>(
      ta, tb, tv, kblocks, gx, gy, gz, tile_prefix, a_batch, b_batch, n_valid, m_valid, es, ea, ey,
      status, wait_cycles, withhold);
  return cudaGetLastError();
}

template <int PREC, int BN>
cudaError_t gemm1_impl(const TcBatch& b, cudaStream_t st) {
  cudaError_t e;
  CUtensorMap mA1, mB1;
  if ((e = make_map<PREC>(&mA1, b.A1, b.k1p, b.n_out, b.slots_cap, BM)) != cudaSuccess) return e;
  if ((e = make_map<PREC>(&mB1, b.B1, b.k1p, 2 * b.n_in, b.slots_cap * b.n_types, BN)) !=
      cudaSuccess)
    return e;
  const int64_t pstride = (int64_t)b.n_out * b.k2p;
  EpiStore es{b.M1, Prec<PREC>::PLANES * pstride, pstride, b.k2p, b.n_out, b.k2p};
  EpiAbs2 ea{};
  EpiSpread ey{};
  return launch_gemm<0, PREC, BN>(mA1, mB1, mB1, b.k1p / Prec<PREC>::BK, (b.k2p + BN - 1) / BN,
                              (b.n_out + BM - 1) / BM, b.n_sites * b.n_types, nullptr, b.a_batch1,
                              b.b_batch1, b.n_valid1, nullptr, es, ea, ey, b.status, st, 0, b.wait_cycles, b.withhold);
}

template <int PREC, int BN>
cudaError_t gemm2_impl(const TcBatch& b, cudaStream_t st) {
  cudaError_t e;
  CUtensorMap mM1, mB2;
  if ((e = make_map<PREC>(&mM1, b.M1, b.k2p, b.n_out, b.slots_cap * b.n_types, BM)) !=
      cudaSuccess)
    return e;
  if ((e = make_map<PREC>(&mB2, b.B2, b.k2p, 2 * b.nr_cap, b.slots_cap, BN)) != cudaSuccess)
    return e;
  EpiStore es{};
  EpiAbs2 ea{b.z_site, b.z_type, b.xoff, b.xcnt, b.xlist, b.yoff, b.ylist, b.n_sx, b.n_sy,
             b.map, b.n_out, b.n_types};
  EpiSpread ey{};
  return launch_gemm<1, PREC, BN>(mM1, mB2, mB2, b.k2p / Prec<PREC>::BK, (2 * b.nr_cap + BN - 1) / BN,
                              (b.n_out + BM - 1) / BM, b.n_sites * b.n_types, b.tiles_v,
                              b.a_batch2, b.b_batch2, b.n_valid2, nullptr, es, ea, ey, b.status,
                              st, b.n_tiles_v, b.wait_cycles, b.withhold);
}

// Association with the probe sum first: gathers for GEMM-Y (A1 is shared with GEMM-V).
template <int PREC>
cudaError_t gather_y_impl(const TcBatch& b, cudaStream_t st) {
  cudaError_t e;
  k_gather_sout<PREC><<<dim3((b.n_out + kSoutBeams - 1) / kSoutBeams, b.n_sites), 256, 0, st>>>(
      b.Sout, b.nh, b.n_out, b.w, b.slot_site, b.wx, b.wy, b.A1, b.k1p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_gather_arows<PREC><<<dim3((b.nr_cap + kArowRows - 1) / kArowRows, b.n_sites), 256, 0, st>>>(
      b.axT, b.ayT, b.n_in, b.n_sx, b.n_sy, b.slot_site, b.xoff, b.xcnt, b.xlist, b.yoff, b.ycnt, b.ylist,
      b.nr_cap, b.AY, b.k2p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  dim3 gt((b.k1p / 2 + 31) / 32, (b.k2p / 2 + 31) / 32, b.n_sites);
  k_gather_sin_t<PREC><<<gt, 256, 0, st>>>(b.Sin, b.nh, b.n_in, b.w, b.slot_site, b.wx, b.wy,
                                            b.BY, b.k1p, b.k2p);
  return cudaGetLastError();
}

template <int PREC, int BN>
cudaError_t gemm_y_impl(const TcBatch& b, cudaStream_t st) {
  cudaError_t e;
  CUtensorMap mAY, mBY;
  if ((e = make_map<PREC>(&mAY, b.AY, b.k2p, b.nr_cap, b.slots_cap, BM)) != cudaSuccess) return e;
  if ((e = make_map<PREC>(&mBY, b.BY, b.k2p, b.k1p, b.slots_cap, BN)) != cudaSuccess) return e;
  const int64_t pstride = (int64_t)2 * b.nr_cap * b.k1p;
  EpiStore es{nullptr, 0, 0, 0, 0, b.k1p};
  EpiAbs2 ea{};
  EpiSpread ey{b.BV, Prec<PREC>::PLANES * pstride, pstride, b.k1p, b.nr_cap, b.w * b.w,
               b.n_types, b.H, b.h_mul, b.slot_site};
  // store map of GEMM-Y's output: BV rows (2 per probe) in boxes of 64 bytes x 256 rows
  // of one plane (16 TF32 or 32 BF16 columns), 64-byte swizzle
  CUtensorMap mBV;
  if ((e = make_map<PREC>(&mBV, b.BV, b.k1p, 2 * b.nr_cap, b.slots_cap * b.n_types, 2 * BM,
                          ws::STG_ROW / (int)sizeof(typename Prec<PREC>::T),
                          CU_TENSOR_MAP_SWIZZLE_64B)) != cudaSuccess)
    return e;
  return launch_gemm<2, PREC, BN>(mAY, mBY, mBV, b.k2p / Prec<PREC>::BK, (b.k1p + BN - 1) / BN,
                              (b.nr_cap + BM - 1) / BM, b.n_sites, b.tiles_y, b.a_batch_y,
                              b.a_batch_y, b.n_valid_y, b.m_valid_y, es, ea, ey, b.status, st,
                              b.n_tiles_y, b.wait_cycles, b.withhold);
}

template <int PREC, int BN>
cudaError_t gemm_v_impl(const TcBatch& b, cudaStream_t st) {
  cudaError_t e;
  CUtensorMap mA1, mBV;
  if ((e = make_map<PREC>(&mA1, b.A1, b.k1p, b.n_out, b.slots_cap, BM)) != cudaSuccess) return e;
  if ((e = make_map<PREC>(&mBV, b.BV, b.k1p, 2 * b.nr_cap, b.slots_cap * b.n_types, BN)) !=
      cudaSuccess)
    return e;
  EpiStore es{};
  EpiAbs2 ea{b.z_site, b.z_type, b.xoff, b.xcnt, b.xlist, b.yoff, b.ylist, b.n_sx, b.n_sy,
             b.map, b.n_out, b.n_types};
  EpiSpread ey{};
  return launch_gemm<1, PREC, BN>(mA1, mBV, mBV, b.k1p / Prec<PREC>::BK, (2 * b.nr_cap + BN - 1) / BN,
                              (b.n_out + BM - 1) / BM, b.n_sites * b.n_types, b.tiles_v,
                              b.a_batch1, b.b_batch1, b.n_valid2, nullptr, es, ea, ey, b.status,
                              st, b.n_tiles_v, b.wait_cycles, b.withhold);
}

}  // namespace

cudaError_t tc_gather_y(const TcBatch& b, cudaStream_t st) {
  if (b.n_sites <= 0) return cudaSuccess;
  return b.prec == EELS_TC_BF16X3 ? gather_y_impl<EELS_TC_BF16X3>(b, st)
                                  : gather_y_impl<EELS_TC_TF32>(b, st);
}

cudaError_t tc_gemm_y(const TcBatch& b, cudaStream_t st) {
  if (b.n_sites <= 0) return cudaSuccess;
  const bool narrow = b.bn_first == BN_NARROW;
  if (b.prec == EELS_TC_BF16X3)
    return narrow ? gemm_y_impl<EELS_TC_BF16X3, BN_NARROW>(b, st) : gemm_y_impl<EELS_TC_BF16X3, BN_WIDE>(b, st);
  return narrow ? gemm_y_impl<EELS_TC_TF32, BN_NARROW>(b, st) : gemm_y_impl<EELS_TC_TF32, BN_WIDE>(b, st);
}

cudaError_t tc_gemm_v(const TcBatch& b, cudaStream_t st) {
  if (b.n_sites <= 0) return cudaSuccess;
  const bool narrow = b.bn_second == BN_NARROW;
  if (b.prec == EELS_TC_BF16X3)
    return narrow ? gemm_v_impl<EELS_TC_BF16X3, BN_NARROW>(b, st) : gemm_v_impl<EELS_TC_BF16X3, BN_WIDE>(b, st);
  return narrow ? gemm_v_impl<EELS_TC_TF32, BN_NARROW>(b, st) : gemm_v_impl<EELS_TC_TF32, BN_WIDE>(b, st);
}

int tc_value_bytes(int prec) {
  return prec == EELS_TC_BF16X3
             ? Prec<EELS_TC_BF16X3>::PLANES * (int)sizeof(Prec<EELS_TC_BF16X3>::T)
             : Prec<EELS_TC_TF32>::PLANES * (int)sizeof(Prec<EELS_TC_TF32>::T);
}

int tc_tile_width(int narrow) { return narrow ? BN_NARROW : BN_WIDE; }

int tc_k_align(int prec) {
  return prec == EELS_TC_BF16X3 ? Prec<EELS_TC_BF16X3>::BK : Prec<EELS_TC_TF32>::BK;
}

cudaError_t tc_gather(const TcBatch& b, cudaStream_t st) {
  if (b.n_sites <= 0) return cudaSuccess;
  return b.prec == EELS_TC_BF16X3 ? gather_impl<EELS_TC_BF16X3>(b, st)
                                  : gather_impl<EELS_TC_TF32>(b, st);
}

cudaError_t tc_gemm1(const TcBatch& b, cudaStream_t st) {
  if (b.n_sites <= 0) return cudaSuccess;
  const bool narrow = b.bn_first == BN_NARROW;
  if (b.prec == EELS_TC_BF16X3)
    return narrow ? gemm1_impl<EELS_TC_BF16X3, BN_NARROW>(b, st) : gemm1_impl<EELS_TC_BF16X3, BN_WIDE>(b, st);
  return narrow ? gemm1_impl<EELS_TC_TF32, BN_NARROW>(b, st) : gemm1_impl<EELS_TC_TF32, BN_WIDE>(b, st);
}

cudaError_t tc_gemm2(const TcBatch& b, cudaStream_t st) {
  if (b.n_sites <= 0) return cudaSuccess;
  const bool narrow = b.bn_second == BN_NARROW;
  if (b.prec == EELS_TC_BF16X3)
    return narrow ? gemm2_impl<EELS_TC_BF16X3, BN_NARROW>(b, st) : gemm2_impl<EELS_TC_BF16X3, BN_WIDE>(b, st);
  return narrow ? gemm2_impl<EELS_TC_TF32, BN_NARROW>(b, st) : gemm2_impl<EELS_TC_TF32, BN_WIDE>(b, st);
}

EELS_CHECK_COLLECTOR(collect_checks_tc)

}  // namespace eels
