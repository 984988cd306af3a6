// Inelastic contraction on the tcgen05 tensor cores (TF32 operands, FP32
// accumulation in TMEM), Eq. SHn0 and the |.|^2 scan sum of Sec. III.
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
// Operands are gathered into K-padded buffers (rounded to TF32 nearest) and
// streamed by TMA (128-byte swizzle) through a 4-stage mbarrier pipeline.  One
// 128 x 256 tile per CTA: warp 0 lane 0 issues TMA, warp 1 lane 0 issues MMA,
// all four warps drain TMEM in the epilogue.
#include <cudaTypedefs.h>

#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace eels {

namespace {

constexpr int BM = 128, BN = 256, BK = 32, STAGES = 4;
constexpr int A_BYTES = BM * BK * 4;
constexpr int B_BYTES = BN * BK * 4;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t IDESC = tc::idesc_tf32(BM, BN);
constexpr size_t GEMM_SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256;

struct EpiStore {
  float* out;
  int64_t z_stride;
  int64_t row_pitch;
  int rows;
  int cols;
};

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
};

template <int MODE>
__global__ void __launch_bounds__(128, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
          int kblocks, const int* __restrict__ a_batch, const int* __restrict__ b_batch,
          const int* __restrict__ n_valid, EpiStore es, EpiAbs2 ea, int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ float red[BN / 2];
  const int z = blockIdx.z;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int nv = n_valid[z];
  if (n0 >= nv) return;
  const uint32_t raw = tc::smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(full + s, 1);
      tc::mbar_init(empty + s, 1);
    }
    tc::mbar_init(done, 1);
    tc::fence_barrier_init();
    tc::tma_prefetch(&ta);
    tc::tma_prefetch(&tb);
  }
  if (warp == 0) tc::tmem_alloc(tmem_holder, BN);
  if (MODE == 1)
    for (int i = threadIdx.x; i < BN / 2; i += blockDim.x) red[i] = 0.f;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  bool ok = true;

  if (warp == 0 && lane == 0) {
    const int ab = a_batch[z], bb = b_batch[z];
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES) ok &= tc::mbar_wait(empty + s, ((kb / STAGES) - 1) & 1);
      uint8_t* sa = sm + s * STAGE_BYTES;
      tc::mbar_arrive_expect_tx(full + s, STAGE_BYTES);
      tc::tma_load_3d(sa, &ta, full + s, kb * BK, m0, ab);
      tc::tma_load_3d(sa + A_BYTES, &tb, full + s, kb * BK, n0, bb);
    }
  } else if (warp == 1 && lane == 0) {
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb % STAGES;
      ok &= tc::mbar_wait(full + s, (kb / STAGES) & 1);
      tc::fence_after_sync();
      const uint32_t sa = tc::smem_u32(sm + s * STAGE_BYTES);
      const uint32_t sb = sa + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk)
        tc::mma_tf32(tmem, tc::desc_sw128(sa + kk * 32), tc::desc_sw128(sb + kk * 32), IDESC,
                     (kb | kk) != 0 ? 1u : 0u);
      tc::mma_commit(empty + s);
    }
    tc::mma_commit(done);
  }
  __syncwarp();
  ok &= tc::mbar_wait(done, 0);
  tc::fence_after_sync();

  const int row = m0 + warp * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  if constexpr (MODE == 0) {
    float* dst = es.out + (int64_t)z * es.z_stride + (int64_t)row * es.row_pitch;
    for (int c = 0; c < BN; c += 16) {
      float v[16];
      tc::tmem_ld16(trow + c, v);
      const int col = n0 + c;
      if (row < es.rows && col < es.cols) {
        float4* d4 = reinterpret_cast<float4*>(dst + col);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          d4[q] = make_float4(tc::to_tf32(v[4 * q]), tc::to_tf32(v[4 * q + 1]),
                              tc::to_tf32(v[4 * q + 2]), tc::to_tf32(v[4 * q + 3]));
      }
    }
  } else {
    const bool live = row < ea.rows;
    for (int c = 0; c < BN; c += 16) {
      float v[16];
      tc::tmem_ld16(trow + c, v);
      float p[8];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        p[q] = live ? fmaf(v[2 * q], v[2 * q], v[2 * q + 1] * v[2 * q + 1]) : 0.f;
      // reduce-scatter over the 32 rows of the warp: halve the value set at each of the
      // lane bits 4, 3, 2, then sum over bits 1, 0.  Lane L ends with the warp total of
      // value ((L >> 4) & 1) * 4 + ((L >> 3) & 1) * 2 + ((L >> 2) & 1).
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
      if ((lane & 3) == 0) atomicAdd(&red[c / 2 + (b4 ? 4 : 0) + (b3 ? 2 : 0) + (b2 ? 1 : 0)], r1);
    }
    __syncthreads();
    const int s = ea.z_site[z];
    const int nx = ea.xcnt[s];
    for (int i = threadIdx.x; i < BN / 2; i += blockDim.x) {
      const int r = n0 / 2 + i;
      if (2 * r < nv) {
        const int ix = ea.xlist[ea.xoff[s] + r % nx];
        const int iy = ea.ylist[ea.yoff[s] + r / nx];
        const int64_t idx = ((int64_t)ea.z_type[z] * ea.n_sy + iy) * ea.n_sx + ix;
        atomicAdd(ea.map + idx, (double)red[i]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, BN);
  if (!ok && status) atomicExch(status, 1);
}

// A1[slot][d][2p + c] = tf32(Sout[d][pixel p of the window of site slot_site[slot]])
__global__ void k_gather_sout(const float2* __restrict__ Sout, int nh, int n_out, int w,
                              const int* __restrict__ slot_site, const int* __restrict__ wx,
                              const int* __restrict__ wy, float* __restrict__ A1, int k1p) {
  const int d = blockIdx.x, slot = blockIdx.y;
  const int s = slot_site[slot];
  const int64_t plane = (int64_t)nh * nh;
  float2* row = reinterpret_cast<float2*>(A1 + ((int64_t)slot * n_out + d) * k1p);
  const float2* src = Sout + (int64_t)d * plane;
  const int P = w * w;
  for (int p = threadIdx.x; p < k1p / 2; p += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (p < P) {
      const int gy = (wy[s] + p / w) % nh, gx = (wx[s] + p % w) % nh;
      v = src[(int64_t)gy * nh + gx];
    }
    row[p] = make_float2(tc::to_tf32(v.x), tc::to_tf32(v.y));
  }
}

// B1[z][2j][2p + c] = tf32(H_z[p] Sin[j][p]),  B1[z][2j+1] = tf32(-i H_z[p] Sin[j][p])
__global__ void k_gather_sin_h(const float2* __restrict__ Sin, int nh, int n_in, int w,
                               const int* __restrict__ z_site, const int* __restrict__ z_type,
                               const float2* __restrict__ H, int n_types,
                               const int* __restrict__ wx, const int* __restrict__ wy,
                               float* __restrict__ B1, int k1p) {
  const int j = blockIdx.x, z = blockIdx.y;
  const int s = z_site[z];
  const int64_t plane = (int64_t)nh * nh;
  const float2* Hz = H + ((int64_t)s * n_types + z_type[z]) * w * w;
  float2* r0 = reinterpret_cast<float2*>(B1 + ((int64_t)z * 2 * n_in + 2 * j) * k1p);
  float2* r1 = r0 + k1p / 2;
  const float2* src = Sin + (int64_t)j * plane;
  const int P = w * w;
  for (int p = threadIdx.x; p < k1p / 2; p += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (p < P) {
      const int gy = (wy[s] + p / w) % nh, gx = (wx[s] + p % w) % nh;
      v = cmul(Hz[p], src[(int64_t)gy * nh + gx]);
    }
    r0[p] = make_float2(tc::to_tf32(v.x), tc::to_tf32(v.y));
    r1[p] = make_float2(tc::to_tf32(v.y), tc::to_tf32(-v.x));
  }
}

// B2[slot][2r] = conj(a_r), B2[slot][2r+1] = i conj(a_r), a_r[j] = ax[j][ix(r)] ay[j][iy(r)]
__global__ void k_gather_probe(const float2* __restrict__ ax, const float2* __restrict__ ay,
                               int n_in, int n_sx, int n_sy, const int* __restrict__ slot_site,
                               const int* __restrict__ xoff, const int* __restrict__ xcnt,
                               const int* __restrict__ xlist, const int* __restrict__ yoff,
                               const int* __restrict__ ycnt, const int* __restrict__ ylist,
                               int nr_cap, float* __restrict__ B2, int k2p) {
  const int r = blockIdx.x, slot = blockIdx.y;
  const int s = slot_site[slot];
  const int nx = xcnt[s], nr = nx * ycnt[s];
  float2* r0 = reinterpret_cast<float2*>(B2 + ((int64_t)slot * 2 * nr_cap + 2 * r) * k2p);
  float2* r1 = r0 + k2p / 2;
  int ix = 0, iy = 0;
  if (r < nr) {
    ix = xlist[xoff[s] + r % nx];
    iy = ylist[yoff[s] + r / nx];
  }
  for (int j = threadIdx.x; j < k2p / 2; j += blockDim.x) {
    float2 a = make_float2(0.f, 0.f);
    if (r < nr && j < n_in) a = cmul(ax[(int64_t)j * n_sx + ix], ay[(int64_t)j * n_sy + iy]);
    r0[j] = make_float2(tc::to_tf32(a.x), tc::to_tf32(-a.y));
    r1[j] = make_float2(tc::to_tf32(a.y), tc::to_tf32(a.x));
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

// 3D FP32 tensor map (k, rows, batch), K-major rows of k elements, box (32, box_rows, 1),
// 128-byte swizzle; out-of-range rows read as zero.
cudaError_t make_map(CUtensorMap* map, float* base, int k, int rows, int batch, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)k * 4, (cuuint64_t)k * 4 * (cuuint64_t)rows};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t tc_gather(const TcBatch& b, cudaStream_t st) {
  if (b.n_sites <= 0) return cudaSuccess;
  const int nz = b.n_sites * b.n_types;
  cudaError_t e;
  k_gather_sout<<<dim3(b.n_out, b.n_sites), 256, 0, st>>>(b.Sout, b.nh, b.n_out, b.w, b.slot_site,
                                                           b.wx, b.wy, b.A1, b.k1p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_gather_sin_h<<<dim3(b.n_in, nz), 256, 0, st>>>(b.Sin, b.nh, b.n_in, b.w, b.z_site, b.z_type,
                                                    b.H, b.n_types, b.wx, b.wy, b.B1, b.k1p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_gather_probe<<<dim3(b.nr_cap, b.n_sites), 256, 0, st>>>(
      b.ax, b.ay, b.n_in, b.n_sx, b.n_sy, b.slot_site, b.xoff, b.xcnt, b.xlist, b.yoff, b.ycnt,
      b.ylist, b.nr_cap, b.B2, b.k2p);
  return cudaGetLastError();
}

namespace {
cudaError_t set_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)GEMM_SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tc_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)GEMM_SMEM);
  if (e == cudaSuccess) done = true;
  return e;
}
}  // namespace

cudaError_t tc_gemm1(const TcBatch& b, cudaStream_t st) {
  if (b.n_sites <= 0) return cudaSuccess;
  cudaError_t e;
  if ((e = set_attrs()) != cudaSuccess) return e;
  CUtensorMap mA1, mB1;
  if ((e = make_map(&mA1, b.A1, b.k1p, b.n_out, b.slots_cap, BM)) != cudaSuccess) return e;
  if ((e = make_map(&mB1, b.B1, b.k1p, 2 * b.n_in, b.slots_cap * b.n_types, BN)) != cudaSuccess)
    return e;
  EpiStore es{b.M1, (int64_t)b.n_out * b.k2p, b.k2p, b.n_out, b.k2p};
  EpiAbs2 ea{};
  dim3 g1((b.k2p + BN - 1) / BN, (b.n_out + BM - 1) / BM, b.n_sites * b.n_types);
  k_tc_gemm<0><<<g1, 128, GEMM_SMEM, st>>>(mA1, mB1, b.k1p / BK, b.a_batch1, b.b_batch1,
                                            b.n_valid1, es, ea, b.status);
  return cudaGetLastError();
}

cudaError_t tc_gemm2(const TcBatch& b, cudaStream_t st) {
  if (b.n_sites <= 0) return cudaSuccess;
  cudaError_t e;
  if ((e = set_attrs()) != cudaSuccess) return e;
  CUtensorMap mM1, mB2;
  if ((e = make_map(&mM1, b.M1, b.k2p, b.n_out, b.slots_cap * b.n_types, BM)) != cudaSuccess)
    return e;
  if ((e = make_map(&mB2, b.B2, b.k2p, 2 * b.nr_cap, b.slots_cap, BN)) != cudaSuccess) return e;
  EpiStore es{};
  EpiAbs2 ea{b.z_site, b.z_type, b.xoff, b.xcnt, b.xlist, b.yoff, b.ylist, b.n_sx, b.n_sy,
             b.map, b.n_out};
  dim3 g2((2 * b.nr_cap + BN - 1) / BN, (b.n_out + BM - 1) / BM, b.n_sites * b.n_types);
  k_tc_gemm<1><<<g2, 128, GEMM_SMEM, st>>>(mM1, mB2, b.k2p / BK, b.a_batch2, b.b_batch2,
                                            b.n_valid2, es, ea, b.status);
  return cudaGetLastError();
}

}  // namespace eels
