// eels_fp32_fma_rate: measured FP32 FMA throughput of the CUDA cores, the denominator of
// the ALU roofline of the FP32 contraction and of the multislice passes.  Independent
// FMA chains per thread keep every FP32 pipe issuing; the result is read back only so
// that the compiler keeps the chains.
#include <cuda_runtime.h>

#include "stem_eels.h"

namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(256) k_fma_chains(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == 1234.5f) out[blockIdx.x] = s;   // practically never taken
}

}  // namespace

extern "C" eels_status eels_fp32_fma_rate(int device, int iters, double* flops_per_s) {
  if (!flops_per_s || iters <= 0) return EELS_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return EELS_ERR_CUDA;
  (void)cudaGetLastError();
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return EELS_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  eels_status st = EELS_ERR_CUDA;
  if (cudaMalloc((void**)&out, sizeof(float) * blocks) == cudaSuccess &&
      cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    k_fma_chains<<<blocks, threads>>>(out, iters / 8 + 1, 0.999f, 1e-4f);   // warm-up
    cudaEventRecord(e0);
    k_fma_chains<<<blocks, threads>>>(out, iters, 0.999f, 1e-4f);
    cudaEventRecord(e1);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess &&
        cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
      const double flops = 2.0 * kChains * (double)iters * blocks * threads;
      *flops_per_s = flops / (1e-3 * ms);
      st = EELS_OK;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  return st;
}
