// hfx_probe_fp64: the FP64 rates of this GPU that bound the HFX_FP64 mode.
//
// The FP64 build runs its contractions as DFMA on CUDA cores rather than on
// the FP64 tensor-core path (mma.sync m8n8k4 f64), because on this part the
// two reach about the same rate.  This probe measures both, so the choice can
// be re-checked on any GPU: every SM runs blocks of warps that issue long
// chains of independent multiply-adds, timed with CUDA events.
#include <cuda_runtime.h>

#include "hfx_internal.h"

namespace {

constexpr int kChains = 8;      // independent accumulators per thread
constexpr int kIters = 4096;    // loop trips per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

// kChains independent DFMA chains per thread; the result is stored so the
// work cannot be dropped.
__global__ void __launch_bounds__(kThreads) k_dfma(double x, double y, double *out) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = x + c;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], y, x);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Four independent m8n8k4 FP64 tensor-core products per warp and trip: each
// adds an 8x4 by 4x8 product (256 multiply-adds) into its 8x8 accumulator.
__global__ void __launch_bounds__(kThreads) k_dmma(double x, double y, double *out) {
  double d[4][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) d[c][0] = d[c][1] = 0.0;
  const double a = x + (threadIdx.x & 3), b = y - (threadIdx.x & 7);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
          : "+d"(d[c][0]), "+d"(d[c][1])
          : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += d[c][0] + d[c][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" hfx_status hfx_probe_fp64(double *dfma_tflops, double *dmma_tflops) {
  if (!dfma_tflops || !dmma_tflops) return HFX_E_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HFX_E_CUDA;
  const int blocks = nsm * kBlocksPerSm;
  double *out = nullptr;
  if (cudaMalloc((void **)&out, sizeof(double) * blocks * kThreads) != cudaSuccess)
    return HFX_E_NOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hfx_status st = HFX_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = HFX_E_CUDA;
  float ms[2] = {0.f, 0.f};
  for (int k = 0; k < 2 && st == HFX_OK; ++k) {
    for (int rep = 0; rep < 2 && st == HFX_OK; ++rep) {  // the first run warms up
      cudaEventRecord(e0);
      if (k == 0) k_dfma<<<blocks, kThreads>>>(1.0, 0.999999, out);
      else k_dmma<<<blocks, kThreads>>>(1.0, 0.999999, out);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        st = HFX_E_CUDA;
      else
        cudaEventElapsedTime(&ms[k], e0, e1);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (st != HFX_OK) return st;
  const double threads = (double)blocks * kThreads;
  // 2 flops per multiply-add; the m8n8k4 product is 256 multiply-adds per warp
  const double fma_flops = 2.0 * threads * kChains * kIters;
  const double mma_flops = 2.0 * (threads / 32.0) * 4.0 * kIters * 256.0;
  *dfma_tflops = fma_flops / (ms[0] * 1e-3) / 1e12;
  *dmma_tflops = mma_flops / (ms[1] * 1e-3) / 1e12;
  return HFX_OK;
}
