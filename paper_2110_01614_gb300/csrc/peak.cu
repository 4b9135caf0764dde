// Measured FP32 FMA throughput of the current GPU: the denominator of the
// FP32 form's roofline fraction.  Every thread of a grid that fills every SM
// runs 16 independent FMA chains (enough to cover the FMA pipe's latency),
// timed with CUDA events on the caller's stream.

#include "nsdf_debug.h"
#include "nsdf_internal.h"

namespace nsdf {
namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_peak_kernel(float *out, int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 1234.5f) out[blockIdx.x] = s;      // keeps the chains live; never true in practice
}

}  // namespace
}  // namespace nsdf

using namespace nsdf;

extern "C" nsdf_status nsdf_debug_fp32_fma_peak(double *tflops, nsdf_stream stream) {
  if (!tflops) return NSDF_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel, kThreads, 0) !=
          cudaSuccess)
    return NSDF_ERR_CUDA;
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  const int iters = 8192;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return NSDF_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return NSDF_ERR_CUDA;
  }
  float best = 3.0e38f;
  nsdf_status st = NSDF_OK;
  for (int rep = 0; rep < 4 && st == NSDF_OK; ++rep) {      // the first is a warm-up
    cudaEventRecord(e0, s);
    fma_peak_kernel<<<grid, kThreads, 0, s>>>(nullptr, iters, 0.9999999f, 1e-7f);
    cudaEventRecord(e1, s);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      st = NSDF_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NSDF_OK) return st;
  const double flop = 2.0 * kChains * (double)iters * (double)grid * kThreads;
  *tflops = flop / (best * 1e-3) / 1e12;
  return NSDF_OK;
}
