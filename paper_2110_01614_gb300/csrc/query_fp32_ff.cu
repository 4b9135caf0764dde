// Instantiations of the FP32 fused query kernel for networks with the
// Fourier-feature input layer of Sec. 4.3, in a translation unit of their own
// (compiled in parallel with query_fp32.cu).

#include "query_fp32_kernel.cuh"

namespace nsdf {

int fp32_ff_per_sm(int width, int pt) {
#define CASE(W) \
  if (width == W) return pt == 4 ? per_sm_t<W, 4, true>() : per_sm_t<W, 8, true>();
  NSDF_FP32_WIDTHS(CASE)
#undef CASE
  return 1;
}

cudaError_t fp32_ff_launch(const QueryParams &p, int pt, int grid, cudaStream_t s) {
#define CASE(W)                                                                         \
  if (p.width == W)                                                                     \
    return pt == 4 ? launch_t<W, 4, true>(p, grid, s) : launch_t<W, 8, true>(p, grid, s);
  NSDF_FP32_WIDTHS(CASE)
#undef CASE
  return cudaErrorInvalidValue;
}

}  // namespace nsdf
