// Launchers of the FP32 fused query kernel.  The kernel is in
// query_fp32_kernel.cuh; this file instantiates it for networks without
// Fourier features, query_fp32_ff.cu for networks with them (Sec. 4.3).

#include "query_fp32_kernel.cuh"

namespace nsdf {

// query_fp32_ff.cu
int fp32_ff_per_sm(int width, int pt);
cudaError_t fp32_ff_launch(const QueryParams &p, int pt, int grid, cudaStream_t s);

bool query_fp32_supported(int width) {
  return width == 32 || width == 64 || width == 128 || width == 256 || width == 512;
}

int fp32_tile_points(int width, int pt) {
#define CASE(W) \
  if (width == W) return pt == 4 ? Cfg<W, 4>::P : Cfg<W, 8>::P;
  NSDF_FP32_WIDTHS(CASE)
#undef CASE
  return 0;
}

int fp32_ctas_per_sm(int width, int pt, bool ff) {
  if (ff) return fp32_ff_per_sm(width, pt);
#define CASE(W) \
  if (width == W) return pt == 4 ? per_sm_t<W, 4, false>() : per_sm_t<W, 8, false>();
  NSDF_FP32_WIDTHS(CASE)
#undef CASE
  return 1;
}

// The single-network launch uses 8 points per thread.
int query_fp32_grid(int width, int64_t n, int num_sms, bool ff) {
  const int P = fp32_tile_points(width, 8);
  if (P == 0) return 0;
  const int64_t tiles = (n + P - 1) / P;
  const int64_t cap = (int64_t)num_sms * fp32_ctas_per_sm(width, 8, ff);
  return (int)(tiles < cap ? (tiles < 1 ? 1 : tiles) : cap);
}

size_t query_fp32_scratch_bytes(int width, int n_hidden, int grid) {
  return fp32_scratch_bytes_pt(width, 8, n_hidden, grid);
}

size_t fp32_scratch_bytes_pt(int width, int pt, int n_hidden, int grid) {
  const int slabs = n_hidden > 1 ? n_hidden - 1 : 1;
  return sizeof(float) * (size_t)grid * slabs * fp32_tile_points(width, pt) * width;
}

cudaError_t launch_query_fp32_grouped(const QueryParams &p, int pt, int grid, cudaStream_t s) {
  if (p.ff > 0) return fp32_ff_launch(p, pt, grid, s);
#define CASE(W)                                                                           \
  if (p.width == W)                                                                       \
    return pt == 4 ? launch_t<W, 4, false>(p, grid, s) : launch_t<W, 8, false>(p, grid, s);
  NSDF_FP32_WIDTHS(CASE)
#undef CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_query_fp32(const QueryParams &p, int num_sms, cudaStream_t s) {
  const int grid = query_fp32_grid(p.width, p.n, num_sms, p.ff > 0);
  if (grid == 0) return cudaErrorInvalidValue;
  return launch_query_fp32_grouped(p, 8, grid, s);
}

}  // namespace nsdf
