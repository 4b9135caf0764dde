// Many bodies in one launch (batching form): every network of a context
// answers its own range of points, all in one persistent grouped launch.
//
// The work list is built on the device from the counts, so a CUDA graph that
// captured nsdf_query_grouped replays correctly after the counts change:
// tile_start[k] = sum_{j<k} ceil(counts[j] / P), and tile t belongs to the
// network k with tile_start[k] <= t < tile_start[k+1].  The FP32 fused query
// kernel then walks the tiles persistently, fetching each tile's network
// weights from a device table of per-network pointers.  The tile shape (points
// per thread, hence points per tile) and the CTAs per SM come from the
// context's tuned configuration (nsdf_autotune_grouped).

#include "nsdf_internal.h"

namespace nsdf {
namespace {

// One thread builds the prefix sum (at most a few thousand networks).  An
// entry outside [0, max_total) is dropped (zero tiles) and flagged.
__global__ void build_tile_list_kernel(const int64_t *__restrict__ offsets,
                                       const int64_t *__restrict__ counts, int n_nets, int P,
                                       int64_t max_total, int32_t *__restrict__ tile_start,
                                       int *err) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t acc = 0;
  tile_start[0] = 0;
  for (int k = 0; k < n_nets; ++k) {
    const int64_t o = offsets[k], c = counts[k];
    int64_t tiles = 0;
    if (c > 0) {
      if (o < 0 || o > max_total - c) atomicExch(err, kDevBadWork);
      else tiles = (c + P - 1) / P;
    }
    acc += tiles;
    tile_start[k + 1] = (int32_t)acc;
  }
}

}  // namespace

cudaError_t launch_build_tile_list(const int64_t *offsets, const int64_t *counts, int n_nets, int P,
                                   int64_t max_total, int32_t *tile_start, int *err,
                                   cudaStream_t s) {
  build_tile_list_kernel<<<1, 32, 0, s>>>(offsets, counts, n_nets, P, max_total, tile_start, err);
  return cudaGetLastError();
}

}  // namespace nsdf
