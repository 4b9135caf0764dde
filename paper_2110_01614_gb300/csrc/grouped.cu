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
// entry outside [0, max_total) is dropped (zero tiles) and flagged.  Each
// network's tile count is rounded up to a multiple of `round_to` (the
// tensor-core kernel hands tiles to 2-CTA clusters in pairs that must share
// a network).
__global__ void build_tile_list_kernel(const int64_t *__restrict__ offsets,
                                       const int64_t *__restrict__ counts, int n_nets, int P,
                                       int round_to, int64_t max_total,
                                       int32_t *__restrict__ tile_start, int *err) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t acc = 0;
  tile_start[0] = 0;
  for (int k = 0; k < n_nets; ++k) {
    const int64_t o = offsets[k], c = counts[k];
    int64_t tiles = 0;
    if (c > 0) {
      if (o < 0 || o > max_total - c) atomicExch(err, kDevBadWork);
      else tiles = ((c + P - 1) / P + round_to - 1) / round_to * round_to;
    }
    acc += tiles;
    tile_start[k + 1] = (int32_t)acc;
  }
}

// One thread per body: T = [A | t; 0 0 0 1] (the last row is not read) gives
// the point map T^{-1} = [A^{-1} | -A^{-1} t] of Sec. 4.2, inverted in FP64
// through the adjugate, and the normal rotation A.  A singular A is flagged
// and replaced by the identity.
__global__ void body_transforms_kernel(const float *__restrict__ T, int n_nets,
                                       float *__restrict__ out, int *err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_nets) return;
  const float *t = T + 16 * k;
  const double a[9] = {t[0], t[1], t[2], t[4], t[5], t[6], t[8], t[9], t[10]};
  const double tx = t[3], ty = t[7], tz = t[11];
  // adjugate, row-major: adj[r][c] = cofactor of a[c][r]
  double adj[9] = {a[4] * a[8] - a[5] * a[7], a[2] * a[7] - a[1] * a[8], a[1] * a[5] - a[2] * a[4],
                   a[5] * a[6] - a[3] * a[8], a[0] * a[8] - a[2] * a[6], a[2] * a[3] - a[0] * a[5],
                   a[3] * a[7] - a[4] * a[6], a[1] * a[6] - a[0] * a[7], a[0] * a[4] - a[1] * a[3]};
  const double det = a[0] * adj[0] + a[1] * adj[3] + a[2] * adj[6];
  float *o = out + (size_t)kBodyFloats * k;
  const bool ok = fabs(det) > 1e-30 && isfinite(det);
  if (!ok) atomicExch(err, kDevBadWork);
  for (int r = 0; r < 3; ++r) {
    double inv[3];
    for (int c = 0; c < 3; ++c) inv[c] = ok ? adj[r * 3 + c] / det : (r == c ? 1.0 : 0.0);
    o[r * 4 + 0] = (float)inv[0];
    o[r * 4 + 1] = (float)inv[1];
    o[r * 4 + 2] = (float)inv[2];
    o[r * 4 + 3] = ok ? (float)(-(inv[0] * tx + inv[1] * ty + inv[2] * tz)) : 0.f;
  }
  for (int i = 0; i < 9; ++i) o[12 + i] = ok ? (float)a[i] : (i % 4 == 0 ? 1.f : 0.f);
  for (int i = 21; i < kBodyFloats; ++i) o[i] = 0.f;
}

}  // namespace

cudaError_t launch_body_transforms(const float *T, int n_nets, float *out, int *err,
                                   cudaStream_t s) {
  body_transforms_kernel<<<(n_nets + 127) / 128, 128, 0, s>>>(T, n_nets, out, err);
  return cudaGetLastError();
}

cudaError_t launch_build_tile_list(const int64_t *offsets, const int64_t *counts, int n_nets, int P,
                                   int64_t max_total, int32_t *tile_start, int *err,
                                   cudaStream_t s, int round_to) {
  build_tile_list_kernel<<<1, 32, 0, s>>>(offsets, counts, n_nets, P, round_to, max_total,
                                          tile_start, err);
  return cudaGetLastError();
}

}  // namespace nsdf
