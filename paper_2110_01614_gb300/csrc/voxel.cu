// Voxel SDF baseline: the comparison system of Sec. 4.3 (Table 1), a signed
// distance sampled on a regular N^3 grid and looked up by trilinear
// interpolation, against which the network's memory, speed and accuracy are
// set.
//
// Build: every grid node's exact signed distance to the mesh, from the
// brute-force kernel (mesh_sdf.cu) run over the implicit grid.
// Query (one thread per point, float4 in and out): u = (p - lo) / h clamped
// to the box; the cell c = min(floor(u), N - 2) and t = u - c; sdf = the
// trilinear interpolant of the cell's 8 nodes; grad = its analytic gradient
// (each axis a difference of the two faces, interpolated bilinearly in the
// other two axes, divided by h).  A point outside the box gets the value at
// its clamped point plus its distance d to the box, and the gradient plus
// the outward direction (p - clamp(p)) / d.  Then Eq. 2, the test f < eps
// and Eq. 3 as in the network query.  Bound: the 8 gathers per point (the
// 64 MB grid of N = 256 stays in L2).

#include <cmath>

#include "nsdf_internal.h"

namespace nsdf {
namespace {

struct Box {
  int n;
  float lo[3], h[3], inv_h[3];
};

__global__ void __launch_bounds__(256) voxel_collide_kernel(const float *__restrict__ grid, Box b,
                                                            const float4 *__restrict__ pts, int64_t n,
                                                            float eps, float4 *__restrict__ out_pts,
                                                            float4 *__restrict__ out_n_sdf,
                                                            uint8_t *__restrict__ out_hit) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = pts[i];
  const float pc[3] = {p.x, p.y, p.z};
  float t[3], out[3];
  int c[3];
  float d2 = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float u = (pc[a] - b.lo[a]) * b.inv_h[a];
    const float top = (float)(b.n - 1);
    float q = pc[a];
    if (!(u >= 0.f)) { u = 0.f; q = b.lo[a]; }          // below the box, or NaN: cell 0
    else if (u > top) { u = top; q = b.lo[a] + top * b.h[a]; }
    out[a] = pc[a] - q;
    d2 = fmaf(out[a], out[a], d2);
    int ci = (int)floorf(u);
    if (ci > b.n - 2) ci = b.n - 2;
    c[a] = ci;
    t[a] = u - (float)ci;
  }
  const int64_t N = b.n;
  const float *g = grid + ((int64_t)c[2] * N + c[1]) * N + c[0];
  const int64_t sy = N, sz = N * N;
  const float v000 = __ldg(g), v100 = __ldg(g + 1);
  const float v010 = __ldg(g + sy), v110 = __ldg(g + sy + 1);
  const float v001 = __ldg(g + sz), v101 = __ldg(g + sz + 1);
  const float v011 = __ldg(g + sz + sy), v111 = __ldg(g + sz + sy + 1);
  const float tx = t[0], ty = t[1], tz = t[2];
  // along x, then y, then z
  const float x00 = fmaf(tx, v100 - v000, v000), x10 = fmaf(tx, v110 - v010, v010);
  const float x01 = fmaf(tx, v101 - v001, v001), x11 = fmaf(tx, v111 - v011, v011);
  const float y0 = fmaf(ty, x10 - x00, x00), y1 = fmaf(ty, x11 - x01, x01);
  float f = fmaf(tz, y1 - y0, y0);
  // the gradient of the interpolant (zero along an axis where p was clamped)
  const float dx0 = fmaf(ty, (v110 - v010) - (v100 - v000), v100 - v000);
  const float dx1 = fmaf(ty, (v111 - v011) - (v101 - v001), v101 - v001);
  const float dy0 = x10 - x00, dy1 = x11 - x01;
  float gx = fmaf(tz, dx1 - dx0, dx0) * b.inv_h[0];
  float gy = fmaf(tz, dy1 - dy0, dy0) * b.inv_h[1];
  float gz = (y1 - y0) * b.inv_h[2];
  if (out[0] != 0.f) gx = 0.f;
  if (out[1] != 0.f) gy = 0.f;
  if (out[2] != 0.f) gz = 0.f;
  if (!(d2 <= 0.f)) {          // outside the box (a NaN coordinate makes f NaN too)
    const float d = sqrtf(d2);
    f += d;
    gx += out[0] / d;
    gy += out[1] / d;
    gz += out[2] / d;
  }
  const float nrm = sqrtf(gx * gx + gy * gy + gz * gz);
  float nx = 0.f, ny = 0.f, nz = 0.f;
  if (nrm >= 1e-20f) { nx = gx / nrm; ny = gy / nrm; nz = gz / nrm; }
  const bool hit = f < eps;
  float4 q = p;
  if (hit) {
    const float dd = eps - f;
    q.x = fmaf(dd, nx, q.x); q.y = fmaf(dd, ny, q.y); q.z = fmaf(dd, nz, q.z);
  }
  out_pts[i] = q;
  if (out_n_sdf) out_n_sdf[i] = make_float4(nx, ny, nz, f);
  if (out_hit) out_hit[i] = hit ? 1 : 0;
}

bool make_box(int n, const float *lo, const float *hi, Box *b) {
  if (n < 2 || n > 2048 || !lo || !hi) return false;
  b->n = n;
  for (int a = 0; a < 3; ++a) {
    if (!(hi[a] > lo[a]) || !std::isfinite(lo[a]) || !std::isfinite(hi[a])) return false;
    b->lo[a] = lo[a];
    b->h[a] = (hi[a] - lo[a]) / (float)(n - 1);
    b->inv_h[a] = 1.0f / b->h[a];
  }
  return true;
}

}  // namespace
}  // namespace nsdf

using namespace nsdf;

extern "C" nsdf_status nsdf_voxel_build(const float *verts, int64_t n_verts, const int32_t *faces,
                                        int64_t n_faces, int n, const float *lo, const float *hi,
                                        float *grid, nsdf_stream stream) {
  Box b{};
  if (!make_box(n, lo, hi, &b) || !verts || !faces || !grid || n_faces <= 0 || n_verts < 3)
    return NSDF_ERR_INVALID_ARG;
  if (!device_memory(verts) || !device_memory(faces) || !device_memory(grid)) return NSDF_ERR_INVALID_ARG;
  const int64_t nodes = (int64_t)n * n * n;
  return launch_mesh_sdf(verts, n_verts, faces, n_faces, nullptr, nodes, grid, n, b.lo, b.h,
                         reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? NSDF_OK
             : NSDF_ERR_CUDA;
}

extern "C" nsdf_status nsdf_voxel_collide(const float *grid, int n, const float *lo, const float *hi,
                                          const float *pts, int64_t n_pts, float eps, float *out_pts,
                                          float *out_n_sdf, uint8_t *out_hit, nsdf_stream stream) {
  Box b{};
  if (!make_box(n, lo, hi, &b) || n_pts < 0 || !std::isfinite(eps)) return NSDF_ERR_INVALID_ARG;
  if (n_pts == 0) return NSDF_OK;
  if (!grid || !pts || !out_pts) return NSDF_ERR_INVALID_ARG;
  auto mis = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
  if (mis(pts) || mis(out_pts) || (out_n_sdf && mis(out_n_sdf))) return NSDF_ERR_MISALIGNED;
  if (!device_memory(grid) || !device_memory(pts) || !device_memory(out_pts) ||
      (out_n_sdf && !device_memory(out_n_sdf)) || (out_hit && !device_memory(out_hit)))
    return NSDF_ERR_INVALID_ARG;
  const int64_t blocks = (n_pts + 255) / 256;
  voxel_collide_kernel<<<(unsigned)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      grid, b, reinterpret_cast<const float4 *>(pts), n_pts, eps, reinterpret_cast<float4 *>(out_pts),
      reinterpret_cast<float4 *>(out_n_sdf), out_hit);
  return cudaGetLastError() == cudaSuccess ? NSDF_OK : NSDF_ERR_CUDA;
}
