// One explicit Verlet step of a rectangular quad cloth (Sec. 4.1).
//
// Each thread owns one vertex and gathers the Hooke forces of its (up to)
// eight springs from the implicit grid topology: four structural neighbours
// (rest lengths hx along a row, hz between rows) and four shear neighbours
// (rest length sqrt(hx^2 + hz^2)).  Unit mass:
//   x_new = 2 x - x_prev + dt^2 (sum_j k (|d_j| - r_j) d_j/|d_j| + (0, -g, 0)).
// Gathering per vertex needs no atomics; every spring is evaluated from both
// ends, with equal and opposite results.  x_new overwrites x_prev in place
// (each thread reads and writes only its own x_prev entry).  The step is
// memory-bound: one float4 read of x_prev, one write, and x reads that hit
// L1/L2 for the neighbours.

#include "nsdf_internal.h"

namespace nsdf {
namespace {

__global__ void __launch_bounds__(256) cloth_step_kernel(const float4 *__restrict__ x,
                                                         float4 *__restrict__ xprev, int nx, int ny,
                                                         float hx, float hz, float k, float g,
                                                         float dt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;   // column (along x)
  const int i = blockIdx.y;                              // row (along z)
  if (j >= nx || i >= ny) return;
  const int64_t v = (int64_t)i * nx + j;
  const float4 p = x[v];
  const float hd = sqrtf(hx * hx + hz * hz);
  float ax = 0.f, ay = -g, az = 0.f;
  const int di[8] = {0, 0, -1, 1, -1, -1, 1, 1};
  const int dj[8] = {-1, 1, 0, 0, -1, 1, -1, 1};
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int ii = i + di[s], jj = j + dj[s];
    if (ii < 0 || ii >= ny || jj < 0 || jj >= nx) continue;
    const float rest = s < 2 ? hx : (s < 4 ? hz : hd);
    const float4 q = x[(int64_t)ii * nx + jj];
    const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
    const float len = sqrtf(dx * dx + dy * dy + dz * dz);
    const float f = len > 0.f ? k * (len - rest) / len : 0.f;
    ax = fmaf(f, dx, ax); ay = fmaf(f, dy, ay); az = fmaf(f, dz, az);
  }
  const float4 pp = xprev[v];
  const float dt2 = dt * dt;
  float4 o;
  o.x = 2.f * p.x - pp.x + dt2 * ax;
  o.y = 2.f * p.y - pp.y + dt2 * ay;
  o.z = 2.f * p.z - pp.z + dt2 * az;
  o.w = p.w;
  xprev[v] = o;
}

}  // namespace
}  // namespace nsdf

extern "C" nsdf_status nsdf_cloth_step(const float *x, float *x_prev_inout, int nx, int ny, float hx,
                                       float hz, float k_over_m, float g, float dt,
                                       nsdf_stream stream) {
  if (nx < 0 || ny < 0 || !(hx > 0.f) || !(hz > 0.f) || !(dt > 0.f)) return NSDF_ERR_INVALID_ARG;
  if (nx == 0 || ny == 0) return NSDF_OK;
  if (!x || !x_prev_inout || x == x_prev_inout || ny > 65535 || nx > (1 << 30))
    return NSDF_ERR_INVALID_ARG;   // grid.y limit; the column index stays an int
  if ((reinterpret_cast<uintptr_t>(x) & 15u) || (reinterpret_cast<uintptr_t>(x_prev_inout) & 15u))
    return NSDF_ERR_MISALIGNED;
  if (!nsdf::device_memory(x) || !nsdf::device_memory(x_prev_inout)) return NSDF_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  dim3 grid((nx + 255) / 256, ny);
  nsdf::cloth_step_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const float4 *>(x),
                                               reinterpret_cast<float4 *>(x_prev_inout), nx, ny,
                                               hx, hz, k_over_m, g, dt);
  return cudaGetLastError() == cudaSuccess ? NSDF_OK : NSDF_ERR_CUDA;
}
