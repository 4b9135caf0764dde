// Brute-force exact signed distance to a watertight triangle mesh: the
// ground truth a network is fitted to (Sec. 3.1) and the plain reference a
// cloth run can collide against.
//
// Per point: unsigned distance = min over triangles of the distance to the
// triangle's closest point (barycentric Voronoi-region test: vertex, edge or
// face region); sign from the generalized winding number
// w = sum_t Omega_t / (4 pi), inside (negative, Sec. 3.2) when w > 1/2, with
// Omega_t from the Van Oosterom-Strackee formula.
//
// Triangles stream through shared memory in chunks; each thread owns one
// point: an explicit float4, or node (i, j, k) of a regular grid (i fastest)
// when the voxel baseline builds its grid.  w is accumulated in FP32; for points where that is not decisive
// (|w - 1/2| < 0.25, or distance < 1e-3 where one nearby triangle's solid
// angle is ill-conditioned) the warp recomputes w in FP64, all 32 lanes
// splitting the triangles of one such point at a time.

#include "nsdf_internal.h"

namespace nsdf {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 512;           // triangles per shared-memory chunk
constexpr float kInv4Pi = 0.0795774715459476679f;

struct TriChunk {
  float ax[kChunk], ay[kChunk], az[kChunk];
  float bx[kChunk], by[kChunk], bz[kChunk];
  float cx[kChunk], cy[kChunk], cz[kChunk];
};

// A face with a vertex index outside [0, nv) is replaced by a triangle
// collapsed onto a point 1e30 away: it is never the closest and its solid
// angle is zero, so it drops out without an out-of-bounds read.
__device__ void load_chunk(TriChunk &t, const float *__restrict__ V, int64_t nv,
                           const int32_t *__restrict__ F, int64_t f0, int64_t nf) {
  for (int i = threadIdx.x; i < kChunk; i += blockDim.x) {
    const int64_t f = f0 + i;
    if (f < nf) {
      const int64_t a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
      if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) {
        t.ax[i] = t.bx[i] = t.cx[i] = 1e30f;
        t.ay[i] = t.by[i] = t.cy[i] = 0.f;
        t.az[i] = t.bz[i] = t.cz[i] = 0.f;
        continue;
      }
      t.ax[i] = V[3 * a]; t.ay[i] = V[3 * a + 1]; t.az[i] = V[3 * a + 2];
      t.bx[i] = V[3 * b]; t.by[i] = V[3 * b + 1]; t.bz[i] = V[3 * b + 2];
      t.cx[i] = V[3 * c]; t.cy[i] = V[3 * c + 1]; t.cz[i] = V[3 * c + 2];
    }
  }
}

template <typename T>
struct V3 {
  T x, y, z;
};
template <typename T>
__device__ __forceinline__ V3<T> sub(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T>
__device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
__device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Squared distance from p to triangle (a, b, c) by its Voronoi regions.
__device__ __forceinline__ float tri_dist2(V3<float> p, V3<float> a, V3<float> b, V3<float> c) {
  const V3<float> ab = sub(b, a), ac = sub(c, a), ap = sub(p, a);
  const float d1 = dot(ab, ap), d2 = dot(ac, ap);
  V3<float> q;
  if (d1 <= 0.f && d2 <= 0.f) {
    q = a;
  } else {
    const V3<float> bp = sub(p, b);
    const float d3 = dot(ab, bp), d4 = dot(ac, bp);
    if (d3 >= 0.f && d4 <= d3) {
      q = b;
    } else {
      const float vc = d1 * d4 - d3 * d2;
      if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
        const float v = d1 / (d1 - d3);
        q = {a.x + v * ab.x, a.y + v * ab.y, a.z + v * ab.z};
      } else {
        const V3<float> cp = sub(p, c);
        const float d5 = dot(ab, cp), d6 = dot(ac, cp);
        if (d6 >= 0.f && d5 <= d6) {
          q = c;
        } else {
          const float vb = d5 * d2 - d1 * d6;
          if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
            const float w = d2 / (d2 - d6);
            q = {a.x + w * ac.x, a.y + w * ac.y, a.z + w * ac.z};
          } else {
            const float va = d3 * d6 - d5 * d4;
            if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
              const float w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
              q = {b.x + w * (c.x - b.x), b.y + w * (c.y - b.y), b.z + w * (c.z - b.z)};
            } else {
              const float den = 1.f / (va + vb + vc);
              const float v = vb * den, w = vc * den;
              q = {a.x + ab.x * v + ac.x * w, a.y + ab.y * v + ac.y * w, a.z + ab.z * v + ac.z * w};
            }
          }
        }
      }
    }
  }
  const V3<float> d = sub(p, q);
  return dot(d, d);
}

template <typename T>
__device__ __forceinline__ T solid_angle(V3<T> p, V3<T> a, V3<T> b, V3<T> c) {
  const V3<T> A = sub(a, p), B = sub(b, p), C = sub(c, p);
  const T la = sqrt(dot(A, A)), lb = sqrt(dot(B, B)), lc = sqrt(dot(C, C));
  const T num = dot(A, cross(B, C));
  const T den = la * lb * lc + dot(A, B) * lc + dot(A, C) * lb + dot(B, C) * la;
  return T(2) * atan2(num, den);
}

// Points of the implicit grid: node (i, j, k) at lo + (i, j, k) * h, index
// i + N (j + N k).
struct GridPts {
  int n;
  float lo[3], h[3];
};

__global__ void __launch_bounds__(kThreads) mesh_sdf_kernel(const float *__restrict__ V, int64_t nv,
                                                            const int32_t *__restrict__ F,
                                                            int64_t nf, const float4 *__restrict__ pts,
                                                            int64_t n, float *__restrict__ out,
                                                            const GridPts grid) {
  extern __shared__ float4 smem4[];
  TriChunk &tc = *reinterpret_cast<TriChunk *>(smem4);
  __shared__ double wacc[kThreads / 32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (idx < n) {
    if (pts) {
      p4 = pts[idx];
    } else {
      const int64_t N = grid.n;
      p4.x = grid.lo[0] + grid.h[0] * (float)(idx % N);
      p4.y = grid.lo[1] + grid.h[1] * (float)((idx / N) % N);
      p4.z = grid.lo[2] + grid.h[2] * (float)(idx / (N * N));
    }
  }
  const V3<float> p = {p4.x, p4.y, p4.z};
  float best = 3.4e38f, wsum = 0.f;
  for (int64_t f0 = 0; f0 < nf; f0 += kChunk) {
    __syncthreads();
    load_chunk(tc, V, nv, F, f0, nf);
    __syncthreads();
    const int m = (int)((nf - f0) < kChunk ? (nf - f0) : kChunk);
    for (int i = 0; i < m; ++i) {
      const V3<float> a = {tc.ax[i], tc.ay[i], tc.az[i]};
      const V3<float> b = {tc.bx[i], tc.by[i], tc.bz[i]};
      const V3<float> c = {tc.cx[i], tc.cy[i], tc.cz[i]};
      best = fminf(best, tri_dist2(p, a, b, c));
      wsum += solid_angle<float>(p, a, b, c);
    }
  }
  const float dist = sqrtf(best);
  float w = wsum * kInv4Pi;
  const bool redo = (idx < n) && (fabsf(w - 0.5f) < 0.25f || dist < 1e-3f);
  // FP64 winding number for the undecided points of this CTA
  const int any = __syncthreads_or(redo ? 1 : 0);
  if (any) {
    const unsigned mask = __ballot_sync(0xffffffffu, redo);
    wacc[warp][lane] = 0.0;
    for (int64_t f0 = 0; f0 < nf; f0 += kChunk) {
      __syncthreads();
      load_chunk(tc, V, nv, F, f0, nf);
      __syncthreads();
      const int m = (int)((nf - f0) < kChunk ? (nf - f0) : kChunk);
      unsigned todo = mask;
      while (todo) {
        const int q = __ffs(todo) - 1;
        todo &= todo - 1;
        const V3<double> pq = {(double)__shfl_sync(0xffffffffu, p.x, q),
                               (double)__shfl_sync(0xffffffffu, p.y, q),
                               (double)__shfl_sync(0xffffffffu, p.z, q)};
        double part = 0.0;
        for (int i = lane; i < m; i += 32) {
          const V3<double> a = {tc.ax[i], tc.ay[i], tc.az[i]};
          const V3<double> b = {tc.bx[i], tc.by[i], tc.bz[i]};
          const V3<double> c = {tc.cx[i], tc.cy[i], tc.cz[i]};
          part += solid_angle<double>(pq, a, b, c);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) wacc[warp][q] += part;
      }
    }
    __syncwarp();
    if (redo) w = (float)(wacc[warp][lane] / (4.0 * 3.14159265358979323846));
  }
  if (idx < n) out[idx] = (w > 0.5f) ? -dist : dist;
}

}  // namespace

cudaError_t launch_mesh_sdf(const float *verts, int64_t n_verts, const int32_t *faces,
                            int64_t n_faces, const float4 *pts, int64_t n, float *out, int grid_n,
                            const float *lo, const float *h, cudaStream_t s) {
  const size_t smem = sizeof(TriChunk);
  cudaError_t e = cudaFuncSetAttribute(mesh_sdf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  GridPts g{};
  if (!pts) {
    g.n = grid_n;
    for (int c = 0; c < 3; ++c) {
      g.lo[c] = lo[c];
      g.h[c] = h[c];
    }
  }
  const int64_t blocks = (n + kThreads - 1) / kThreads;
  mesh_sdf_kernel<<<(unsigned)blocks, kThreads, smem, s>>>(verts, n_verts, faces, n_faces, pts, n,
                                                          out, g);
  return cudaGetLastError();
}

}  // namespace nsdf

extern "C" nsdf_status nsdf_mesh_sdf(const float *verts, int64_t n_verts, const int32_t *faces,
                                     int64_t n_faces, const float *pts, int64_t n, float *out_sdf,
                                     nsdf_stream stream) {
  if (n < 0 || n_verts < 0 || n_faces < 0) return NSDF_ERR_INVALID_ARG;
  if (n == 0) return NSDF_OK;
  if (!verts || !faces || !pts || !out_sdf || n_faces == 0 || n_verts < 3) return NSDF_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(pts) & 15u) != 0) return NSDF_ERR_MISALIGNED;
  if (!nsdf::device_memory(verts) || !nsdf::device_memory(faces) || !nsdf::device_memory(pts) ||
      !nsdf::device_memory(out_sdf))
    return NSDF_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  return nsdf::launch_mesh_sdf(verts, n_verts, faces, n_faces, reinterpret_cast<const float4 *>(pts),
                               n, out_sdf, 0, nullptr, nullptr, s) == cudaSuccess
             ? NSDF_OK
             : NSDF_ERR_CUDA;
}
