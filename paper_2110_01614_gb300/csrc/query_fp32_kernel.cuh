// FP32 CUDA-core form of the fused collision query.
//
// One persistent CTA (256 threads) walks tiles of P points.  For each tile it
// runs, without leaving the SM:
//   * L0 (K = 3) on CUDA cores,
//   * the hidden layers z_l = W_l x_l + b_l, h_l = softplus_beta(z_l) (Eq. 1)
//     as register-blocked products against weight panels staged in shared
//     memory with cp.async,
//   * the output unit f = w_out . h + b_out,
//   * the Jacobian-transpose chain of Sec. 3.2: delta_l = sigmoid(beta z_l) *
//     g_l, g_{l-1} = W_l^T delta_l, down to grad f = W_0^T delta_0 (plus the
//     skip connection's direct term),
//   * Eq. 2 (normalise), the collision test f < eps and the contact point of
//     Eq. 3, with the optional rigid transform of Sec. 4.2.
// The paper's own networks (Sec. 4.3: a Fourier-feature layer, then ReLU
// layers) run through the same loop: gamma(p) = [sin(2 pi B p),
// cos(2 pi B p)] is written as the input tile of L0, which becomes a
// width x width panel product; the ReLU slope is the 0/1 step; and the
// reverse chain ends with g_gamma = W_0^T delta_0 folded into grad f through
// the feature Jacobian.
// sigmoid(beta z_l) of every hidden layer is parked in a per-CTA scratch
// slab between the forward and the reverse pass; it is written and read by
// the same thread in a lane-contiguous order (coalesced, L2-resident).

#pragma once

#include "nsdf_internal.h"
#include "ff_phase.cuh"

namespace nsdf {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr float kInvSqrt2 = 0.70710678118654752f;

template <int W, int PT_ = 8>
struct Cfg {
  static constexpr int WG = (W >= 256) ? 2 : 1;   // warps sharing a point group
  static constexpr int PT = PT_;                   // points per thread (tile shape)
  static constexpr int GROUPS = kWarps / WG;
  static constexpr int P = GROUPS * PT;            // points per tile
  static constexpr int CT = W / (32 * WG);         // columns per thread
  static constexpr int KC0 = 8192 / W;
  static constexpr int KC = KC0 > W ? W : (KC0 < 4 ? 4 : KC0);   // panel rows
  static constexpr int NCHUNK = W / KC;
  static_assert(W % (32 * WG) == 0, "width");
  static_assert(W % KC == 0 && KC % 4 == 0, "panel");
  // shared memory carve-up (floats)
  static constexpr int X_OFF = 0;
  static constexpr int Y_OFF = X_OFF + P * W;
  static constexpr int M_OFF = Y_OFF + P * W;
  static constexpr int PS_OFF = M_OFF + 2 * KC * W;          // float4 [P]
  static constexpr int RED_OFF = PS_OFF + 4 * P;             // [WG][P][4]
  static constexpr int DIR_OFF = RED_OFF + WG * P * 4;       // [P][4]
  static constexpr int SMEM_FLOATS = DIR_OFF + 4 * P;
  static constexpr size_t SMEM_BYTES = sizeof(float) * SMEM_FLOATS;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// softplus_beta(z) = max(z,0) + log1p(u)/beta and its derivative
// sigmoid(beta z), both from the same u = exp(-beta|z|) in (0, 1].  The
// hardware approximations suffice for the FP32 form: log(1 + u) on [1, 2]
// carries an absolute error of about 2^-21 and forming 1 + u at most ulp(1)/2,
// both divided by beta (1e-9 for beta = 100); exp and the reciprocal err by
// a few ulp relative, which moves u and the slope by about 1e-6 relative.
__device__ __forceinline__ void softplus_and_slope(float z, float beta, float inv_beta, float &h,
                                                   float &s) {
  const float u = __expf(-beta * fabsf(z));
  const float one_u = 1.0f + u;
  h = fmaf(__logf(one_u), inv_beta, fmaxf(z, 0.0f));
  const float inv = __fdividef(1.0f, one_u);
  s = (z >= 0.0f) ? inv : u * inv;
}

// The activation (softplus_beta or ReLU) and its slope.
__device__ __forceinline__ void act_and_slope(float z, float beta, float inv_beta, int relu, float &h,
                                              float &s) {
  if (relu) {
    h = fmaxf(z, 0.0f);
    s = z > 0.0f ? 1.0f : 0.0f;   // no gradient through a ReLU that outputs 0
  } else {
    softplus_and_slope(z, beta, inv_beta, h, s);
  }
}

// Stage rows [k0, k0+KC) of a row-major [W x W] panel into shared memory.
template <int W, int PT_ = 8>
__device__ __forceinline__ void stage_panel(float *dst, const float *src, int k0) {
  using C = Cfg<W, PT_>;
  constexpr int VEC = C::KC * W / 4;
  const float4 *s4 = reinterpret_cast<const float4 *>(src + (size_t)k0 * W);
  float4 *d4 = reinterpret_cast<float4 *>(dst);
  for (int v = threadIdx.x; v < VEC; v += kThreads) cp_async16(d4 + v, s4 + v);
  cp_async_commit();
}

// acc[i][j] = sum_k X[g*PT + i][k] * M[k][col_j] for the thread's PT points
// and CT columns; M is a global [W x W] row-major panel streamed through
// two shared buffers.  All threads of the CTA must call this together.
template <int W, int PT_ = 8>
__device__ __forceinline__ void panel_product(const float *X, const float *M, float *Ms,
                                              int g, int colbase,
                                              float (&acc)[Cfg<W, PT_>::PT][Cfg<W, PT_>::CT]) {
  using C = Cfg<W, PT_>;
#pragma unroll
  for (int i = 0; i < C::PT; ++i)
#pragma unroll
    for (int j = 0; j < C::CT; ++j) acc[i][j] = 0.0f;
  stage_panel<W, PT_>(Ms, M, 0);
  for (int kc = 0; kc < C::NCHUNK; ++kc) {
    if (kc + 1 < C::NCHUNK) {
      stage_panel<W, PT_>(Ms + ((kc + 1) & 1) * C::KC * W, M, (kc + 1) * C::KC);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float *Mc = Ms + (kc & 1) * C::KC * W;
    const float *Xr = X + (g * C::PT) * W + kc * C::KC;
#pragma unroll 1
    for (int kk = 0; kk < C::KC; kk += 4) {
      float4 xv[C::PT];
#pragma unroll
      for (int i = 0; i < C::PT; ++i) xv[i] = *reinterpret_cast<const float4 *>(Xr + i * W + kk);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float wv[C::CT];
#pragma unroll
        for (int j = 0; j < C::CT; ++j) wv[j] = Mc[(kk + q) * W + colbase + 32 * j];
#pragma unroll
        for (int i = 0; i < C::PT; ++i) {
          float xs = q == 0 ? xv[i].x : q == 1 ? xv[i].y : q == 2 ? xv[i].z : xv[i].w;
#pragma unroll
          for (int j = 0; j < C::CT; ++j) acc[i][j] = fmaf(xs, wv[j], acc[i][j]);
        }
      }
    }
    __syncthreads();
  }
}

// FF: the network has the Fourier-feature input layer (compiled separately,
// so that networks without it keep the registers, hence the occupancy, of a
// kernel without that code).
template <int W, int PT_ = 8, bool FF = false>
__global__ void __launch_bounds__(kThreads, 1) query_fp32_kernel(QueryParams prm) {
  using C = Cfg<W, PT_>;
  extern __shared__ float4 smem4[];
  float *smem = reinterpret_cast<float *>(smem4);
  float *X = smem + C::X_OFF;
  float *Y = smem + C::Y_OFF;
  float *Ms = smem + C::M_OFF;
  float4 *Ps = reinterpret_cast<float4 *>(smem + C::PS_OFF);
  float *red = smem + C::RED_OFF;
  float *dir = smem + C::DIR_OFF;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp / C::WG, part = warp % C::WG;
  const int colbase = part * (W / C::WG) + lane;
  const int L = prm.n_hidden;
  const int skip = prm.skip;
  const int nshort = W - 3;   // outputs of the layer feeding the skip
  const float beta = prm.beta;
  const float inv_beta = 1.0f / prm.beta;
  const bool grouped = prm.g_nets > 0;
  const int64_t ntiles = grouped ? (int64_t)prm.g_tile_start[prm.g_nets] : (prm.n + C::P - 1) / C::P;
  // per-CTA slope slab: [L-1][PT][CT][kThreads]
  float *slab = prm.scratch + (size_t)blockIdx.x * (size_t)(L - 1) * C::P * W;
  auto slot = [&](int l, int i, int j) -> float * {
    return slab + (((size_t)l * C::PT + i) * C::CT + j) * kThreads + tid;
  };

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // the tile's points [base, base + nvalid) and its network
    int64_t base, nvalid;
    const float *w0 = prm.w0, *bias = prm.bias, *fwd_t = prm.fwd_t, *bwdw = prm.bwd,
                *wout = prm.wout, *bout = prm.bout;
    const float *ffB = prm.ffB, *ff0_t = prm.ff0_t, *ff0 = prm.ff0;
    // the tile's body in a posed grouped launch (its pose is g_T[body]), or -1
    int body = -1;
    if (grouped) {
      int lo = 0, hi = prm.g_nets;               // last k with tile_start[k] <= tile
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prm.g_tile_start[mid] <= tile) lo = mid; else hi = mid;
      }
      const int64_t local = tile - prm.g_tile_start[lo];
      base = prm.g_offsets[lo] + local * C::P;
      nvalid = prm.g_counts[lo] - local * C::P;
      const NetPtrs &np = prm.g_netptrs[lo];
      w0 = np.w0; bias = np.bias; fwd_t = np.fwd_t; bwdw = np.bwd; wout = np.wout; bout = np.bout;
      ffB = np.ffB; ff0_t = np.ff0_t; ff0 = np.ff0;
      if (prm.g_T) body = lo;
    } else {
      base = tile * C::P;
      nvalid = prm.n - base;
    }
    if (nvalid > C::P) nvalid = C::P;
    // ---- a1: point load (+ T^{-1}) ----
    if (tid < C::P) {
      int64_t idx = base + tid;
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tid < nvalid) p = prm.pts[idx];
      if (body >= 0 || prm.has_T) {   // p' = T^{-1} p (Sec. 4.2)
        const float *t = body >= 0 ? prm.g_T + (size_t)kBodyFloats * body : prm.Ti;
        float x = t[0] * p.x + t[1] * p.y + t[2] * p.z + t[3];
        float y = t[4] * p.x + t[5] * p.y + t[6] * p.z + t[7];
        float z = t[8] * p.x + t[9] * p.y + t[10] * p.z + t[11];
        p.x = x; p.y = y; p.z = z;
      }
      Ps[tid] = p;
#pragma unroll
      for (int k = 0; k < 4; ++k) dir[tid * 4 + k] = 0.0f;
    }
    __syncthreads();

    float acc[C::PT][C::CT];
    float fpart[C::PT];
#pragma unroll
    for (int i = 0; i < C::PT; ++i) fpart[i] = 0.0f;

    const int m = FF ? prm.ff : 0;
    if (m > 0) {
      // ---- Fourier features gamma(p) (2m = W values) as L0's input tile ----
      // (columns not unrolled: this phase must not raise the kernel's registers)
#pragma unroll 1
      for (int j = 0; j < C::CT; ++j) {
        const int c = colbase + 32 * j;
        const int fi = c < m ? c : c - m;
        const float bx = ffB[fi * 3 + 0], by = ffB[fi * 3 + 1], bz = ffB[fi * 3 + 2];
#pragma unroll
        for (int i = 0; i < C::PT; ++i) {
          const int pr = g * C::PT + i;
          const float4 p = Ps[pr];
          float sn, cs;
          ff_sincos(bx, by, bz, p.x, p.y, p.z, sn, cs);
          X[pr * W + c] = c < m ? sn : cs;
        }
      }
      __syncthreads();
      panel_product<W, PT_>(X, ff0_t, Ms, g, colbase, acc);
    } else {
      // ---- a2: L0 (K = 3) on CUDA cores ----
#pragma unroll
      for (int j = 0; j < C::CT; ++j) {
        const int c = colbase + 32 * j;
        const float w0x = w0[c * 3 + 0], w0y = w0[c * 3 + 1], w0z = w0[c * 3 + 2];
#pragma unroll
        for (int i = 0; i < C::PT; ++i) {
          float4 p = Ps[g * C::PT + i];
          acc[i][j] = fmaf(w0x, p.x, fmaf(w0y, p.y, w0z * p.z));
        }
      }
    }

    // ---- a3/a4/a5: hidden layers, activation epilogue, output unit ----
    for (int l = 0; l < L; ++l) {
      if (l > 0) {
        float *t = X; X = Y; Y = t;
        panel_product<W, PT_>(X, fwd_t + (size_t)(l - 1) * W * W, Ms, g, colbase, acc);
      }
      const float *b = bias + (size_t)l * W;
      const bool last = (l == L - 1);
      const bool feeds_skip = (skip > 0 && l == skip - 1);
#pragma unroll
      for (int j = 0; j < C::CT; ++j) {
        const int c = colbase + 32 * j;
        const float bc = b[c];
        const float wo = last ? wout[c] : 0.0f;
#pragma unroll
        for (int i = 0; i < C::PT; ++i) {
          float h, s;
          act_and_slope(acc[i][j] + bc, beta, inv_beta, prm.relu, h, s);
          const int pr = g * C::PT + i;
          if (last) {
            fpart[i] = fmaf(wo, h, fpart[i]);
            Y[pr * W + c] = s * wo;          // delta_{L-1} = sigmoid' * w_out
          } else {
            *slot(l, i, j) = s;
            float v = h;
            if (feeds_skip) {
              if (c < nshort) {
                v = h * kInvSqrt2;
              } else {
                float4 p = Ps[pr];
                const int k = c - nshort;
                v = (k == 0 ? p.x : k == 1 ? p.y : p.z) * kInvSqrt2;
              }
            }
            Y[pr * W + c] = v;
          }
        }
      }
      __syncthreads();
    }

    // f: reduce the partial dot products over lanes, then over the WG warps
#pragma unroll
    for (int i = 0; i < C::PT; ++i) {
      float v = fpart[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[(part * C::P + g * C::PT + i) * 4 + 3] = v;
    }

    // ---- a6: Jacobian-transpose chain ----
    float gp[C::PT][3];
#pragma unroll
    for (int i = 0; i < C::PT; ++i) gp[i][0] = gp[i][1] = gp[i][2] = 0.0f;
    for (int l = L - 1; l >= 1; --l) {
      float *t = X; X = Y; Y = t;                       // X = delta_l
      panel_product<W, PT_>(X, bwdw + (size_t)(l - 1) * W * W, Ms, g, colbase, acc);
      const bool at_skip = (skip > 0 && l == skip);
#pragma unroll
      for (int j = 0; j < C::CT; ++j) {
        const int c = colbase + 32 * j;
#pragma unroll
        for (int i = 0; i < C::PT; ++i) {
          const int pr = g * C::PT + i;
          float u = acc[i][j];
          if (at_skip) {
            u *= kInvSqrt2;
            if (c >= nshort) {                 // direct path to the input
              dir[pr * 4 + (c - nshort)] += u;
              u = 0.0f;
            }
          }
          const float d = *slot(l - 1, i, j) * u;
          if (l - 1 > 0 || m > 0) {
            Y[pr * W + c] = d;                 // delta_{l-1} (delta_0 feeds W_0^T below)
          } else {
            gp[i][0] = fmaf(d, w0[c * 3 + 0], gp[i][0]);
            gp[i][1] = fmaf(d, w0[c * 3 + 1], gp[i][1]);
            gp[i][2] = fmaf(d, w0[c * 3 + 2], gp[i][2]);
          }
        }
      }
      __syncthreads();
    }
    if (m > 0) {
      // ---- g_gamma = W_0^T delta_0, then through the feature Jacobian ----
      //   d sin(2 pi b.p)/dp = 2 pi cos(2 pi b.p) b,
      //   d cos(2 pi b.p)/dp = -2 pi sin(2 pi b.p) b
      float *t = X; X = Y; Y = t;                       // X = delta_0
      panel_product<W, PT_>(X, ff0, Ms, g, colbase, acc);
      // park g_gamma in Y (each thread its own elements, so no barrier), so
      // that acc is dead while the sines and cosines are evaluated
#pragma unroll
      for (int j = 0; j < C::CT; ++j)
#pragma unroll
        for (int i = 0; i < C::PT; ++i) Y[(g * C::PT + i) * W + colbase + 32 * j] = acc[i][j];
      constexpr float kTwoPi = 6.28318530717958648f;
#pragma unroll 1
      for (int j = 0; j < C::CT; ++j) {
        const int c = colbase + 32 * j;
        const int fi = c < m ? c : c - m;
        const float bx = ffB[fi * 3 + 0], by = ffB[fi * 3 + 1], bz = ffB[fi * 3 + 2];
#pragma unroll
        for (int i = 0; i < C::PT; ++i) {
          const int pr = g * C::PT + i;
          const float4 p = Ps[pr];
          const float gg = Y[pr * W + c];
          float sn, cs;
          ff_sincos(bx, by, bz, p.x, p.y, p.z, sn, cs);
          const float coef = kTwoPi * (c < m ? gg * cs : -gg * sn);
          gp[i][0] = fmaf(coef, bx, gp[i][0]);
          gp[i][1] = fmaf(coef, by, gp[i][1]);
          gp[i][2] = fmaf(coef, bz, gp[i][2]);
        }
      }
    } else if (L == 1) {
      // no hidden-to-hidden product: delta_0 = sigmoid'(z_0) * w_out sits in Y
#pragma unroll
      for (int j = 0; j < C::CT; ++j) {
        const int c = colbase + 32 * j;
#pragma unroll
        for (int i = 0; i < C::PT; ++i) {
          const float d = Y[(g * C::PT + i) * W + c];
          gp[i][0] = fmaf(d, w0[c * 3 + 0], gp[i][0]);
          gp[i][1] = fmaf(d, w0[c * 3 + 1], gp[i][1]);
          gp[i][2] = fmaf(d, w0[c * 3 + 2], gp[i][2]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < C::PT; ++i) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float v = gp[i][k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[(part * C::P + g * C::PT + i) * 4 + k] = v;
      }
    }
    __syncthreads();

    // ---- a7/a8/a9: normalise, collision test, projection ----
    if (tid < C::P) {
      const int64_t idx = base + tid;
      float gx = dir[tid * 4 + 0], gy = dir[tid * 4 + 1], gz = dir[tid * 4 + 2];
      float f = bout[0];
#pragma unroll
      for (int q = 0; q < C::WG; ++q) {
        const float *r = red + (q * C::P + tid) * 4;
        gx += r[0]; gy += r[1]; gz += r[2]; f += r[3];
      }
      if (tid < nvalid) {
        const float nrm = sqrtf(gx * gx + gy * gy + gz * gz);
        float nx = 0.f, ny = 0.f, nz = 0.f;
        if (nrm >= 1e-20f) { nx = gx / nrm; ny = gy / nrm; nz = gz / nrm; }
        if (prm.grad_scale) {
          const float a = prm.grad_scale[idx];
          prm.out_grad[idx] = make_float4(a * gx, a * gy, a * gz, 0.f);
        } else if (!prm.collide) {
          if (prm.raw_gradient) { nx = gx; ny = gy; nz = gz; }
          prm.out_n_sdf[idx] = make_float4(nx, ny, nz, f);
        } else {
          if (body >= 0 || prm.has_T) {   // N rotated by T[:3,:3]
            const float *R = body >= 0 ? prm.g_T + (size_t)kBodyFloats * body + 12 : prm.R;
            float wx = R[0] * nx + R[1] * ny + R[2] * nz;
            float wy = R[3] * nx + R[4] * ny + R[5] * nz;
            float wz = R[6] * nx + R[7] * ny + R[8] * nz;
            nx = wx; ny = wy; nz = wz;
          }
          const bool hit = f < prm.eps;
          float4 p = prm.pts[idx];
          if (hit) {
            const float d = prm.eps - f;
            p.x = fmaf(d, nx, p.x); p.y = fmaf(d, ny, p.y); p.z = fmaf(d, nz, p.z);
          }
          if (prm.out_pts) prm.out_pts[idx] = p;
          if (prm.out_n_sdf) prm.out_n_sdf[idx] = make_float4(nx, ny, nz, f);
          if (prm.out_hit) prm.out_hit[idx] = hit ? 1 : 0;
        }
      }
    }
    __syncthreads();
  }
}

// Host helpers of one (W, PT, FF) instantiation.
template <int W, int PT_, bool FF>
int per_sm_t() {
  using C = Cfg<W, PT_>;
  int per_sm = 1;
  // the occupancy of a kernel above 48 KB of dynamic shared memory is only
  // known once its opt-in attribute is set
  cudaFuncSetAttribute(query_fp32_kernel<W, PT_, FF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)C::SMEM_BYTES);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, query_fp32_kernel<W, PT_, FF>, kThreads,
                                                C::SMEM_BYTES);
  return per_sm < 1 ? 1 : per_sm;
}

template <int W, int PT_, bool FF>
cudaError_t launch_t(const QueryParams &p, int grid, cudaStream_t s) {
  using C = Cfg<W, PT_>;
  cudaError_t e = cudaFuncSetAttribute(query_fp32_kernel<W, PT_, FF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  query_fp32_kernel<W, PT_, FF><<<grid, kThreads, C::SMEM_BYTES, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

#define NSDF_FP32_WIDTHS(X) X(32) X(64) X(128) X(256) X(512)

}  // namespace nsdf
