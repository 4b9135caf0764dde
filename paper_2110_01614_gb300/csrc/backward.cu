// Hand-written backward of the network query (FP32, CUDA cores).
//
// For L = sum_i a_i f(p_i) + v_i . grad f(p_i) (a = g_sdf, v = g_grad) this
// computes dL/dtheta (all weights and biases, blob layout) and dL/dp_i.
// v . grad f is the directional derivative of f along v, so each tile of
// points runs one forward pass carrying a primal stream (x, z, h) and a
// tangent stream (xd = v at the input, zd = W xd, hd = s * zd with
// s = sigmoid(beta z)), then plain reverse mode over both streams:
//   zdb = s * hdb,   zb = s * hb + zd * hdb * beta s (1 - s),
//   dW += zb x^T + zdb xd^T,   db += zb,   (hb, hdb) <- W^T (zb, zdb).
// The d sigmoid / dz = beta s (1 - s) term is the second-order part that the
// eikonal term of a fitting loss needs.  Activations are recomputed per tile
// (never stored for the whole batch): the tile's layer inputs, slopes and
// tangents live in shared memory only while that tile is processed.
// Weight gradients accumulate per CTA in shared memory; the partial sums of
// all CTAs are then added in CTA order by a second kernel (deterministic).

#include "nsdf_internal.h"

namespace nsdf {
namespace {

constexpr int kThreads = 256;
constexpr int kP = 32;                      // points per tile
constexpr int kMaxL = 16;
constexpr float kInvSqrt2 = 0.70710678118654752f;

struct BwdParams {
  const float4 *pts;
  int64_t n;
  const float *a;        // [n]
  const float4 *v;       // [n] or null
  float *g_partial;      // [grid][n_params] or null
  float4 *g_pts;         // [n] or null
  const float *w0, *bias, *fwd_t, *bwd, *wout, *bout;
  int W, L, skip;
  float beta;
  int64_t n_params;
  int64_t woff[kMaxL + 1], boff[kMaxL + 1];
  int out[kMaxL + 1];
};

__device__ __forceinline__ void sp_and_slope(float z, float beta, float &h, float &s) {
  const float e = expf(-beta * fabsf(z));
  h = fmaxf(z, 0.0f) + log1pf(e) / beta;
  const float inv = 1.0f / (1.0f + e);
  s = (z >= 0.0f) ? inv : e * inv;
}

// Shared-memory carve-up (floats), identical on host and device.
struct BwdLayout {
  int W, L;
  __host__ __device__ int wt() const { return 0; }                         // [L-1][W(k)][W(n)]
  __host__ __device__ int xs() const { return wt() + (L - 1) * W * W; }    // [L][P][W]
  __host__ __device__ int xds() const { return xs() + L * kP * W; }
  __host__ __device__ int ss() const { return xds() + L * kP * W; }
  __host__ __device__ int zds() const { return ss() + L * kP * W; }
  __host__ __device__ int hb() const { return zds() + L * kP * W; }       // [P][W]
  __host__ __device__ int hdb() const { return hb() + kP * W; }
  __host__ __device__ int zb() const { return hdb() + kP * W; }
  __host__ __device__ int zdb() const { return zb() + kP * W; }
  __host__ __device__ int pb() const { return zdb() + kP * W; }           // [P][4]
  __host__ __device__ int av() const { return pb() + 4 * kP; }            // [P] a, [P][4] v
  __host__ __device__ int gw(int64_t) const { return av() + 5 * kP; }     // [n_params]
  __host__ __device__ int64_t total(int64_t n_params) const { return gw(0) + n_params; }
};

__global__ void __launch_bounds__(kThreads) backward_kernel(const BwdParams prm) {
  extern __shared__ float4 smem4[];
  float *sm = reinterpret_cast<float *>(smem4);
  const int W = prm.W, L = prm.L, skip = prm.skip;
  const BwdLayout lay{W, L};
  float *Wt = sm + lay.wt();
  float *X = sm + lay.xs(), *XD = sm + lay.xds(), *S = sm + lay.ss(), *ZD = sm + lay.zds();
  float *HB = sm + lay.hb(), *HDB = sm + lay.hdb(), *ZB = sm + lay.zb(), *ZDB = sm + lay.zdb();
  float *PB = sm + lay.pb(), *AV = sm + lay.av();
  float *GW = sm + lay.gw(prm.n_params);
  const int tid = threadIdx.x;
  const int nshort = W - 3;
  const float beta = prm.beta;

  // weights of layers 1..L-1, transposed ([k][n]), and a zeroed gradient accumulator
  for (int64_t i = tid; i < (int64_t)(L - 1) * W * W; i += kThreads) Wt[i] = prm.fwd_t[i];
  for (int64_t i = tid; i < prm.n_params; i += kThreads) GW[i] = 0.0f;
  __syncthreads();

  const int64_t ntiles = (prm.n + kP - 1) / kP;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * kP;
    // ---- inputs: x_0 = p, xd_0 = v, a ----
    if (tid < kP) {
      const int64_t i = base + tid;
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
      float a = 0.f;
      if (i < prm.n) {
        p = prm.pts[i];
        a = prm.a[i];
        if (prm.v) v = prm.v[i];
      }
      float *x0 = X + tid * W, *xd0 = XD + tid * W;
      x0[0] = p.x; x0[1] = p.y; x0[2] = p.z;
      xd0[0] = v.x; xd0[1] = v.y; xd0[2] = v.z;
      AV[tid] = a;
      float *vv = AV + kP + 4 * tid;
      vv[0] = v.x; vv[1] = v.y; vv[2] = v.z;
      float *pb = PB + 4 * tid;
      pb[0] = pb[1] = pb[2] = pb[3] = 0.f;
    }
    __syncthreads();

    // ---- forward, primal and tangent ----
    for (int l = 0; l < L; ++l) {
      const int K = (l == 0) ? 3 : W;
      const float *xl = X + (size_t)l * kP * W, *xdl = XD + (size_t)l * kP * W;
      const float *b = prm.bias + (size_t)l * W;
      for (int idx = tid; idx < kP * W; idx += kThreads) {
        const int p = idx / W, c = idx % W;
        float z = __ldg(b + c), zd = 0.f;
        if (l == 0) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float w = __ldg(prm.w0 + 3 * c + k);
            z = fmaf(w, xl[p * W + k], z);
            zd = fmaf(w, xdl[p * W + k], zd);
          }
        } else {
          const float *wt = Wt + (size_t)(l - 1) * W * W;
          for (int k = 0; k < K; ++k) {
            const float w = wt[k * W + c];
            z = fmaf(w, xl[p * W + k], z);
            zd = fmaf(w, xdl[p * W + k], zd);
          }
        }
        float h, s;
        sp_and_slope(z, beta, h, s);
        const float hd = s * zd;
        S[(size_t)l * kP * W + idx] = s;
        ZD[(size_t)l * kP * W + idx] = zd;
        if (l + 1 < L) {
          float xn = h, xdn = hd;
          if (l + 1 == skip) {
            if (c < nshort) {
              xn = h * kInvSqrt2;
              xdn = hd * kInvSqrt2;
            } else {
              const int j = c - nshort;
              xn = X[p * W + j] * kInvSqrt2;             // p_j (layer-0 input)
              xdn = AV[kP + 4 * p + j] * kInvSqrt2;      // v_j
            }
          }
          X[(size_t)(l + 1) * kP * W + idx] = xn;
          XD[(size_t)(l + 1) * kP * W + idx] = xdn;
        } else {
          HB[idx] = h;      // last hidden layer: keep h, hd for the output-layer gradient
          HDB[idx] = hd;
        }
      }
      __syncthreads();
    }

    // ---- output layer: f = w_out . h + b_out; seeds of the reverse pass ----
    {
      const int64_t wo = prm.woff[L], bo = prm.boff[L];
      for (int c = tid; c < W; c += kThreads) {
        float acc = 0.f;
        for (int p = 0; p < kP; ++p) acc += AV[p] * HB[p * W + c] + HDB[p * W + c];
        GW[wo + c] += acc;
      }
      if (tid == 0) {
        float acc = 0.f;
        for (int p = 0; p < kP; ++p) acc += AV[p];
        GW[bo] += acc;
      }
      __syncthreads();
      for (int idx = tid; idx < kP * W; idx += kThreads) {
        const int p = idx / W, c = idx % W;
        const float w = __ldg(prm.wout + c);
        HB[idx] = AV[p] * w;
        HDB[idx] = w;
      }
      __syncthreads();
    }

    // ---- reverse over both streams ----
    for (int l = L - 1; l >= 0; --l) {
      const int K = (l == 0) ? 3 : W;
      const int outl = prm.out[l];
      const float *xl = X + (size_t)l * kP * W, *xdl = XD + (size_t)l * kP * W;
      const float *sl = S + (size_t)l * kP * W, *zdl = ZD + (size_t)l * kP * W;
      for (int idx = tid; idx < kP * W; idx += kThreads) {
        const int c = idx % W;
        const float s = sl[idx], hdb = HDB[idx];
        const float zdb = s * hdb;
        float zb = fmaf(s, HB[idx], zdl[idx] * hdb * beta * s * (1.0f - s));
        ZB[idx] = c < outl ? zb : 0.f;
        ZDB[idx] = c < outl ? zdb : 0.f;
      }
      __syncthreads();
      // weight and bias gradients of layer l (blob layout, unpadded)
      const int64_t wo = prm.woff[l], bo = prm.boff[l];
      for (int idx = tid; idx < outl * K; idx += kThreads) {
        const int c = idx / K, k = idx % K;
        float acc = 0.f;
        for (int p = 0; p < kP; ++p)
          acc += ZB[p * W + c] * xl[p * W + k] + ZDB[p * W + c] * xdl[p * W + k];
        GW[wo + idx] += acc;
      }
      for (int c = tid; c < outl; c += kThreads) {
        float acc = 0.f;
        for (int p = 0; p < kP; ++p) acc += ZB[p * W + c];
        GW[bo + c] += acc;
      }
      // gradients with respect to this layer's inputs
      for (int idx = tid; idx < kP * K; idx += kThreads) {
        const int p = idx / K, k = idx % K;
        float xb = 0.f, xdb = 0.f;
        if (l == 0) {
          for (int c = 0; c < W; ++c) {
            const float w = __ldg(prm.w0 + 3 * c + k);
            xb = fmaf(ZB[p * W + c], w, xb);
          }
          PB[4 * p + k] += xb;
        } else {
          const float *wl = prm.bwd + (size_t)(l - 1) * W * W;    // [n][k] = W_l[n][k]
          for (int c = 0; c < W; ++c) {
            const float w = __ldg(wl + (size_t)c * W + k);
            xb = fmaf(ZB[p * W + c], w, xb);
            xdb = fmaf(ZDB[p * W + c], w, xdb);
          }
          if (l == skip) {
            xb *= kInvSqrt2;
            xdb *= kInvSqrt2;
            if (k >= nshort) {
              PB[4 * p + (k - nshort)] += xb;       // direct path of the skip input
              xb = 0.f;
              xdb = 0.f;
            }
          }
          HB[p * W + k] = xb;
          HDB[p * W + k] = xdb;
        }
      }
      __syncthreads();
    }

    if (prm.g_pts && tid < kP) {
      const int64_t i = base + tid;
      if (i < prm.n) prm.g_pts[i] = make_float4(PB[4 * tid], PB[4 * tid + 1], PB[4 * tid + 2], 0.f);
    }
    __syncthreads();
  }
  if (prm.g_partial) {
    float *dst = prm.g_partial + (size_t)blockIdx.x * prm.n_params;
    for (int64_t i = tid; i < prm.n_params; i += kThreads) dst[i] = GW[i];
  }
}

// g[i] = sum over CTAs b (in order) of partial[b][i].
__global__ void reduce_partials_kernel(const float *__restrict__ partial, int blocks, int64_t n,
                                       float *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int b = 0; b < blocks; ++b) acc += partial[(size_t)b * n + i];
    out[i] = acc;
  }
}

}  // namespace

size_t backward_smem_bytes(int width, int n_hidden, int64_t n_params) {
  const BwdLayout lay{width, n_hidden};
  return sizeof(float) * (size_t)lay.total(n_params);
}

bool backward_supported(int width, int n_hidden, int64_t n_params) {
  return n_hidden <= kMaxL && width <= 128 &&
         backward_smem_bytes(width, n_hidden, n_params) <= 227 * 1024;
}

cudaError_t launch_backward(const float4 *pts, int64_t n, const float *a, const float4 *v,
                            float *g_partial, int grid, float4 *g_pts, float *g_weights,
                            const NetDevice &net, int width, int n_hidden, int skip, float beta,
                            const int64_t *woff, const int64_t *boff, const int *out,
                            int64_t n_params, cudaStream_t s) {
  BwdParams p{};
  p.pts = pts; p.n = n; p.a = a; p.v = v; p.g_partial = g_weights ? g_partial : nullptr;
  p.g_pts = g_pts;
  p.w0 = net.w0; p.bias = net.bias; p.fwd_t = net.fwd_t; p.bwd = net.bwd; p.wout = net.wout;
  p.bout = net.bout;
  p.W = width; p.L = n_hidden; p.skip = skip; p.beta = beta; p.n_params = n_params;
  for (int l = 0; l <= n_hidden; ++l) {
    p.woff[l] = woff[l];
    p.boff[l] = boff[l];
    p.out[l] = out[l];
  }
  const size_t smem = backward_smem_bytes(width, n_hidden, n_params);
  cudaError_t e = cudaFuncSetAttribute(backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  backward_kernel<<<grid, kThreads, smem, s>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess || !g_weights) return e;
  reduce_partials_kernel<<<(int)((n_params + 255) / 256 < 1024 ? (n_params + 255) / 256 : 1024), 256,
                           0, s>>>(g_partial, grid, n_params, g_weights);
  return cudaGetLastError();
}

int backward_grid(int64_t n, int num_sms) {
  const int64_t tiles = (n + kP - 1) / kP;
  return (int)(tiles < num_sms ? (tiles < 1 ? 1 : tiles) : num_sms);
}

}  // namespace nsdf
