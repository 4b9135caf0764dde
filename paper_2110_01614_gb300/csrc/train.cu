// Gradient of the L1 fitting loss of Sec. 3.1 for 16-bit (tensor-core)
// contexts: L = (1/n) sum_i |f(p_i) - d_i| over training points p_i with
// exact signed distances d_i.
//
// With a_i = sign(f_i - d_i) (0 at equality) and delta_l(i) = d f(p_i) / d z_l
// (the quantities the query's Jacobian-transpose chain already forms), the
// gradient of every layer is a sum over the points:
//   dL/dW_l = (1/n) sum_i a_i delta_l(i) x_l(i)^T,   dL/db_l = (1/n) sum_i a_i delta_l(i),
// x_l the layer's input.  The training form of the tensor-core kernel writes
// every layer's A operand out (h_l on the forward pass, delta_l on the
// reverse pass, 16-bit, one row per point); the rows of delta are then
// multiplied by a_i (a sign flip or a zero: exact in 16 bits), the
// hidden-layer weight gradients are contractions over the points on the
// tensor cores (wgrad_tc.cu: tcgen05, FP32 accumulation in TMEM, split over
// the points and reduced in a fixed order), and the remaining sums (biases, W_0 on p, the skip layer's
// columns on p / sqrt(2), w_out and b_out) are FP32 per-block partial sums
// reduced in block order, so the result does not depend on scheduling.
//
// Fourier-feature ReLU networks (Sec. 4.3) take the same route with their own
// tensor-core kernel: layer 0 is a 256 x 256 product too, its input (the
// features, saved in the kernel's permuted column order) gets its own GEMM,
// whose columns are put back in feature order; the frequencies B are not
// trained (random Fourier features) and get a zero gradient.

#include <cmath>
#include <new>

#include "nsdf_internal.h"

namespace nsdf {

namespace {

constexpr int kRowsPerBlock = 1024;   // points per block of the small sums
constexpr float kInvSqrt2 = 0.70710678118654752f;

// Blob offsets of every layer (the layout of nsdf_num_params).
struct BlobPlan {
  int L, W, skip;
  int ff;                       // Fourier frequencies m (0: none)
  int64_t woff[66], boff[66];   // layers 0..L, then woff[L+1] = the blob size
  int out[66];
};

// a_i = sign(f_i - d_i) for i < n, 0 for the padding rows; per-block sums of
// |f_i - d_i| (reduced in order by l1_loss_kernel).
__global__ void l1_sign_kernel(const float4 *__restrict__ ns, const float *__restrict__ d,
                               int64_t n, int64_t n_pad, float *__restrict__ a,
                               float *__restrict__ loss_part) {
  __shared__ float red[32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < n_pad) {
    float s = 0.f;
    if (i < n) {
      const float r = ns[i].w - d[i];
      s = r > 0.f ? 1.f : (r < 0.f ? -1.f : 0.f);
      l = fabsf(r);
    }
    a[i] = s;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    loss_part[blockIdx.x] = t;
  }
}

__global__ void l1_loss_kernel(const float *__restrict__ loss_part, int nb, int64_t n,
                               float *__restrict__ loss) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += loss_part[b];
  *loss = (float)(t / (double)n);
}

// delta rows times a_i: flip the sign bit of every 16-bit value, or zero it
// (16 bytes = 8 values per access).
__global__ void scale_rows_kernel(uint4 *__restrict__ d, int64_t vecs, int64_t n_pad, int W,
                                  const float *__restrict__ a) {
  const int64_t per_row = W / 8;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < vecs;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float s = a[(t / per_row) % n_pad];
    if (s > 0.f) continue;
    uint4 v = d[t];
    if (s == 0.f) {
      v = make_uint4(0u, 0u, 0u, 0u);
    } else {
      v.x ^= 0x80008000u;
      v.y ^= 0x80008000u;
      v.z ^= 0x80008000u;
      v.w ^= 0x80008000u;
    }
    d[t] = v;
  }
}

__device__ __forceinline__ float2 unpack16(uint32_t w, int fp16) {
  if (fp16) return __half22float2(*reinterpret_cast<const __half2 *>(&w));
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
}

// Per-block partial sums over kRowsPerBlock points, for job j = blockIdx.y:
//   j <  L : sum_i delta_j(i)[c]                         (bias of layer j)
//   j == L : sum_i delta_0(i)[c] p_i[k], k = 0..2         (W_0; not for ff)
//   j == L+1: sum_i delta_s(i)[c] p_i[k] / sqrt(2)        (skip layer s, its p columns)
//   j == L+2: sum_i a_i h_{L-1}(i)[c]; and sum_i a_i      (w_out, b_out)
// Thread t covers columns 8t .. 8t+7 (one 16-byte load per row); part[j][block][c][3].
__global__ void small_partials_kernel(const uint16_t *__restrict__ save_h,
                                      const uint16_t *__restrict__ save_d,
                                      const float4 *__restrict__ pts, const float *__restrict__ a,
                                      int L, int W, int skip, int ff, int64_t n, int64_t n_pad,
                                      int fp16, float *__restrict__ part) {
  const int j = blockIdx.y;
  const int c = 8 * threadIdx.x;
  if (c >= W) return;
  const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
  int64_t r1 = r0 + kRowsPerBlock;
  if (r1 > n_pad) r1 = n_pad;
  const uint16_t *src = nullptr;
  if (j < L) src = save_d + (size_t)j * n_pad * W;
  else if (j == L) src = ff ? nullptr : save_d;
  else if (j == L + 1) src = skip > 0 ? save_d + (size_t)skip * n_pad * W : nullptr;
  else src = save_h + (size_t)(L - 1) * n_pad * W;
  float acc[8][3];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u][0] = acc[u][1] = acc[u][2] = 0.f;
  float asum = 0.f;
  if (src) {
    // four rows' loads in flight per thread (r1 - r0 is a multiple of 128;
    // four measured faster than one or eight);
    // the sums still run in row order
    for (int64_t r4 = r0; r4 < r1; r4 += 4) {
      uint4 wq[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) wq[i] = *reinterpret_cast<const uint4 *>(src + (size_t)(r4 + i) * W + c);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t r = r4 + i;
        const uint32_t ww[4] = {wq[i].x, wq[i].y, wq[i].z, wq[i].w};
        float v[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 f2 = unpack16(ww[u], fp16);
          v[2 * u] = f2.x;
          v[2 * u + 1] = f2.y;
        }
        if (j < L) {
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u][0] += v[u];
        } else if (j <= L + 1) {
          float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
          if (r < n) p = pts[r];
          const float sc = j == L ? 1.f : kInvSqrt2;
          const float q[3] = {p.x * sc, p.y * sc, p.z * sc};
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[u][k] = fmaf(v[u], q[k], acc[u][k]);
        } else {
          const float s = a[r];
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u][0] = fmaf(s, v[u], acc[u][0]);
          asum += s;
        }
      }
    }
  }
  float *o = part + (((size_t)j * gridDim.x + blockIdx.x) * W + c) * 3;
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int k = 0; k < 3; ++k) o[3 * u + k] = acc[u][k];
  if (j == L + 2 && threadIdx.x == 0) o[2] = asum;   // column 0, slot 2: sum a_i
}

// small[j][c][k] = sum over blocks, in block order.
__global__ void small_reduce_kernel(const float *__restrict__ part, int jobs, int nb, int W,
                                    float *__restrict__ small) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per_job = (int64_t)W * 3;
  if (t >= (int64_t)jobs * per_job) return;
  const int j = (int)(t / per_job);
  const int64_t e = t % per_job;
  float s = 0.f;
  for (int b = 0; b < nb; ++b) s += part[((size_t)j * nb + b) * per_job + e];
  small[t] = s;
}

// The gradient in blob layout, times 1/n.
__global__ void scatter_grad_kernel(const float *__restrict__ G, const float *__restrict__ small,
                                    BlobPlan plan, int64_t total, float inv_n,
                                    float *__restrict__ g) {
  const int L = plan.L, W = plan.W;
  const int64_t per_job = (int64_t)W * 3;
  auto sm = [&](int j, int c, int k) { return small[j * per_job + (int64_t)c * 3 + k]; };
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < plan.woff[0]) {                       // the frequencies B: not trained
      g[t] = 0.f;
      continue;
    }
    int l = 0;
    while (l < L && t >= plan.woff[l + 1]) ++l;   // layer of element t
    float v;
    if (t >= plan.boff[l]) {                      // bias
      const int nn = (int)(t - plan.boff[l]);
      v = l < L ? sm(l, nn, 0) : sm(L + 2, 0, 2);
    } else {
      const int64_t e = t - plan.woff[l];
      if (plan.ff > 0 && l < L) {
        // G_l[n][c] for every layer; layer 0's columns are in the kernel's
        // feature order: feature k = s m + 64 g + i sits in column 128 g + 64 s + i
        const int nn = (int)(e / W), k = (int)(e % W);
        int c = k;
        if (l == 0) {
          const int sgn = k / plan.ff, j = k % plan.ff;
          c = 128 * (j / 64) + 64 * sgn + (j % 64);
        }
        v = G[((size_t)l * W + nn) * W + c];
      } else if (l == 0) {
        v = sm(L, (int)(e / 3), (int)(e % 3));
      } else if (l == L) {
        v = sm(L + 2, (int)e, 0);
      } else {
        const int nn = (int)(e / W), k = (int)(e % W);
        v = (l == plan.skip && k >= W - 3) ? sm(L + 1, nn, k - (W - 3))
                                           : G[((size_t)(l - 1) * W + nn) * W + k];
      }
    }
    g[t] = v * inv_n;
  }
}

struct TrainState {
  int64_t cap = 0;   // rows the buffers hold (a multiple of 128)
  uint16_t *save_h = nullptr, *save_d = nullptr;
  float4 *ns = nullptr;
  float *a = nullptr, *loss_part = nullptr, *part = nullptr, *small = nullptr, *G = nullptr,
        *loss_tmp = nullptr;
  float *ws = nullptr;   // split partials of the weight-gradient products
  int64_t part_floats = 0;
};

void free_all(TrainState *t) {
  cudaFree(t->save_h);
  cudaFree(t->save_d);
  cudaFree(t->ns);
  cudaFree(t->a);
  cudaFree(t->loss_part);
  cudaFree(t->part);
  cudaFree(t->small);
  cudaFree(t->G);
  cudaFree(t->loss_tmp);
  cudaFree(t->ws);
  t->save_h = t->save_d = nullptr;
  t->ns = nullptr;
  t->a = t->loss_part = t->part = t->small = t->G = t->loss_tmp = t->ws = nullptr;
  t->cap = 0;
}

template <typename T>
bool dalloc(T **p, size_t count) {
  void *q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *p = static_cast<T *>(q);
  return true;
}

}  // namespace

void train_state_free(void *p) {
  if (!p) return;
  TrainState *t = static_cast<TrainState *>(p);
  free_all(t);
  delete t;
}

}  // namespace nsdf

using namespace nsdf;

extern "C" nsdf_status nsdf_l1_grad(nsdf_ctx *ctx, const float *pts, int64_t n, const float *targets,
                                    float *g_weights, float *loss, nsdf_stream stream) {
  if (!ctx || n < 0 || !g_weights) return NSDF_ERR_INVALID_ARG;
  QueryParams p{};
  int num_sms = 0, W = 0, L = 0;
  bool tc16 = false, fp16 = false;
  const NetDevice *net = nullptr;
  nsdf_status st = ctx_query_setup(ctx, &p, &num_sms, &W, &L, &tc16, &fp16, &net);
  if (st != NSDF_OK) return st;
  if (!tc16 || !wgrad_supported(W)) return NSDF_ERR_UNSUPPORTED;   // FP32 contexts: nsdf_backward
  const bool ff = p.ff > 0;                  // the Fourier-feature ReLU kernel
  if (n == 0) return NSDF_ERR_INVALID_ARG;
  if (!pts || !targets) return NSDF_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(pts) & 15u) || (reinterpret_cast<uintptr_t>(g_weights) & 3u) ||
      (reinterpret_cast<uintptr_t>(targets) & 3u))
    return NSDF_ERR_MISALIGNED;
  if (!device_memory(pts) || !device_memory(targets) || !device_memory(g_weights) ||
      (loss && !device_memory(loss)))
    return NSDF_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void **slot = ctx_train_slot(ctx);
  if (!*slot) *slot = new (std::nothrow) TrainState;
  TrainState *t = static_cast<TrainState *>(*slot);
  if (!t) return NSDF_ERR_OOM;
  const int64_t n_pad = (n + 127) / 128 * 128;
  const int nb = (int)((n_pad + kRowsPerBlock - 1) / kRowsPerBlock);
  const int jobs = L + 3;
  if (n_pad > t->cap) {
    cudaStreamSynchronize(s);
    free_all(t);
    const size_t rows = (size_t)n_pad;
    // ff: h_0 .. h_{L-1} and the features (slot L); G for every layer
    const size_t hslots = ff ? (size_t)L + 1 : (size_t)L;
    const size_t gslots = ff ? (size_t)L : (size_t)(L > 1 ? L - 1 : 1);
    const int S = wgrad_splits(W, (int)gslots, n_pad, num_sms);
    bool ok = dalloc(&t->save_h, hslots * rows * W) && dalloc(&t->save_d, (size_t)L * rows * W) &&
              dalloc(&t->ns, rows) && dalloc(&t->a, rows) &&
              dalloc(&t->loss_part, (rows + 255) / 256) &&
              dalloc(&t->part, (size_t)jobs * nb * W * 3) && dalloc(&t->small, (size_t)jobs * W * 3) &&
              dalloc(&t->G, gslots * W * W) && dalloc(&t->loss_tmp, 1) &&
              dalloc(&t->ws, gslots * (size_t)S * W * W);
    if (!ok) {
      free_all(t);
      return NSDF_ERR_OOM;
    }
    t->cap = n_pad;
  }
  // 1. the training form of the query: f per point, every A operand saved
  p.pts = reinterpret_cast<const float4 *>(pts);
  p.n = n;
  p.collide = 0;
  p.out_n_sdf = t->ns;
  p.save_h = t->save_h;
  p.save_d = t->save_d;
  st = ctx_query_scratch(ctx, n, &p);
  if (st != NSDF_OK) return st;
  cudaError_t e = ff ? launch_query_tc16_ff(p, *net, fp16, num_sms, s)
                     : launch_query_tc16_net(p, *net, fp16, num_sms, s);
  if (e != cudaSuccess) return NSDF_ERR_CUDA;
  // 2. a_i and the loss; delta rows times a_i
  const int lb = (int)((n_pad + 255) / 256);
  l1_sign_kernel<<<lb, 256, 0, s>>>(t->ns, targets, n, n_pad, t->a, t->loss_part);
  l1_loss_kernel<<<1, 32, 0, s>>>(t->loss_part, lb, n, loss ? loss : t->loss_tmp);
  const int64_t vecs = (int64_t)L * n_pad * W / 8;
  scale_rows_kernel<<<8 * num_sms, 256, 0, s>>>(reinterpret_cast<uint4 *>(t->save_d), vecs, n_pad,
                                                W, t->a);
  // 3. hidden-layer weight gradients on the tensor cores:
  //    G_l[n][k] = sum_i delta_l(i)[n] h_{l-1}(i)[k]
  WgradJob job{};
  job.save_h = t->save_h;
  job.save_d = t->save_d;
  job.h_rows = (int64_t)(ff ? L + 1 : L) * n_pad;
  job.d_rows = (int64_t)L * n_pad;
  job.n_pad = n_pad;
  job.W = W;
  job.layers = 0;
  for (int l = ff ? 0 : 1; l < L; ++l, ++job.layers) {
    // layer l reads h_{l-1} (for ff layer 0: the features, slot L)
    job.hslot[job.layers] = (ff && l == 0) ? L : l - 1;
    job.dslot[job.layers] = l;
    job.gslot[job.layers] = ff ? l : l - 1;
  }
  job.S = wgrad_splits(W, job.layers, n_pad, num_sms);
  job.ws = t->ws;
  job.G = t->G;
  job.err = p.err;
  job.wait_budget = p.wait_budget;
  job.fp16 = fp16;
  job.num_sms = num_sms;
  if (job.layers > 0 && launch_wgrad_tc(job, s) != cudaSuccess) return NSDF_ERR_CUDA;
  // 4. the small sums, reduced in block order
  small_partials_kernel<<<dim3(nb, jobs), W / 8, 0, s>>>(t->save_h, t->save_d, p.pts, t->a, L, W,
                                                         p.skip, p.ff, n, n_pad, fp16 ? 1 : 0,
                                                         t->part);
  const int64_t nsmall = (int64_t)jobs * W * 3;
  small_reduce_kernel<<<(int)((nsmall + 255) / 256), 256, 0, s>>>(t->part, jobs, nb, W, t->small);
  // 5. scatter into the blob layout
  BlobPlan plan{};
  plan.L = L;
  plan.W = W;
  plan.skip = p.skip;
  plan.ff = p.ff;
  const int64_t total = ctx_blob_offsets(ctx, plan.woff, plan.boff, plan.out);
  plan.woff[L + 1] = total;
  scatter_grad_kernel<<<4 * num_sms, 256, 0, s>>>(t->G, t->small, plan, total, 1.0f / (float)n,
                                                  g_weights);
  return cudaGetLastError() == cudaSuccess ? NSDF_OK : NSDF_ERR_CUDA;
}
