// Host runtime and C ABI of the nsdf library (declared in include/nsdf.h).
//
// Owns contexts, converts weight blobs into the kernels' device layouts,
// validates arguments, sizes scratch and launches the kernels on the
// caller's stream.  Host-memory collision calls are streamed through device
// staging buffers in chunks on two internal streams so that copies overlap
// compute.

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "nsdf_internal.h"
#include "nsdf_debug.h"

using namespace nsdf;

namespace {

constexpr int kMaxLayers = 64;

bool arch_valid(const nsdf_arch *a) {
  if (!a) return false;
  if (a->in_dim != 3 || a->width < 4 || a->n_hidden < 1 || a->n_hidden > kMaxLayers - 1) return false;
  if (!(a->beta > 0.0f) || !std::isfinite(a->beta)) return false;
  if (a->skip_layer != -1 && (a->skip_layer < 1 || a->skip_layer >= a->n_hidden)) return false;
  if (a->activation != NSDF_ACT_SOFTPLUS && a->activation != NSDF_ACT_RELU) return false;
  if (a->ff_freqs < 0) return false;
  if (a->ff_freqs > 0 && (2 * a->ff_freqs != a->width || a->skip_layer != -1)) return false;
  return true;
}

int layer_out(const nsdf_arch &a, int l) {
  if (l == a.n_hidden) return 1;
  if (a.skip_layer > 0 && l == a.skip_layer - 1) return a.width - a.in_dim;
  return a.width;
}
int layer_in(const nsdf_arch &a, int l) {
  if (l > 0) return a.width;
  return a.ff_freqs > 0 ? 2 * a.ff_freqs : a.in_dim;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// 0: device (or managed), 1: host (pinned or pageable, or unknown to CUDA)
int pointer_kind(const void *p) { return device_memory(p) ? 0 : 1; }

bool invert4x4(const double *m, double *inv) {
  double a[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 8; ++c) a[r][c] = c < 4 ? m[r * 4 + c] : (c - 4 == r ? 1.0 : 0.0);
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
    if (std::fabs(a[piv][c]) < 1e-300) return false;
    if (piv != c)
      for (int k = 0; k < 8; ++k) std::swap(a[c][k], a[piv][k]);
    const double d = a[c][c];
    for (int k = 0; k < 8; ++k) a[c][k] /= d;
    for (int r = 0; r < 4; ++r)
      if (r != c) {
        const double f = a[r][c];
        for (int k = 0; k < 8; ++k) a[r][k] -= f * a[c][k];
      }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) inv[r * 4 + c] = a[r][c + 4];
  return true;
}

struct PackPlan {
  int width, n_hidden, skip;
  int ff;   // m, frequencies [m][3] at the start of the blob
  int64_t woff[kMaxLayers];
  int64_t boff[kMaxLayers];
  int out[kMaxLayers];
};

struct PackTargets {
  float *w0, *bias, *fwd_t, *bwd, *wout, *bout;
  float *ffB, *ff0_t, *ff0;
  uint16_t *fwd16, *bwd16;
  int fp16;   // 16-bit copies as FP16 (1) or BF16 (0)
  uint16_t *fwd16_lo;   // nullable: BF16 residual W - bf16(W) of the hidden layers
};

__device__ __forceinline__ uint16_t to16(float v, int fp16) {
  if (fp16) {
    __half h = __float2half_rn(v);
    return *reinterpret_cast<uint16_t *>(&h);
  }
  __nv_bfloat16 b = __float2bfloat16_rn(v);
  return *reinterpret_cast<uint16_t *>(&b);
}

// Converts the packed FP32 blob into every device layout the kernels read.
__global__ void pack_weights_kernel(const float *__restrict__ blob, PackPlan plan, PackTargets net) {
  const int W = plan.width, L = plan.n_hidden;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // L0 weights and all hidden biases, output layer
  if (plan.ff > 0) {
    // B, then L0 (width x 2m = width x width) as two panels
    for (int64_t t = t0; t < (int64_t)plan.ff * 3; t += stride) net.ffB[t] = blob[t];
    const float *W0 = blob + plan.woff[0];
    for (int64_t t = t0; t < (int64_t)W * W; t += stride) {
      const int r = (int)(t / W), c = (int)(t % W);
      net.ff0_t[t] = W0[(int64_t)c * W + r];   // [k=r][n=c] = W_0[n][k]
      net.ff0[t] = W0[t];                      // [n=r][k=c] = W_0[n][k]
      if (net.fwd16) {
        // slot 0 of the 16-bit copies, feature columns / rows permuted
        net.fwd16[t] = to16(W0[(int64_t)r * W + ff_feature_of_column(c, plan.ff)], net.fp16);
        net.bwd16[t] = to16(W0[(int64_t)c * W + ff_feature_of_column(r, plan.ff)], net.fp16);
      }
    }
  } else {
    for (int64_t t = t0; t < (int64_t)W * 3; t += stride) {
      const int n = (int)(t / 3), k = (int)(t % 3);
      net.w0[t] = n < plan.out[0] ? blob[plan.woff[0] + (int64_t)n * 3 + k] : 0.0f;
    }
  }
  for (int64_t t = t0; t < (int64_t)L * W; t += stride) {
    const int l = (int)(t / W), n = (int)(t % W);
    net.bias[t] = n < plan.out[l] ? blob[plan.boff[l] + n] : 0.0f;
  }
  for (int64_t t = t0; t < W; t += stride) net.wout[t] = blob[plan.woff[L] + t];
  if (t0 == 0) net.bout[0] = blob[plan.boff[L]];
  // hidden layers l = 1 .. L-1, padded to W x W
  const int64_t per = (int64_t)W * W;
  for (int64_t t = t0; t < (int64_t)(L - 1) * per; t += stride) {
    const int l = 1 + (int)(t / per);
    const int64_t e = t % per;
    const int r = (int)(e / W), c = (int)(e % W);
    const float *Wl = blob + plan.woff[l];          // [out_l x W] row-major
    // row-major [r][c] element of each layout
    const float w_rc = r < plan.out[l] ? Wl[(int64_t)r * W + c] : 0.0f;   // W_l[r][c]
    const float w_cr = c < plan.out[l] ? Wl[(int64_t)c * W + r] : 0.0f;   // W_l[c][r]
    const int64_t o = (int64_t)(l - 1) * per + e;
    net.fwd_t[o] = w_cr;   // [k=r][n=c] = W_l[n][k]
    net.bwd[o] = w_rc;     // [n=r][k=c] = W_l[n][k]
    if (net.fwd16) {
      // Fourier-feature nets keep layer 0 in slot 0 of the 16-bit copies
      const int64_t o16 = plan.ff > 0 ? o + per : o;
      net.fwd16[o16] = to16(w_rc, net.fp16);   // [n=r][k=c]
      net.bwd16[o16] = to16(w_cr, net.fp16);   // [k=r][n=c]
      if (net.fwd16_lo) {
        const uint16_t hi = to16(w_rc, 0);
        net.fwd16_lo[o16] = to16(w_rc - __uint_as_float((uint32_t)hi << 16), 0);
      }
    }
  }
}

cudaError_t last_err() { return cudaGetLastError(); }

}  // namespace

struct nsdf_ctx {
  nsdf_arch arch{};
  nsdf_precision prec = NSDF_FP32;
  int n_nets = 0;
  int device = 0;
  int num_sms = 0;
  std::vector<NetDevice> nets;
  std::vector<void *> allocations;
  float *scratch = nullptr;     // per-CTA slope slabs of the query kernels
  size_t scratch_bytes = 0;
  int *d_err = nullptr;         // device error word
  float *bwd_partial = nullptr; // per-CTA weight-gradient partial sums of nsdf_backward
  size_t bwd_partial_bytes = 0;
  // host-buffer pipeline
  cudaStream_t pipe[2] = {nullptr, nullptr};
  cudaEvent_t ev_start = nullptr, ev_done[2] = {nullptr, nullptr};
  float *stage = nullptr;       // 2 x chunk x (4 + 4 + 4 floats) + 2 x chunk bytes
  float *pipe_scratch[2] = {nullptr, nullptr};
  size_t pipe_scratch_bytes = 0;
  int64_t chunk = 0;
  // bounded waits and test-only fault injection (see include/nsdf_debug.h)
  long long wait_budget = 4000000000LL;   // ~2 s of SM clock per mbarrier wait
  int drop_load = -1;
  // grouped launches: device table of per-network pointers, work list, tuned shape
  NetPtrs *d_netptrs = nullptr;
  int32_t *d_tile_start = nullptr;
  float *d_body = nullptr;     // [n_nets][kBodyFloats] poses of nsdf_query_grouped_T
  void *train = nullptr;       // buffers of nsdf_l1_grad (train.cu)
  int grouped_pt = 8;          // points per thread of the FP32 tile (4 or 8)
  int grouped_cps = 0;         // CTAs per SM (0: as many as fit)
};

namespace {

nsdf_status map_err(cudaError_t e) {
  if (e == cudaSuccess) return NSDF_OK;
  if (e == cudaErrorMemoryAllocation) return NSDF_ERR_OOM;
  return NSDF_ERR_CUDA;
}

template <typename T>
nsdf_status ctx_alloc(nsdf_ctx *ctx, T **p, size_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return NSDF_ERR_OOM;
  }
  ctx->allocations.push_back(q);
  *p = static_cast<T *>(q);
  return NSDF_OK;
}

// BF16 and FP16 contexts share the 16-bit tensor-core kernel.
bool use_bf16(const nsdf_ctx *ctx) { return ctx->prec == NSDF_BF16 || ctx->prec == NSDF_FP16; }

// 16-bit Fourier-feature ReLU contexts run query_tc16_ff.cu.
bool use_tc16_ff(const nsdf_ctx *ctx) { return use_bf16(ctx) && ctx->arch.ff_freqs > 0; }

// 16-bit width-64 softplus contexts run query_tc16_w64.cu (no scratch).
bool use_w64(const nsdf_ctx *ctx) {
  return use_bf16(ctx) && ctx->arch.ff_freqs == 0 && ctx->arch.width == 64;
}

int query_grid(const nsdf_ctx *ctx, int64_t n) {
  if (use_w64(ctx)) return ctx->num_sms;
  if (use_tc16_ff(ctx)) return query_tc16_ff_grid(n, ctx->num_sms);
  if (use_bf16(ctx)) return query_tc16_grid(ctx->arch.width, n, ctx->num_sms);
  return query_fp32_grid(ctx->arch.width, n, ctx->num_sms, ctx->arch.ff_freqs > 0);
}

size_t query_scratch(const nsdf_ctx *ctx, int grid) {
  if (use_w64(ctx)) return 0;
  if (use_tc16_ff(ctx)) return query_tc16_ff_scratch_bytes(grid);
  if (use_bf16(ctx))
    return query_tc16_scratch_bytes(ctx->arch.width, ctx->arch.n_hidden, grid, ctx->prec == NSDF_FP16);
  return query_fp32_scratch_bytes(ctx->arch.width, ctx->arch.n_hidden, grid);
}

nsdf_status ensure_scratch(nsdf_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->scratch_bytes) return NSDF_OK;
  if (ctx->scratch) cudaFree(ctx->scratch);
  ctx->scratch = nullptr;
  ctx->scratch_bytes = 0;
  void *q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    return NSDF_ERR_OOM;
  }
  ctx->scratch = static_cast<float *>(q);
  ctx->scratch_bytes = bytes;
  return NSDF_OK;
}

void fill_net(const nsdf_ctx *ctx, int net, QueryParams &p) {
  const NetDevice &d = ctx->nets[net];
  p.w0 = d.w0; p.bias = d.bias; p.fwd_t = d.fwd_t; p.bwd = d.bwd; p.wout = d.wout; p.bout = d.bout;
  p.fwd16 = d.fwd16; p.bwd16 = d.bwd16; p.fwd16_lo = d.fwd16_lo;
  p.ffB = d.ffB; p.ff0_t = d.ff0_t; p.ff0 = d.ff0;
  p.width = ctx->arch.width;
  p.n_hidden = ctx->arch.n_hidden;
  p.skip = ctx->arch.skip_layer;
  p.beta = ctx->arch.beta;
  p.relu = ctx->arch.activation == NSDF_ACT_RELU ? 1 : 0;
  p.ff = ctx->arch.ff_freqs;
  p.err = ctx->d_err;
  p.wait_budget = ctx->wait_budget;
  p.drop_load = ctx->drop_load;
}

cudaError_t launch_query(const nsdf_ctx *ctx, int net, const QueryParams &p, cudaStream_t s) {
  if (use_w64(ctx)) return launch_query_w64(p, ctx->prec == NSDF_FP16, ctx->num_sms, 0, s);
  if (use_tc16_ff(ctx))
    return launch_query_tc16_ff(p, ctx->nets[net], ctx->prec == NSDF_FP16, ctx->num_sms, s);
  if (use_bf16(ctx))
    return launch_query_tc16_net(p, ctx->nets[net], ctx->prec == NSDF_FP16, ctx->num_sms, s);
  return launch_query_fp32(p, ctx->num_sms, s);
}

nsdf_status set_transform(const float *T, QueryParams &p) {
  p.has_T = 0;
  if (!T) return NSDF_OK;
  double m[16], inv[16];
  for (int i = 0; i < 16; ++i) m[i] = T[i];
  if (!invert4x4(m, inv)) return NSDF_ERR_INVALID_ARG;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c) p.Ti[r * 4 + c] = (float)inv[r * 4 + c];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) p.R[r * 3 + c] = T[r * 4 + c];
  p.has_T = 1;
  return NSDF_OK;
}

nsdf_status ensure_pipeline(nsdf_ctx *ctx) {
  if (ctx->stage) return NSDF_OK;
  // about 256K points per chunk; the tensor-core kernels (one 128-point tile
  // per CTA and iteration) get a whole number of grid-wide iterations, so no
  // chunk ends in a partly filled wave of tiles
  int64_t chunk = 1 << 18;
  if (use_bf16(ctx) && !use_w64(ctx)) {
    const int64_t wave = (int64_t)query_grid(ctx, chunk) * 128;
    const int64_t waves = (chunk + wave / 2) / wave;
    chunk = (waves > 0 ? waves : 1) * wave;
  }
  cudaError_t e;
  for (int i = 0; i < 2; ++i) {
    e = cudaStreamCreateWithFlags(&ctx->pipe[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) return map_err(e);
    e = cudaEventCreateWithFlags(&ctx->ev_done[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return map_err(e);
  }
  e = cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming);
  if (e != cudaSuccess) return map_err(e);
  const size_t per = (size_t)chunk * (3 * 16 + 1);
  void *q = nullptr;
  if (cudaMalloc(&q, 2 * per + 64) != cudaSuccess) {
    cudaGetLastError();
    return NSDF_ERR_OOM;
  }
  ctx->stage = static_cast<float *>(q);
  const int grid = query_grid(ctx, chunk);
  const size_t sb = query_scratch(ctx, grid);
  for (int i = 0; i < 2; ++i) {
    if (cudaMalloc(&q, sb) != cudaSuccess) {
      cudaGetLastError();
      return NSDF_ERR_OOM;
    }
    ctx->pipe_scratch[i] = static_cast<float *>(q);
  }
  ctx->pipe_scratch_bytes = sb;
  ctx->chunk = chunk;
  return NSDF_OK;
}

// Collision solve on host buffers: chunks alternate between two streams;
// each chunk is copied in, solved and copied out on its stream.
nsdf_status collide_host(nsdf_ctx *ctx, QueryParams base, const float *pts, int64_t n,
                         float *out_pts, float *out_n_sdf, uint8_t *out_hit, cudaStream_t s) {
  nsdf_status st = ensure_pipeline(ctx);
  if (st != NSDF_OK) return st;
  const int64_t chunk = ctx->chunk;
  cudaError_t e = cudaEventRecord(ctx->ev_start, s);
  if (e != cudaSuccess) return map_err(e);
  for (int i = 0; i < 2; ++i) cudaStreamWaitEvent(ctx->pipe[i], ctx->ev_start, 0);
  const size_t per = (size_t)chunk * (3 * 16 + 1);
  for (int64_t c0 = 0, k = 0; c0 < n; c0 += chunk, ++k) {
    const int b = (int)(k & 1);
    cudaStream_t ps = ctx->pipe[b];
    char *base_b = reinterpret_cast<char *>(ctx->stage) + b * per;
    float4 *d_in = reinterpret_cast<float4 *>(base_b);
    float4 *d_out = d_in + chunk;
    float4 *d_nsdf = d_out + chunk;
    uint8_t *d_hit = reinterpret_cast<uint8_t *>(d_nsdf + chunk);
    const int64_t m = (n - c0 < chunk) ? n - c0 : chunk;
    e = cudaMemcpyAsync(d_in, pts + 4 * c0, (size_t)m * 16, cudaMemcpyHostToDevice, ps);
    if (e != cudaSuccess) return map_err(e);
    QueryParams p = base;
    p.pts = d_in;
    p.n = m;
    p.out_pts = d_out;
    p.out_n_sdf = out_n_sdf ? d_nsdf : nullptr;
    p.out_hit = out_hit ? d_hit : nullptr;
    p.scratch = ctx->pipe_scratch[b];
    e = launch_query(ctx, 0, p, ps);
    if (e != cudaSuccess) return map_err(e);
    if (out_pts) {
      e = cudaMemcpyAsync(out_pts + 4 * c0, d_out, (size_t)m * 16, cudaMemcpyDeviceToHost, ps);
      if (e != cudaSuccess) return map_err(e);
    }
    if (out_n_sdf) {
      e = cudaMemcpyAsync(out_n_sdf + 4 * c0, d_nsdf, (size_t)m * 16, cudaMemcpyDeviceToHost, ps);
      if (e != cudaSuccess) return map_err(e);
    }
    if (out_hit) {
      e = cudaMemcpyAsync(out_hit + c0, d_hit, (size_t)m, cudaMemcpyDeviceToHost, ps);
      if (e != cudaSuccess) return map_err(e);
    }
  }
  for (int i = 0; i < 2; ++i) {
    cudaEventRecord(ctx->ev_done[i], ctx->pipe[i]);
    cudaStreamWaitEvent(s, ctx->ev_done[i], 0);
  }
  e = cudaStreamSynchronize(s);
  return map_err(e);
}

}  // namespace

namespace nsdf {

bool device_memory(const void *p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

nsdf_status ctx_query_setup(nsdf_ctx *ctx, QueryParams *p, int *num_sms, int *width,
                            int *n_hidden, bool *tc16, bool *fp16, const NetDevice **net) {
  if (!ctx->nets[0].loaded) return NSDF_ERR_NOT_LOADED;
  fill_net(ctx, 0, *p);
  *num_sms = ctx->num_sms;
  *width = ctx->arch.width;
  *n_hidden = ctx->arch.n_hidden;
  *tc16 = use_bf16(ctx);
  *fp16 = ctx->prec == NSDF_FP16;
  *net = &ctx->nets[0];
  return NSDF_OK;
}

nsdf_status ctx_set_transform(const float *T, QueryParams *p) { return set_transform(T, *p); }

nsdf_status ctx_query_scratch(nsdf_ctx *ctx, int64_t n, QueryParams *p) {
  nsdf_status st = ensure_scratch(ctx, query_scratch(ctx, query_grid(ctx, n)));
  if (st == NSDF_OK) p->scratch = ctx->scratch;
  return st;
}

int64_t ctx_blob_offsets(const nsdf_ctx *ctx, int64_t *woff, int64_t *boff, int *out) {
  const nsdf_arch &a = ctx->arch;
  int64_t off = (int64_t)a.ff_freqs * a.in_dim;
  for (int l = 0; l <= a.n_hidden; ++l) {
    out[l] = layer_out(a, l);
    woff[l] = off;
    off += (int64_t)layer_out(a, l) * layer_in(a, l);
    boff[l] = off;
    off += layer_out(a, l);
  }
  return off;
}

void **ctx_train_slot(nsdf_ctx *ctx) { return &ctx->train; }

}  // namespace nsdf

extern "C" {

size_t nsdf_num_params(const nsdf_arch *arch) {
  if (!arch_valid(arch)) return 0;
  size_t total = (size_t)arch->ff_freqs * arch->in_dim;
  for (int l = 0; l <= arch->n_hidden; ++l)
    total += (size_t)layer_out(*arch, l) * layer_in(*arch, l) + layer_out(*arch, l);
  return total;
}

const char *nsdf_status_string(nsdf_status s) {
  switch (s) {
    case NSDF_OK: return "ok";
    case NSDF_ERR_INVALID_ARG: return "invalid argument";
    case NSDF_ERR_MISALIGNED: return "pointer not 16-byte aligned";
    case NSDF_ERR_NOT_LOADED: return "weights not loaded";
    case NSDF_ERR_OOM: return "device allocation failed";
    case NSDF_ERR_CUDA: return "CUDA runtime error";
    case NSDF_ERR_UNSUPPORTED: return "unsupported shape or precision";
    case NSDF_ERR_TIMEOUT: return "bounded wait in a kernel ran out";
    case NSDF_ERR_TOO_LARGE: return "request exceeds the fixed scratch of the allocation-free entry point";
  }
  return "unknown status";
}

nsdf_status nsdf_create(const nsdf_arch *arch, nsdf_precision prec, int n_nets, nsdf_ctx **out) {
  if (!out) return NSDF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!arch_valid(arch) || n_nets < 1 || n_nets > 4096) return NSDF_ERR_INVALID_ARG;
  if (prec != NSDF_FP32 && prec != NSDF_BF16 && prec != NSDF_FP16) return NSDF_ERR_INVALID_ARG;
  if (prec == NSDF_FP32 && !query_fp32_supported(arch->width)) return NSDF_ERR_UNSUPPORTED;
  if (prec != NSDF_FP32) {
    const bool ff_relu = arch->ff_freqs > 0 &&
                         query_tc16_ff_supported(arch->width, arch->n_hidden, arch->ff_freqs,
                                                 arch->activation == NSDF_ACT_RELU);
    const bool softplus = arch->ff_freqs == 0 && arch->activation == NSDF_ACT_SOFTPLUS &&
                          (query_tc16_supported(arch->width, arch->n_hidden, arch->skip_layer) ||
                           query_w64_supported(arch->width, arch->n_hidden, arch->skip_layer));
    if (!ff_relu && !softplus) return NSDF_ERR_UNSUPPORTED;
  }
  nsdf_ctx *ctx = new (std::nothrow) nsdf_ctx;
  if (!ctx) return NSDF_ERR_OOM;
  ctx->arch = *arch;
  ctx->prec = prec;
  ctx->n_nets = n_nets;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e != cudaSuccess) {
    delete ctx;
    return map_err(e);
  }
  const int W = arch->width, L = arch->n_hidden;
  ctx->nets.resize(n_nets);
  nsdf_status st = NSDF_OK;
  // Fourier-feature 16-bit contexts keep every network's 16-bit weights in one
  // array, network k at k * n_hidden * W * W, so that one tensor map (that of
  // network 0) reaches all of them in a grouped launch
  uint16_t *ff16_fwd = nullptr, *ff16_bwd = nullptr;
  const size_t ff16_per = (size_t)L * W * W;
  if (prec != NSDF_FP32 && arch->ff_freqs > 0) {
    st = ctx_alloc(ctx, &ff16_fwd, ff16_per * n_nets);
    if (st == NSDF_OK) st = ctx_alloc(ctx, &ff16_bwd, ff16_per * n_nets);
  }
  for (int k = 0; k < n_nets && st == NSDF_OK; ++k) {
    NetDevice &d = ctx->nets[k];
    const size_t hid = (size_t)(L > 1 ? L - 1 : 1) * W * W;
    if (st == NSDF_OK) st = ctx_alloc(ctx, &d.w0, (size_t)W * 3);
    if (st == NSDF_OK) st = ctx_alloc(ctx, &d.bias, (size_t)L * W);
    if (st == NSDF_OK) st = ctx_alloc(ctx, &d.fwd_t, hid);
    if (st == NSDF_OK) st = ctx_alloc(ctx, &d.bwd, hid);
    if (st == NSDF_OK) st = ctx_alloc(ctx, &d.wout, (size_t)W);
    if (st == NSDF_OK) st = ctx_alloc(ctx, &d.bout, 4);
    if (st == NSDF_OK && arch->ff_freqs > 0) {
      st = ctx_alloc(ctx, &d.ffB, (size_t)arch->ff_freqs * 3);
      if (st == NSDF_OK) st = ctx_alloc(ctx, &d.ff0_t, (size_t)W * W);
      if (st == NSDF_OK) st = ctx_alloc(ctx, &d.ff0, (size_t)W * W);
    }
    if (st == NSDF_OK && prec != NSDF_FP32) {
      if (arch->ff_freqs > 0) {        // layer 0 included
        d.fwd16 = ff16_fwd + ff16_per * k;
        d.bwd16 = ff16_bwd + ff16_per * k;
      } else {
        st = ctx_alloc(ctx, &d.fwd16, hid);
        if (st == NSDF_OK) st = ctx_alloc(ctx, &d.bwd16, hid);
        if (st == NSDF_OK && prec == NSDF_BF16 && W == 64) st = ctx_alloc(ctx, &d.fwd16_lo, hid);
      }
    }
  }
  if (st == NSDF_OK) st = ctx_alloc(ctx, &ctx->d_err, 4);
  if (st == NSDF_OK) st = ctx_alloc(ctx, &ctx->d_netptrs, (size_t)n_nets);
  if (st == NSDF_OK) st = ctx_alloc(ctx, &ctx->d_tile_start, (size_t)n_nets + 1);
  if (st == NSDF_OK) st = ctx_alloc(ctx, &ctx->d_body, (size_t)n_nets * kBodyFloats);
  if (st == NSDF_OK) {
    std::vector<NetPtrs> h(n_nets);
    for (int k = 0; k < n_nets; ++k) {
      const NetDevice &d = ctx->nets[k];
      h[k] = NetPtrs{d.w0, d.bias, d.fwd_t, d.bwd, d.wout, d.bout, d.ffB, d.ff0_t, d.ff0,
                     d.fwd16, d.fwd16_lo};
    }
    st = map_err(cudaMemcpy(ctx->d_netptrs, h.data(), sizeof(NetPtrs) * n_nets,
                            cudaMemcpyHostToDevice));
  }
  if (st == NSDF_OK) st = map_err(cudaMemset(ctx->d_err, 0, sizeof(int)));
  if (st != NSDF_OK) {
    nsdf_destroy(ctx);
    return st;
  }
  *out = ctx;
  return NSDF_OK;
}

nsdf_status nsdf_destroy(nsdf_ctx *ctx) {
  if (!ctx) return NSDF_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  for (void *p : ctx->allocations) cudaFree(p);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->bwd_partial) cudaFree(ctx->bwd_partial);
  if (ctx->stage) cudaFree(ctx->stage);
  for (int i = 0; i < 2; ++i) {
    if (ctx->pipe_scratch[i]) cudaFree(ctx->pipe_scratch[i]);
    if (ctx->pipe[i]) cudaStreamDestroy(ctx->pipe[i]);
    if (ctx->ev_done[i]) cudaEventDestroy(ctx->ev_done[i]);
  }
  if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
  train_state_free(ctx->train);
  delete ctx;
  return NSDF_OK;
}

nsdf_status nsdf_load_weights(nsdf_ctx *ctx, int net, const float *w, size_t n_floats,
                              int w_is_device, nsdf_stream stream) {
  if (!ctx || !w || net < 0 || net >= ctx->n_nets) return NSDF_ERR_INVALID_ARG;
  if (n_floats != nsdf_num_params(&ctx->arch)) return NSDF_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const float *src = w;
  float *tmp = nullptr;
  if (!w_is_device) {
    if (cudaMalloc(&tmp, n_floats * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return NSDF_ERR_OOM;
    }
    cudaError_t e = cudaMemcpyAsync(tmp, w, n_floats * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      cudaFree(tmp);
      return map_err(e);
    }
    src = tmp;
  }
  PackPlan plan{};
  const nsdf_arch &a = ctx->arch;
  plan.width = a.width;
  plan.n_hidden = a.n_hidden;
  plan.skip = a.skip_layer;
  plan.ff = a.ff_freqs;
  int64_t off = (int64_t)a.ff_freqs * a.in_dim;
  for (int l = 0; l <= a.n_hidden; ++l) {
    plan.out[l] = layer_out(a, l);
    plan.woff[l] = off;
    off += (int64_t)layer_out(a, l) * layer_in(a, l);
    plan.boff[l] = off;
    off += layer_out(a, l);
  }
  const NetDevice &d = ctx->nets[net];
  PackTargets tg{d.w0,    d.bias,  d.fwd_t, d.bwd,   d.wout,  d.bout, d.ffB,
                 d.ff0_t, d.ff0,   d.fwd16, d.bwd16, ctx->prec == NSDF_FP16 ? 1 : 0,
                 d.fwd16_lo};
  pack_weights_kernel<<<4 * ctx->num_sms, 256, 0, s>>>(src, plan, tg);
  cudaError_t e = last_err();
  if (tmp) {
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(tmp);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return map_err(e);
  const bool fp16 = ctx->prec == NSDF_FP16;
  if (use_tc16_ff(ctx) ? !make_tc16_ff_tmaps(ctx->nets[net], a.n_hidden, net == 0 ? ctx->n_nets : 1, fp16)
                       : use_bf16(ctx) && !use_w64(ctx) &&
                             !make_tc16_tmaps(ctx->nets[net], a.width, a.n_hidden, fp16))
    return NSDF_ERR_CUDA;
  ctx->nets[net].loaded = true;
  return NSDF_OK;
}

nsdf_status nsdf_query(nsdf_ctx *ctx, const float *pts, int64_t n, float *out_n_sdf,
                       uint32_t flags, nsdf_stream stream) {
  if (!ctx || n < 0) return NSDF_ERR_INVALID_ARG;
  if (n == 0) return NSDF_OK;
  if (!pts || !out_n_sdf) return NSDF_ERR_INVALID_ARG;
  if (!aligned16(pts) || !aligned16(out_n_sdf)) return NSDF_ERR_MISALIGNED;
  if (!ctx->nets[0].loaded) return NSDF_ERR_NOT_LOADED;
  if (pointer_kind(pts) != 0 || pointer_kind(out_n_sdf) != 0) return NSDF_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  QueryParams p{};
  fill_net(ctx, 0, p);
  p.pts = reinterpret_cast<const float4 *>(pts);
  p.n = n;
  p.out_n_sdf = reinterpret_cast<float4 *>(out_n_sdf);
  p.collide = 0;
  p.raw_gradient = (flags & NSDF_RAW_GRADIENT) ? 1 : 0;
  const int grid = query_grid(ctx, n);
  nsdf_status st = ensure_scratch(ctx, query_scratch(ctx, grid));
  if (st != NSDF_OK) return st;
  p.scratch = ctx->scratch;
  return map_err(launch_query(ctx, 0, p, s));
}

nsdf_status nsdf_collide(nsdf_ctx *ctx, const float *pts, int64_t n, float eps, const float *T,
                         float *out_pts, float *out_n_sdf, uint8_t *out_hit, nsdf_stream stream) {
  if (!ctx || n < 0 || !std::isfinite(eps)) return NSDF_ERR_INVALID_ARG;
  if (n == 0) return NSDF_OK;
  if (!pts || !out_pts) return NSDF_ERR_INVALID_ARG;
  if (!aligned16(pts) || !aligned16(out_pts) || (out_n_sdf && !aligned16(out_n_sdf)))
    return NSDF_ERR_MISALIGNED;
  if (!ctx->nets[0].loaded) return NSDF_ERR_NOT_LOADED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  QueryParams p{};
  fill_net(ctx, 0, p);
  p.collide = 1;
  p.eps = eps;
  nsdf_status st = set_transform(T, p);
  if (st != NSDF_OK) return st;
  const int kin = pointer_kind(pts);
  const int kout = pointer_kind(out_pts);
  const int kn = out_n_sdf ? pointer_kind(out_n_sdf) : kin;
  const int kh = out_hit ? pointer_kind(out_hit) : kin;
  if (kin != kout || kin != kn || kin != kh) return NSDF_ERR_INVALID_ARG;
  if (kin == 1) return collide_host(ctx, p, pts, n, out_pts, out_n_sdf, out_hit, s);
  p.pts = reinterpret_cast<const float4 *>(pts);
  p.n = n;
  p.out_pts = reinterpret_cast<float4 *>(out_pts);
  p.out_n_sdf = reinterpret_cast<float4 *>(out_n_sdf);
  p.out_hit = out_hit;
  const int grid = query_grid(ctx, n);
  st = ensure_scratch(ctx, query_scratch(ctx, grid));
  if (st != NSDF_OK) return st;
  p.scratch = ctx->scratch;
  return map_err(launch_query(ctx, 0, p, s));
}

nsdf_status nsdf_backward(nsdf_ctx *ctx, const float *pts, int64_t n, const float *g_sdf,
                          const float *g_grad, float *g_weights, float *g_pts, nsdf_stream stream) {
  if (!ctx || n < 0) return NSDF_ERR_INVALID_ARG;
  if (!ctx->nets[0].loaded) return NSDF_ERR_NOT_LOADED;
  const nsdf_arch &a = ctx->arch;
  const int64_t n_params = (int64_t)nsdf_num_params(&a);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    if (g_weights && !device_memory(g_weights)) return NSDF_ERR_INVALID_ARG;
    if (g_weights) return map_err(cudaMemsetAsync(g_weights, 0, sizeof(float) * n_params, s));
    return NSDF_OK;
  }
  if (!pts || !g_sdf || (!g_weights && !g_pts)) return NSDF_ERR_INVALID_ARG;
  if (!aligned16(pts) || (g_grad && !aligned16(g_grad)) || (g_pts && !aligned16(g_pts)))
    return NSDF_ERR_MISALIGNED;
  if (!device_memory(pts) || !device_memory(g_sdf) || (g_grad && !device_memory(g_grad)) ||
      (g_weights && !device_memory(g_weights)) || (g_pts && !device_memory(g_pts)))
    return NSDF_ERR_INVALID_ARG;
  if (!g_grad && !g_weights) {
    // first order only: dL/dp = g_sdf * grad f, through the FP32 query kernel
    if (!query_fp32_supported(a.width)) return NSDF_ERR_UNSUPPORTED;
    QueryParams p{};
    fill_net(ctx, 0, p);
    p.pts = reinterpret_cast<const float4 *>(pts);
    p.n = n;
    p.grad_scale = g_sdf;
    p.out_grad = reinterpret_cast<float4 *>(g_pts);
    const int grid = query_fp32_grid(a.width, n, ctx->num_sms, a.ff_freqs > 0);
    nsdf_status st = ensure_scratch(ctx, query_fp32_scratch_bytes(a.width, a.n_hidden, grid));
    if (st != NSDF_OK) return st;
    p.scratch = ctx->scratch;
    return map_err(launch_query_fp32(p, ctx->num_sms, s));
  }
  if (a.activation != NSDF_ACT_SOFTPLUS || a.ff_freqs > 0 ||
      !backward_supported(a.width, a.n_hidden, n_params))
    return NSDF_ERR_UNSUPPORTED;
  int64_t woff[65], boff[65];
  int out[65];
  int64_t off = 0;
  for (int l = 0; l <= a.n_hidden; ++l) {
    out[l] = layer_out(a, l);
    woff[l] = off;
    off += (int64_t)layer_out(a, l) * layer_in(a, l);
    boff[l] = off;
    off += layer_out(a, l);
  }
  const int grid = backward_grid(n, ctx->num_sms);
  if (g_weights) {
    const size_t need = sizeof(float) * (size_t)grid * n_params;
    if (need > ctx->bwd_partial_bytes) {
      if (ctx->bwd_partial) cudaFree(ctx->bwd_partial);
      ctx->bwd_partial = nullptr;
      ctx->bwd_partial_bytes = 0;
      void *q = nullptr;
      if (cudaMalloc(&q, need) != cudaSuccess) {
        cudaGetLastError();
        return NSDF_ERR_OOM;
      }
      ctx->bwd_partial = static_cast<float *>(q);
      ctx->bwd_partial_bytes = need;
    }
  }
  return map_err(launch_backward(reinterpret_cast<const float4 *>(pts), n, g_sdf,
                                 reinterpret_cast<const float4 *>(g_grad), ctx->bwd_partial, grid,
                                 reinterpret_cast<float4 *>(g_pts), g_weights, ctx->nets[0],
                                 a.width, a.n_hidden, a.skip_layer, a.beta, woff, boff, out,
                                 n_params, s));
}

namespace {

struct GroupedArgs {
  const float *pts;
  const int64_t *offsets, *counts;
  int64_t max_total;
  float eps;
  float *out_pts, *out_n_sdf;
  const float *T = nullptr;   // device [n_nets][16] poses, or none
};

// Above 2^34 points (275 GB of float4 records, more than the GPU holds) the
// device-built tile list could pass 2^31 tiles of the smallest (16-point)
// tile shape and overflow its int32 starts.
constexpr int64_t kMaxGroupedPoints = int64_t(1) << 34;

nsdf_status grouped_check(nsdf_ctx *ctx, const GroupedArgs &g) {
  if (!ctx || g.max_total < 0 || g.max_total > kMaxGroupedPoints || !std::isfinite(g.eps))
    return NSDF_ERR_INVALID_ARG;
  if (g.max_total == 0) return NSDF_OK;
  if (!g.pts || !g.offsets || !g.counts || !g.out_pts) return NSDF_ERR_INVALID_ARG;
  if (!aligned16(g.pts) || !aligned16(g.out_pts) || (g.out_n_sdf && !aligned16(g.out_n_sdf)))
    return NSDF_ERR_MISALIGNED;
  if ((reinterpret_cast<uintptr_t>(g.offsets) & 7u) || (reinterpret_cast<uintptr_t>(g.counts) & 7u))
    return NSDF_ERR_MISALIGNED;
  if (!device_memory(g.pts) || !device_memory(g.offsets) || !device_memory(g.counts) ||
      !device_memory(g.out_pts) || (g.out_n_sdf && !device_memory(g.out_n_sdf)) ||
      (g.T && !device_memory(g.T)))
    return NSDF_ERR_INVALID_ARG;
  for (int k = 0; k < ctx->n_nets; ++k)
    if (!ctx->nets[k].loaded) return NSDF_ERR_NOT_LOADED;
  if (!query_fp32_supported(ctx->arch.width)) return NSDF_ERR_UNSUPPORTED;
  return NSDF_OK;
}

// Grid of a grouped launch for a tile shape and CTAs per SM (0 = as many as fit):
// enough CTAs for the largest possible work list, at most what is resident.
int grouped_grid(const nsdf_ctx *ctx, int pt, int cps, int64_t max_total) {
  const int P = fp32_tile_points(ctx->arch.width, pt);
  const int fit = fp32_ctas_per_sm(ctx->arch.width, pt, ctx->arch.ff_freqs > 0);
  if (cps <= 0 || cps > fit) cps = fit;
  const int64_t max_tiles = (max_total + P - 1) / P + ctx->n_nets;
  const int64_t cap = (int64_t)ctx->num_sms * cps;
  return (int)(max_tiles < cap ? max_tiles : cap);
}

// Grouped launch of the 16-bit Fourier-feature kernel: 128-point tiles, each
// network's tile count rounded up to even (a 2-CTA cluster takes two tiles of
// one network at a time).
nsdf_status grouped_launch_tc16_ff(nsdf_ctx *ctx, const GroupedArgs &g, cudaStream_t s) {
  const int64_t max_tiles = (g.max_total + 127) / 128 + 2 * (int64_t)ctx->n_nets;
  const int grid = query_tc16_ff_grouped_grid(max_tiles, ctx->num_sms);
  nsdf_status st = ensure_scratch(ctx, query_tc16_ff_scratch_bytes(grid));
  if (st != NSDF_OK) return st;
  cudaError_t e = launch_build_tile_list(g.offsets, g.counts, ctx->n_nets, 128, g.max_total,
                                         ctx->d_tile_start, ctx->d_err, s, 2);
  if (e != cudaSuccess) return map_err(e);
  if (g.T) {
    e = launch_body_transforms(g.T, ctx->n_nets, ctx->d_body, ctx->d_err, s);
    if (e != cudaSuccess) return map_err(e);
  }
  QueryParams p{};
  fill_net(ctx, 0, p);
  p.pts = reinterpret_cast<const float4 *>(g.pts);
  p.n = g.max_total;
  p.collide = 1;
  p.eps = g.eps;
  p.out_pts = reinterpret_cast<float4 *>(g.out_pts);
  p.out_n_sdf = reinterpret_cast<float4 *>(g.out_n_sdf);
  p.scratch = ctx->scratch;
  p.g_nets = ctx->n_nets;
  p.g_offsets = g.offsets;
  p.g_counts = g.counts;
  p.g_tile_start = ctx->d_tile_start;
  p.g_netptrs = ctx->d_netptrs;
  p.g_T = g.T ? ctx->d_body : nullptr;
  return map_err(launch_query_tc16_ff(p, ctx->nets[0], ctx->prec == NSDF_FP16, ctx->num_sms, s));
}

// Grouped launch of the 16-bit width-64 kernel: 128-point tiles, each
// network's tile count rounded up to even (the two warpgroups of a CTA take
// a pair of tiles of one network); cps = CTAs per SM (0: as many as fit).
nsdf_status grouped_launch_w64(nsdf_ctx *ctx, const GroupedArgs &g, int cps, cudaStream_t s) {
  cudaError_t e = launch_build_tile_list(g.offsets, g.counts, ctx->n_nets, 128, g.max_total,
                                         ctx->d_tile_start, ctx->d_err, s, 2);
  if (e != cudaSuccess) return map_err(e);
  if (g.T) {
    e = launch_body_transforms(g.T, ctx->n_nets, ctx->d_body, ctx->d_err, s);
    if (e != cudaSuccess) return map_err(e);
  }
  QueryParams p{};
  fill_net(ctx, 0, p);
  p.pts = reinterpret_cast<const float4 *>(g.pts);
  p.n = g.max_total;
  p.collide = 1;
  p.eps = g.eps;
  p.out_pts = reinterpret_cast<float4 *>(g.out_pts);
  p.out_n_sdf = reinterpret_cast<float4 *>(g.out_n_sdf);
  p.g_nets = ctx->n_nets;
  p.g_offsets = g.offsets;
  p.g_counts = g.counts;
  p.g_tile_start = ctx->d_tile_start;
  p.g_netptrs = ctx->d_netptrs;
  p.g_T = g.T ? ctx->d_body : nullptr;
  return map_err(launch_query_w64(p, ctx->prec == NSDF_FP16, ctx->num_sms, cps, s));
}

nsdf_status grouped_launch(nsdf_ctx *ctx, const GroupedArgs &g, int pt, int cps, cudaStream_t s) {
  if (use_tc16_ff(ctx)) return grouped_launch_tc16_ff(ctx, g, s);
  if (use_w64(ctx)) return grouped_launch_w64(ctx, g, cps, s);
  const nsdf_arch &a = ctx->arch;
  const int grid = grouped_grid(ctx, pt, cps, g.max_total);
  nsdf_status st = ensure_scratch(ctx, fp32_scratch_bytes_pt(a.width, pt, a.n_hidden, grid));
  if (st != NSDF_OK) return st;
  cudaError_t e = launch_build_tile_list(g.offsets, g.counts, ctx->n_nets,
                                         fp32_tile_points(a.width, pt), g.max_total,
                                         ctx->d_tile_start, ctx->d_err, s);
  if (e != cudaSuccess) return map_err(e);
  if (g.T) {
    e = launch_body_transforms(g.T, ctx->n_nets, ctx->d_body, ctx->d_err, s);
    if (e != cudaSuccess) return map_err(e);
  }
  QueryParams p{};
  fill_net(ctx, 0, p);
  p.pts = reinterpret_cast<const float4 *>(g.pts);
  p.n = g.max_total;
  p.collide = 1;
  p.eps = g.eps;
  p.out_pts = reinterpret_cast<float4 *>(g.out_pts);
  p.out_n_sdf = reinterpret_cast<float4 *>(g.out_n_sdf);
  p.scratch = ctx->scratch;
  p.g_nets = ctx->n_nets;
  p.g_offsets = g.offsets;
  p.g_counts = g.counts;
  p.g_tile_start = ctx->d_tile_start;
  p.g_netptrs = ctx->d_netptrs;
  p.g_T = g.T ? ctx->d_body : nullptr;
  return map_err(launch_query_fp32_grouped(p, pt, grid, s));
}

}  // namespace

nsdf_status nsdf_query_grouped(nsdf_ctx *ctx, const float *pts, const int64_t *offsets,
                               const int64_t *counts, int64_t max_total, float eps, float *out_pts,
                               float *out_n_sdf, nsdf_stream stream) {
  const GroupedArgs g{pts, offsets, counts, max_total, eps, out_pts, out_n_sdf};
  nsdf_status st = grouped_check(ctx, g);
  if (st != NSDF_OK || max_total == 0) return st;
  return grouped_launch(ctx, g, ctx->grouped_pt, ctx->grouped_cps,
                        reinterpret_cast<cudaStream_t>(stream));
}

nsdf_status nsdf_query_grouped_T(nsdf_ctx *ctx, const float *pts, const int64_t *offsets,
                                 const int64_t *counts, int64_t max_total, float eps,
                                 const float *T, float *out_pts, float *out_n_sdf,
                                 nsdf_stream stream) {
  GroupedArgs g{pts, offsets, counts, max_total, eps, out_pts, out_n_sdf};
  g.T = T;
  nsdf_status st = grouped_check(ctx, g);
  if (st != NSDF_OK || max_total == 0) return st;
  if (!T || (reinterpret_cast<uintptr_t>(T) & 3u)) return NSDF_ERR_INVALID_ARG;
  return grouped_launch(ctx, g, ctx->grouped_pt, ctx->grouped_cps,
                        reinterpret_cast<cudaStream_t>(stream));
}

nsdf_status nsdf_autotune_grouped(nsdf_ctx *ctx, const float *pts, const int64_t *offsets,
                                  const int64_t *counts, int64_t max_total, float eps,
                                  float *out_pts, float *out_n_sdf, nsdf_stream stream,
                                  int *chosen) {
  const GroupedArgs g{pts, offsets, counts, max_total, eps, out_pts, out_n_sdf};
  nsdf_status st = grouped_check(ctx, g);
  if (st != NSDF_OK) return st;
  if (max_total == 0) return NSDF_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (use_tc16_ff(ctx)) {   // one shape: a 128-point tile per CTA, one CTA per SM
    st = grouped_launch(ctx, g, 0, 0, s);
    if (st == NSDF_OK) st = map_err(cudaStreamSynchronize(s));
    if (st == NSDF_OK && chosen) {
      chosen[0] = 0;
      chosen[1] = 1;
    }
    return st;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return NSDF_ERR_CUDA;
  float best = 3.0e38f;
  int best_pt = ctx->grouped_pt, best_cps = ctx->grouped_cps;
  // FP32 kernel: points per thread (4 or 8) and CTAs per SM; 16-bit width-64
  // kernel: CTAs per SM (its tiles are 128 points, two per CTA)
  const bool w64 = use_w64(ctx);
  const int pts_opts[2] = {4, 8};
  for (int oi = 0; oi < (w64 ? 1 : 2); ++oi) {
    const int pt = w64 ? 0 : pts_opts[oi];
    const int fit = w64 ? query_w64_ctas_per_sm(ctx->arch.n_hidden, ctx->prec == NSDF_FP16)
                        : fp32_ctas_per_sm(ctx->arch.width, pt, ctx->arch.ff_freqs > 0);
    for (int cps = 1; cps <= fit; ++cps) {
      st = grouped_launch(ctx, g, pt, cps, s);             // warm-up (and scratch growth)
      if (st != NSDF_OK) break;
      cudaEventRecord(e0, s);
      for (int rep = 0; rep < 3; ++rep) grouped_launch(ctx, g, pt, cps, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = NSDF_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_pt = pt;
        best_cps = cps;
      }
    }
    if (st != NSDF_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NSDF_OK) return st;
  ctx->grouped_pt = best_pt;
  ctx->grouped_cps = best_cps;
  if (chosen) {
    chosen[0] = best_pt;
    chosen[1] = best_cps;
  }
  return NSDF_OK;
}

nsdf_status nsdf_set_grouped_config(nsdf_ctx *ctx, int points_per_thread, int ctas_per_sm) {
  if (!ctx || ctas_per_sm < 0) return NSDF_ERR_INVALID_ARG;
  const bool one_shape = use_tc16_ff(ctx) || use_w64(ctx);
  if (points_per_thread != 4 && points_per_thread != 8 && !(one_shape && points_per_thread == 0))
    return NSDF_ERR_INVALID_ARG;
  if (points_per_thread != 0) ctx->grouped_pt = points_per_thread;
  ctx->grouped_cps = ctas_per_sm;
  return NSDF_OK;
}

nsdf_status nsdf_sync_status(nsdf_ctx *ctx, nsdf_stream stream) {
  if (!ctx) return NSDF_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return map_err(e);
  int h = 0;
  e = cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return map_err(e);
  if (h != kDevOk) {
    cudaMemset(ctx->d_err, 0, sizeof(int));
    return h == kDevBadWork ? NSDF_ERR_INVALID_ARG : NSDF_ERR_TIMEOUT;
  }
  return NSDF_OK;
}

nsdf_status nsdf_debug_inject(nsdf_ctx *ctx, int drop_load, long long wait_budget_cycles) {
  if (!ctx || wait_budget_cycles <= 0) return NSDF_ERR_INVALID_ARG;
  ctx->drop_load = drop_load;
  ctx->wait_budget = wait_budget_cycles;
  return NSDF_OK;
}

}  // extern "C"
