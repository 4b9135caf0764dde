// Internal declarations shared by the host runtime and the kernels of the
// nsdf library.  Nothing here is part of the public ABI (include/nsdf.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <cstddef>

#include "nsdf.h"

namespace nsdf {

// Kernel-side error codes written into a context's device error word.
enum DeviceError : int {
  kDevOk = 0,
  kDevTimeout = 1,   // a bounded mbarrier wait gave up
  kDevBadWork = 2,   // a grouped work list entry lies outside [0, max_total)
};

// Device copies of one network, in the layouts the kernels read.
// Hidden layers l = 1 .. n_hidden-1 are padded to width x width (a layer
// with fewer outputs gets zero rows and zero biases).
struct NetDevice {
  // FP32 forms
  float *w0 = nullptr;     // [width][3]   L0 weights, row n = (W0[n][0..2])
  float *bias = nullptr;   // [n_hidden][width]
  float *fwd_t = nullptr;  // [n_hidden-1][width(k)][width(n)] = W_l[n][k]
  float *bwd = nullptr;    // [n_hidden-1][width(n)][width(k)] = W_l[n][k]
  float *wout = nullptr;   // [width]      output weights (zero padded)
  float *bout = nullptr;   // [1]
  // Fourier-feature networks (ff_freqs = m > 0, 2m = width): B and L0 as
  // width x width panels in the layouts of fwd_t / bwd
  float *ffB = nullptr;    // [m][3]
  float *ff0_t = nullptr;  // [width(k)][width(n)] = W_0[n][k]
  float *ff0 = nullptr;    // [width(n)][width(k)] = W_0[n][k]
  // 16-bit forms (tensor-core B operands, K-major; BF16 or FP16 bits);
  // Fourier-feature networks hold n_hidden layers here, layer 0 first
  uint16_t *fwd16 = nullptr;  // [n_hidden-1][width(n)][width(k)] = W_l
  uint16_t *bwd16 = nullptr;  // [n_hidden-1][width(k)][width(n)] = W_l^T
  // BF16 width-64 contexts: the rounding residual W_l - bf16(W_l), in BF16
  uint16_t *fwd16_lo = nullptr;  // [n_hidden-1][width(n)][width(k)]
  // TMA descriptors of fwd16 / bwd16 (16-bit contexts only)
  CUtensorMap tmap_fwd;
  CUtensorMap tmap_bwd;
  bool loaded = false;
};

// FP32 weight pointers of one network, as a device array for grouped launches.
struct NetPtrs {
  const float *w0, *bias, *fwd_t, *bwd, *wout, *bout;
  const float *ffB, *ff0_t, *ff0;
  const uint16_t *w16, *w16lo;   // 16-bit hidden weights (and residuals) of the width-64 kernel
};

// Everything one fused query launch needs (passed by value).
struct QueryParams {
  const float4 *pts;
  int64_t n;
  float4 *out_n_sdf;   // nullable
  float4 *out_pts;     // nullable (query mode)
  uint8_t *out_hit;    // nullable
  float eps;
  int collide;         // 1: collision solve, 0: plain query
  int raw_gradient;    // query mode: output grad f instead of N
  int has_T;
  float Ti[12];        // T^{-1}, rows 0..2 of the 4x4 (row-major)
  float R[9];          // T[:3,:3]
  // network
  const float *w0, *bias, *fwd_t, *bwd, *wout, *bout;
  const uint16_t *fwd16, *bwd16;
  const uint16_t *fwd16_lo;  // BF16 width-64 contexts: W_l - bf16(W_l)
  int width, n_hidden, skip;
  float beta;
  int relu;                  // activation: 0 softplus_beta, 1 ReLU
  int ff;                    // Fourier features: m (0 = none; 2m = width)
  const float *ffB, *ff0_t, *ff0;
  // per-CTA scratch and the context's error word
  float *scratch;
  int *err;
  // bounded waits: clock cycles one mbarrier wait may spin before the kernel
  // records kDevTimeout and unwinds; drop_load >= 0 skips that weight load
  // (fault injection for tests of the timeout path; -1 in normal use)
  long long wait_budget;
  int drop_load;
  // first-order backward through the query kernel: out_grad[i] = grad_scale[i] * grad f
  const float *grad_scale;   // nullable
  float4 *out_grad;
  // grouped launch (g_nets > 0): tile t of network k covers points
  // g_offsets[k] + (t - g_tile_start[k]) * P ... (capped by g_counts[k])
  int g_nets;
  const int64_t *g_offsets, *g_counts;
  const int32_t *g_tile_start;   // [g_nets + 1], built on the device
  const NetPtrs *g_netptrs;      // [g_nets]
  // training form of the 16-bit kernel (both non-null): every layer's A
  // operand as [n_hidden][ceil(n / 128) * 128][width] 16-bit values:
  // save_h[l] = h_l, save_d[l] = delta_l = d f / d z_l
  uint16_t *save_h, *save_d;
  // grouped: per-network rigid pose, kBodyFloats floats each (T^{-1} rows
  // 0..2, then T[:3,:3]); nullable (no transform)
  const float *g_T;
};

// Floats per network in QueryParams::g_T.
constexpr int kBodyFloats = 24;

// True for memory the GPU addresses as device memory (device or managed
// allocations).  Every entry point that takes DEVICE pointers rejects
// anything else with NSDF_ERR_INVALID_ARG before it launches, so that a host
// array passed by mistake never reaches a kernel.  cudaPointerGetAttributes
// allocates nothing and does not synchronise, so the check also runs while
// a stream is being captured into a CUDA graph.
bool device_memory(const void *p);

// Launchers (return a cudaError_t from the launch).
cudaError_t launch_query_fp32(const QueryParams &p, int num_sms, cudaStream_t s);
size_t query_fp32_scratch_bytes(int width, int n_hidden, int grid);
int query_fp32_grid(int width, int64_t n, int num_sms, bool ff = false);
bool query_fp32_supported(int width);
// grouped FP32 launches with a chosen tile shape (pt = points per thread, 4 or 8)
int fp32_tile_points(int width, int pt);
int fp32_ctas_per_sm(int width, int pt, bool ff = false);
size_t fp32_scratch_bytes_pt(int width, int pt, int n_hidden, int grid);
cudaError_t launch_query_fp32_grouped(const QueryParams &p, int pt, int grid, cudaStream_t s);

// Weight-gradient products of the fitting loss on the tensor cores
// (wgrad_tc.cu): for product i, G[gslot[i]] (W x W, row-major [n][k], FP32)
// = sum over the n_pad points of D(point)[n] H(point)[k], with D rows
// save_d[dslot[i]] and H rows save_h[hslot[i]] (16-bit, [slot][n_pad][W]).
// ws holds layers x S x W x W floats of split partials.
struct WgradJob {
  const uint16_t *save_h, *save_d;
  int64_t h_rows, d_rows;   // rows of the two saved arrays (slots x n_pad)
  int64_t n_pad;
  int W, layers, S;
  int hslot[64], dslot[64], gslot[64];
  float *ws, *G;
  int *err;
  long long wait_budget;
  bool fp16;
  int num_sms;
};
int wgrad_splits(int W, int layers, int64_t n_pad, int num_sms);
bool wgrad_supported(int W);
cudaError_t launch_wgrad_tc(const WgradJob &job, cudaStream_t s);

// 16-bit tensor-core form for width-64 softplus networks (query_tc16_w64.cu):
// single-network launches and grouped launches (QueryParams::g_nets > 0, a
// tile list built with 128-point tiles rounded up to even per network); no
// per-CTA scratch.  ctas_per_sm <= 0: as many as fit.
bool query_w64_supported(int width, int n_hidden, int skip);
int query_w64_ctas_per_sm(int n_hidden, bool fp16);
cudaError_t launch_query_w64(const QueryParams &p, bool fp16, int num_sms, int ctas_per_sm,
                             cudaStream_t s);

// Brute-force mesh SDF (mesh_sdf.cu) of n explicit points, or, with
// pts == nullptr, of the n = grid_n^3 nodes lo + (i, j, k) h of a regular
// grid (index i + grid_n (j + grid_n k)).
cudaError_t launch_mesh_sdf(const float *verts, int64_t n_verts, const int32_t *faces,
                            int64_t n_faces, const float4 *pts, int64_t n, float *out, int grid_n,
                            const float *lo, const float *h, cudaStream_t s);

bool query_tc16_supported(int width, int n_hidden, int skip);
bool make_tc16_tmaps(NetDevice &net, int width, int n_hidden, bool fp16);
cudaError_t launch_query_tc16_net(const QueryParams &p, const NetDevice &net, bool fp16,
                                  int num_sms, cudaStream_t s);
size_t query_tc16_scratch_bytes(int width, int n_hidden, int grid, bool fp16);
int query_tc16_grid(int width, int64_t n, int num_sms);
int query_tc16_min_grid();   // CTAs of one cluster: the smallest grid of the kernel

// 16-bit tensor-core form of the Fourier-feature ReLU networks of Sec. 4.3
// (width 256, m = 128, 1..8 layers; query_tc16_ff.cu).  Its 16-bit weight
// copies hold all n_hidden layers, layer l at [l][256][256], layer 0 with the
// feature columns permuted (ff_feature_of_column).  Its scratch holds the
// ReLU slope bits, one 28 KB slab per CTA.
bool query_tc16_ff_supported(int width, int n_hidden, int ff, int relu);
size_t query_tc16_ff_scratch_bytes(int grid);
// rows_nets: how many networks' weights follow net's 16-bit copies
// contiguously (the map of network 0 covers every network of a context, so
// that a grouped launch addresses network k at rows k * n_hidden * 256)
bool make_tc16_ff_tmaps(NetDevice &net, int n_hidden, int rows_nets, bool fp16);
int query_tc16_ff_grid(int64_t n, int num_sms);
// grouped launches (QueryParams::g_nets > 0): the grid for up to max_tiles tiles
int query_tc16_ff_grouped_grid(int64_t max_tiles, int num_sms);
cudaError_t launch_query_tc16_ff(const QueryParams &p, const NetDevice &net, bool fp16,
                                 int num_sms, cudaStream_t s);
// Column c = 128 g + 64 s + i of that kernel's feature tile holds feature
// s * m + 64 g + i of gamma(p) (sines are features 0..m-1, cosines m..2m-1).
__host__ __device__ inline int ff_feature_of_column(int c, int m) {
  return ((c >> 6) & 1) * m + 64 * (c >> 7) + (c & 63);
}

// Context accessors for entry points defined outside api.cu: the network-0
// launch parameters of a loaded context, and the transform of nsdf_collide.
nsdf_status ctx_query_setup(nsdf_ctx *ctx, QueryParams *p, int *num_sms, int *width,
                            int *n_hidden, bool *tc16, bool *fp16, const NetDevice **net);
nsdf_status ctx_set_transform(const float *T, QueryParams *p);
// Per-CTA scratch of a query over n points (allocated or grown here).
nsdf_status ctx_query_scratch(nsdf_ctx *ctx, int64_t n, QueryParams *p);
// Blob offsets of the weights / biases of layers 0..n_hidden and their
// output counts; returns the blob size.
int64_t ctx_blob_offsets(const nsdf_ctx *ctx, int64_t *woff, int64_t *boff, int *out);
// The context's slot for the training state of train.cu (freed by
// train_state_free in nsdf_destroy).
void **ctx_train_slot(nsdf_ctx *ctx);
void train_state_free(void *state);

cudaError_t launch_build_tile_list(const int64_t *offsets, const int64_t *counts, int n_nets, int P,
                                   int64_t max_total, int32_t *tile_start, int *err,
                                   cudaStream_t s, int round_to = 1);
// T [n_nets][16] (row-major 4x4 poses, device) -> out [n_nets][kBodyFloats]
cudaError_t launch_body_transforms(const float *T, int n_nets, float *out, int *err,
                                   cudaStream_t s);

size_t backward_smem_bytes(int width, int n_hidden, int64_t n_params);
bool backward_supported(int width, int n_hidden, int64_t n_params);
int backward_grid(int64_t n, int num_sms);
cudaError_t launch_backward(const float4 *pts, int64_t n, const float *a, const float4 *v,
                            float *g_partial, int grid, float4 *g_pts, float *g_weights,
                            const NetDevice &net, int width, int n_hidden, int skip, float beta,
                            const int64_t *woff, const int64_t *boff, const int *out,
                            int64_t n_params, cudaStream_t s);

}  // namespace nsdf
