// Allocation-free collision query.
//
// Some callers cannot call cudaMalloc at query time: a physics engine that
// runs the collision solve inside its own fixed-memory budget, a host that
// records the work into a CUDA graph or issues it from a real-time callback
// (where an allocation would synchronise the device or is simply not
// allowed), or an embedding that forbids the library from growing its
// footprint after set-up.  nsdf_collide_noalloc serves them: it runs the same
// fused query kernels as nsdf_collide but takes their per-CTA scratch from a
// fixed, file-scope device array instead of the context's allocations, and
// never calls an allocating routine.
//
// The array is kNoAllocScratchBytes large; every GPU that loads the library
// holds it until the process exits.  The kernels' scratch is one slab per
// CTA, so the launch uses as many CTAs as there are whole slabs in the array
// (at most one per SM): larger networks get fewer CTAs and run slower, and a
// network whose single slab exceeds the array is rejected with
// NSDF_ERR_TOO_LARGE.  Slabs need no clearing: each tile writes its slopes
// before reading them.  All calls share the array: calls whose kernels can
// overlap on the GPU (different streams, or several host threads) race on it
// and must be serialised by the caller.

#include <atomic>
#include <cmath>
#include <mutex>

#include "nsdf_debug.h"
#include "nsdf_internal.h"

namespace nsdf {

// 32 MiB: 36 CTAs for the 512-wide, 8-layer body-scale network in 16 bits
// (896 KiB of slopes per CTA), 73 in FP32.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;

__device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};
// Test-only cap on the bytes of the array a call may use (0 = all of it);
// set through nsdf_debug_noalloc_limit so that a test can reach the
// NSDF_ERR_TOO_LARGE reject, which no network the library accepts reaches
// with the full array.
std::atomic<size_t> g_limit{0};

size_t usable_bytes() {
  const size_t lim = g_limit.load();
  return lim != 0 && lim < kNoAllocScratchBytes ? lim : kNoAllocScratchBytes;
}

// Device address of g_noalloc_scratch on the current device (host code only
// sees a host-side stand-in for the symbol).  Resolved once per device and
// kept for the life of the process: a device reset (cudaDeviceReset) would
// unload the module and leave the kept address dangling, exactly as it frees
// every context's weights, so the library is not used across one.
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace nsdf

using namespace nsdf;

extern "C" nsdf_status nsdf_collide_noalloc(nsdf_ctx *ctx, const float *pts, int64_t n, float eps,
                                            const float *T, float *out_pts, float *out_n_sdf,
                                            uint8_t *out_hit, nsdf_stream stream) {
  if (!ctx || n < 0 || !std::isfinite(eps)) return NSDF_ERR_INVALID_ARG;
  if (n == 0) return NSDF_OK;
  if (!pts || !out_pts) return NSDF_ERR_INVALID_ARG;
  auto mis = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
  if (mis(pts) || mis(out_pts) || (out_n_sdf && mis(out_n_sdf))) return NSDF_ERR_MISALIGNED;
  if (!device_memory(pts) || !device_memory(out_pts) || (out_n_sdf && !device_memory(out_n_sdf)) ||
      (out_hit && !device_memory(out_hit)))
    return NSDF_ERR_INVALID_ARG;
  QueryParams p{};
  int num_sms = 0, width = 0, n_hidden = 0;
  bool tc16 = false, fp16 = false;
  const NetDevice *net = nullptr;
  nsdf_status st = ctx_query_setup(ctx, &p, &num_sms, &width, &n_hidden, &tc16, &fp16, &net);
  if (st != NSDF_OK) return st;
  st = ctx_set_transform(T, &p);
  if (st != NSDF_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  p.pts = reinterpret_cast<const float4 *>(pts);
  p.n = n;
  p.collide = 1;
  p.eps = eps;
  p.out_pts = reinterpret_cast<float4 *>(out_pts);
  p.out_n_sdf = reinterpret_cast<float4 *>(out_n_sdf);
  p.out_hit = out_hit;
  if (tc16 && query_w64_supported(width, n_hidden, p.skip) && p.ff == 0) {
    // width-64 tensor-core kernel: no scratch at all
    const cudaError_t e = launch_query_w64(p, fp16, num_sms, 0, s);
    return e == cudaSuccess ? NSDF_OK : NSDF_ERR_CUDA;
  }
  if (tc16 && p.ff > 0) {   // Fourier-feature tensor-core kernel: one slope-bit slab per CTA
    const int grid = query_tc16_ff_grid(n, num_sms);
    if (query_tc16_ff_scratch_bytes(grid) > usable_bytes()) return NSDF_ERR_TOO_LARGE;
    void *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return NSDF_ERR_CUDA;
    p.scratch = static_cast<float *>(scratch);
    const cudaError_t e = launch_query_tc16_ff(p, *net, fp16, num_sms, s);
    return e == cudaSuccess ? NSDF_OK : NSDF_ERR_CUDA;
  }
  // one slab per CTA; as many CTAs as whole slabs fit.  The launchers size
  // their grid as min(tiles, sm_arg * CTAs per SM), so sm_arg is chosen to
  // keep that product within the slabs the array holds.
  const size_t slab = tc16 ? query_tc16_scratch_bytes(width, n_hidden, 1, fp16)
                           : query_fp32_scratch_bytes(width, n_hidden, 1);
  const int64_t slabs = (int64_t)(usable_bytes() / slab);
  const int per_sm = tc16 ? 1 : query_fp32_grid(width, (int64_t)1 << 40, 1, p.ff > 0);
  if (slabs < per_sm || per_sm < 1) return NSDF_ERR_TOO_LARGE;
  if (tc16 && slabs < query_tc16_min_grid()) return NSDF_ERR_TOO_LARGE;
  int64_t sm_arg = slabs / per_sm;
  if (sm_arg > num_sms) sm_arg = num_sms;
  const int ctas = (int)sm_arg;
  void *scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return NSDF_ERR_CUDA;
  p.scratch = static_cast<float *>(scratch);
  const cudaError_t e = tc16 ? launch_query_tc16_net(p, *net, fp16, ctas, s)
                             : launch_query_fp32(p, ctas, s);
  return e == cudaSuccess ? NSDF_OK : NSDF_ERR_CUDA;
}

extern "C" nsdf_status nsdf_debug_noalloc_limit(size_t bytes) {
  g_limit.store(bytes);
  return NSDF_OK;
}
