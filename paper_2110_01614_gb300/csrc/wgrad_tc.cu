// Weight-gradient products of the fitting loss on the tensor cores.
//
// For every hidden layer l of a 16-bit context the gradient of the L1
// fitting loss (Sec. 3.1) needs G_l[n][k] = sum_i D_l(i)[n] H_l(i)[k], a
// contraction over the training points i of the layer's saved output
// deltas D (already multiplied by sign(f_i - d_i)) and its saved inputs H;
// train.cu saves both as 16-bit rows, one row of W values per point.  As a
// tcgen05 product the points are the reduction dimension K, so both
// operands are MN-major: a TMA box of 64 points x 64 columns (128-byte
// swizzle) is one K x MN block of either operand.
//
// Work units: an output tile of 256 rows (n) x 256 columns (k) of one layer
// and one of S contiguous ranges of the points (split K), ordered range by
// range.  The tile is one CTA pair's product (cta_group::2, M = 256): the two
// CTAs of a 2-CTA cluster each hold 128 of its rows of D and 128 of its
// columns of H, and the even CTA issues the MMAs over both.  A persistent
// pair walks its units; per unit, 64-point steps stream through a 6-stage
// ring (per CTA: A 2 boxes of 64 x 64 = 16 KB, B 2 boxes = 16 KB; the bytes
// of both CTAs are counted on the even CTA's barrier), one thread issues 4
// tcgen05.mma (M=256, N=256, K=16; 16-bit x 16-bit -> FP32) per step into one
// of two TMEM accumulators of 256 columns (each CTA holds its 128 rows), and
// four epilogue warps per CTA move the finished accumulator to the unit's
// FP32 partial (tcgen05.ld) while the next unit is multiplied; the odd CTA's
// "accumulator drained" arrivals reach the even CTA through a relay thread.
// Per SM this streams 32 KB per step instead of the 48 KB of one CTA per
// 128 x 256 tile.  A second kernel sums each output's S partials in split
// order, so the result does not depend on scheduling.
//
// Warp roles (192 threads): warp 0 = TMA producer, warp 1 = MMA issuer (even
// CTA) or relay (odd CTA) and TMEM owner, warps 2..5 = epilogue (warp w reads
// TMEM lanes 32*(w%4)..+31).  Every mbarrier wait is bounded; on expiry the
// kernel records kDevTimeout in the context's error word, drains what it has
// in flight and returns.

#include <cudaTypedefs.h>

#include "nsdf_internal.h"
#include "tc_ptx.cuh"

namespace nsdf {
namespace {

using namespace ptx;

constexpr int kTM = 128;                 // tile rows (n) per CTA: TMEM lanes
constexpr int kPM = 2 * kTM;             // tile rows of the pair's product (MMA M)
constexpr int kTN = 256;                 // tile columns (k): MMA N
constexpr int kStepPts = 64;             // points per pipeline step (K)
constexpr int kStages = 6;
constexpr int kBoxBytes = 64 * 64 * 2;   // one 64-point x 64-column box
constexpr int kABytes = 2 * kBoxBytes;   // 16 KB: this CTA's 128 rows of D
constexpr int kBBytes = 2 * kBoxBytes;   // 16 KB: this CTA's 128 columns of H
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kThreads = 192;
constexpr int kCluster = 2;
constexpr int kOffBar = kStages * kStageBytes;
// barriers: full[kStages], empty[kStages], acc_full[2], acc_empty[2], mma_done
constexpr int kNumBars = 2 * kStages + 5;
constexpr int kOffTmemSlot = kOffBar + 8 * kNumBars;
constexpr int kOffAbort = kOffTmemSlot + 4;
constexpr int kSmemBytes = kOffAbort + 16 + 1024;   // + slack to align the base to 1024
static_assert(kSmemBytes <= 232448, "shared memory budget");

// Shared-memory descriptor of an MN-major operand in the 128-byte swizzle
// layout: 64-element MN blocks `lbo` bytes apart, 8-point K groups 1024 bytes
// apart (one 128-byte row per point), descriptor version 1, SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw128_desc_mn(uint32_t saddr, uint32_t lbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

struct GslotMap {
  int gslot[64];      // per product: slot of its gradient in G
};

struct WgradParams {
  int64_t n_pad;      // points per saved layer (rows), a multiple of 128
  int W;              // width: 256 or 512
  int layers;         // products to form
  int S;              // point ranges per output tile (split K)
  int hslot[64];      // per product: slot of H (its input) in the saved inputs
  int dslot[64];      // per product: slot of D (its output deltas) in the saved deltas
  float *ws;          // partials [layers][S][W][W]
  int *err;
  long long wait_budget;
  uint32_t idesc;
};

__global__ void __launch_bounds__(kThreads, 1)
    wgrad_tc_kernel(const __grid_constant__ WgradParams prm, const __grid_constant__ CUtensorMap map_h,
                    const __grid_constant__ CUtensorMap map_d) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = sbase + kOffBar;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
  auto accf_bar = [&](int b) { return bar0 + 8u * (2 * kStages + b); };
  auto acce_bar = [&](int b) { return bar0 + 8u * (2 * kStages + 2 + b); };
  const uint32_t done_bar = bar0 + 8u * (2 * kStages + 4);
  volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(smem + kOffTmemSlot);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + kOffAbort);
  const long long budget = prm.wait_budget;
  const uint32_t crank = cluster_rank();
  const uint16_t cmask = (uint16_t)((1u << kCluster) - 1u);

  const int W = prm.W;
  const int mt_n = W / kPM, nt_n = W / kTN;
  const int tiles = prm.layers * mt_n * nt_n;
  const int64_t units = (int64_t)tiles * prm.S;
  const int64_t ksteps = prm.n_pad / kStepPts;
  const int64_t pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);      // the even CTA's commit reaches both CTAs
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf_bar(b), 1);
      // one arrival per epilogue warp; the even CTA's also counts the relayed
      // arrival of the odd CTA's epilogue
      mbar_init(acce_bar(b), crank == 0 ? 5 : 4);
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fence_proxy_async();
  }
  if (warp == 1) {   // one warp of each CTA of the pair allocates collectively
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     sbase + kOffTmemSlot),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();    // both CTAs' barriers exist before any load or commit targets them
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto fail = [&]() {
    atomicExch(prm.err, kDevTimeout);
    *abort_flag = 1;
  };
  // unit -> (product, tile row, tile column, first and end step).  Units run
  // tile-minor: the pairs working at the same time share one range of points,
  // so each 64-point box of D and H comes from DRAM once and from L2 for the
  // other tiles of its layer.
  auto decode = [&](int64_t u, int &li, int &mt, int &nt, int64_t &kb, int64_t &ke) {
    const int t = (int)(u % tiles), s = (int)(u / tiles);
    li = t / (mt_n * nt_n);
    const int rem = t % (mt_n * nt_n);
    mt = rem / nt_n;
    nt = rem % nt_n;
    kb = ksteps * s / prm.S;
    ke = ksteps * (s + 1) / prm.S;
  };

  if (warp == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, issued_parity = 0;
      bool ok = true;
      for (int64_t u = pair; ok && u < units; u += npairs) {
        int li, mt, nt;
        int64_t kb, ke;
        decode(u, li, mt, nt, kb, ke);
        const int ya0 = prm.dslot[li], yb0 = prm.hslot[li];
        for (int64_t k = kb; k < ke; ++k) {
          if (!mbar_wait(empty_bar(stage), phase ^ 1u, budget, abort_flag)) {
            fail();
            ok = false;
            break;
          }
          const uint32_t st = sbase + stage * kStageBytes;
          if (crank == 0) mbar_expect_tx(full_bar(stage), kCluster * kStageBytes);
          const uint32_t lead_full = map_to_rank(full_bar(stage), 0);
          const int ya = (int)((int64_t)ya0 * prm.n_pad + k * kStepPts);
          const int yb = (int)((int64_t)yb0 * prm.n_pad + k * kStepPts);
#pragma unroll
          for (int j = 0; j < 2; ++j)      // this CTA's 128 rows of the tile's D
            tma_load_2d_pair(st + j * kBoxBytes, &map_d, mt * kPM + (int)crank * kTM + 64 * j, ya,
                             lead_full);
#pragma unroll
          for (int j = 0; j < 2; ++j)      // this CTA's 128 of the tile's columns of H
            tma_load_2d_pair(st + kABytes + j * kBoxBytes, &map_h,
                             nt * kTN + (int)crank * (kTN / 2) + 64 * j, yb, lead_full);
          issued_mask |= 1u << stage;
          issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
          if (++stage == kStages) stage = 0, phase ^= 1u;
        }
      }
      // every issued load lands before the CTA may exit (the even CTA's
      // barriers count both CTAs' bytes)
      if (crank == 0) {
        for (int s = 0; s < kStages; ++s) {
          if (issued_mask & (1u << s)) {
            volatile int no_abort = 0;
            if (!mbar_wait(full_bar(s), (issued_parity >> s) & 1u, budget, &no_abort)) fail();
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && crank == 0) {
      // ---------------- MMA issuer (the even CTA) ----------------
      int stage = 0;
      uint32_t phase = 0;
      uint32_t acc_phase[2] = {0u, 0u};
      int local = 0;
      bool ok = true;
      for (int64_t u = pair; ok && u < units; u += npairs, ++local) {
        int li, mt, nt;
        int64_t kb, ke;
        decode(u, li, mt, nt, kb, ke);
        const int b = local & 1;
        // both CTAs' epilogues have emptied this accumulator (its previous unit)
        if (!mbar_wait_cluster(acce_bar(b), acc_phase[b] ^ 1u, budget, abort_flag)) {
          fail();
          break;
        }
        acc_phase[b] ^= 1u;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * kTN);
        for (int64_t k = kb; k < ke; ++k) {
          if (!mbar_wait(full_bar(stage), phase, budget, abort_flag)) {
            fail();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = sbase + stage * kStageBytes;
#pragma unroll
          for (int ks = 0; ks < kStepPts / 16; ++ks) {
            // 16 points = two 8-point K groups of 1024 bytes
            const uint64_t ad = sw128_desc_mn(st + ks * 2048, 8192);
            const uint64_t bd = sw128_desc_mn(st + kABytes + ks * 2048, 8192);
            mma_f16_pair(d, ad, bd, prm.idesc, (k > kb || ks > 0) ? 1u : 0u);
          }
          mma_commit_pair_mc(empty_bar(stage), cmask);
          if (++stage == kStages) stage = 0, phase ^= 1u;
        }
        if (!ok) break;
        mma_commit_pair_mc(accf_bar(b), cmask);
      }
      // drain: nothing may still write TMEM when it is freed
      mma_commit_pair(done_bar);
      volatile int no_abort = 0;
      if (!mbar_wait(done_bar, 0, budget, &no_abort)) fail();
    } else if (lane == 0) {
      // ---------------- relay (the odd CTA) ----------------
      // forwards each "accumulator drained" phase of this CTA's epilogue to
      // the even CTA's barrier (an arrive by a thread with no stores in flight)
      uint32_t acc_phase[2] = {0u, 0u};
      const uint32_t remote[2] = {map_to_rank(acce_bar(0), 0), map_to_rank(acce_bar(1), 0)};
      int local = 0;
      for (int64_t u = pair; u < units; u += npairs, ++local) {
        const int b = local & 1;
        if (!mbar_wait(acce_bar(b), acc_phase[b], budget, abort_flag)) {
          fail();
          break;
        }
        acc_phase[b] ^= 1u;
        mbar_arrive_remote(remote[b]);
      }
    }
  } else {
    // ---------------- epilogue warps (both CTAs) ----------------
    const int q = warp & 3;                   // TMEM lane quarter
    const int row = 32 * q + lane;
    uint32_t acc_phase[2] = {0u, 0u};
    int local = 0;
    for (int64_t u = pair; u < units; u += npairs, ++local) {
      int li, mt, nt;
      int64_t kb, ke;
      decode(u, li, mt, nt, kb, ke);
      const int b = local & 1;
      if (!mbar_wait(accf_bar(b), acc_phase[b], budget, abort_flag)) {
        fail();
        break;
      }
      acc_phase[b] ^= 1u;
      tc_fence_after();
      const int s = (int)(u / tiles);
      float *dst = prm.ws + (((size_t)li * prm.S + s) * W + (size_t)mt * kPM + crank * kTM + row) * W +
                   (size_t)nt * kTN;
      const uint32_t t_row = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kTN);
#pragma unroll 1
      for (int c = 0; c < kTN / 32; ++c) {
        uint32_t v[32];
        tmem_ld32_async(t_row + 32 * c, v);
        tmem_wait_ld(v);
        float4 *o = reinterpret_cast<float4 *>(dst + 32 * c);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          o[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                             __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce_bar(b));
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  cluster_sync();    // no CTA leaves (or frees TMEM) while its peer may still use it
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512));
  }
}

// G[gslot][n][k] = sum over s of ws[li][s][n][k], in split order.
__global__ void wgrad_reduce_kernel(const float4 *__restrict__ ws, int S, int W, int layers,
                                    const __grid_constant__ GslotMap gm, float4 *__restrict__ G) {
  const int64_t per = (int64_t)W * W / 4;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < per * layers;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int li = (int)(t / per);
    const int64_t e = t % per;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s = 0; s < S; ++s) {
      const float4 v = ws[((int64_t)li * S + s) * per + e];
      a.x += v.x;
      a.y += v.y;
      a.z += v.z;
      a.w += v.w;
    }
    G[(int64_t)gm.gslot[li] * per + e] = a;
  }
}

bool encode_rows_map(CUtensorMap *map, const void *base, int64_t rows, int W, bool fp16) {
  auto fn = tensor_map_encoder();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)W * 2};
  cuuint32_t box[2] = {64, 64};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

int wgrad_splits(int W, int layers, int64_t n_pad, int num_sms) {
  // about three units per CTA pair
  const int tiles = layers * (W / kPM) * (W / kTN);
  int S = (3 * (num_sms / kCluster) + tiles - 1) / tiles;
  const int64_t ksteps = n_pad / kStepPts;
  if (S > ksteps) S = (int)ksteps;
  return S < 1 ? 1 : S;
}

bool wgrad_supported(int W) { return W == 256 || W == 512; }

cudaError_t launch_wgrad_tc(const WgradJob &job, cudaStream_t s) {
  if (!wgrad_supported(job.W) || job.layers < 1 || job.layers > 64 || job.n_pad <= 0 ||
      job.n_pad % 128 != 0 || job.S < 1)
    return cudaErrorInvalidValue;
  WgradParams p{};
  p.n_pad = job.n_pad;
  p.W = job.W;
  p.layers = job.layers;
  p.S = job.S;
  for (int i = 0; i < job.layers; ++i) {
    p.hslot[i] = job.hslot[i];
    p.dslot[i] = job.dslot[i];
  }
  p.ws = job.ws;
  p.err = job.err;
  p.wait_budget = job.wait_budget;
  p.idesc = idesc_f16(job.fp16, kPM, kTN) | (1u << 15) | (1u << 16);   // A and B MN-major
  CUtensorMap mh, md;
  if (!encode_rows_map(&mh, job.save_h, job.h_rows, job.W, job.fp16) ||
      !encode_rows_map(&md, job.save_d, job.d_rows, job.W, job.fp16))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemBytes);
  if (e != cudaSuccess) return e;
  // one 2-CTA cluster per unit, at most one CTA per SM
  const int64_t units = (int64_t)job.layers * (job.W / kPM) * (job.W / kTN) * job.S;
  const int64_t pairs = job.num_sms / kCluster;
  const int grid = (int)(kCluster * (units < pairs ? units : pairs));
  if (grid < kCluster) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, wgrad_tc_kernel, p, mh, md);
  if (e != cudaSuccess) return e;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  GslotMap gm{};
  for (int i = 0; i < job.layers; ++i) gm.gslot[i] = job.gslot[i];
  const int64_t per = (int64_t)job.W * job.W / 4;
  const int rgrid = (int)((per * job.layers + 255) / 256);
  wgrad_reduce_kernel<<<rgrid < 8 * job.num_sms ? rgrid : 8 * job.num_sms, 256, 0, s>>>(
      reinterpret_cast<const float4 *>(job.ws), job.S, job.W, job.layers, gm,
      reinterpret_cast<float4 *>(job.G));
  return cudaGetLastError();
}

}  // namespace nsdf
