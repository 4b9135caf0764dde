// 16-bit tensor-core form of the fused collision query for narrow networks:
// width 64, softplus_beta, 2..7 hidden layers, no skip connection (the tiny
// network 3-64-64-64-1 and the multi-body scenes built from it), single
// network or grouped (many bodies in one launch).
//
// At width 64 a hidden product is only 64 MAC per output and the
// activation epilogue dominates, so the layout differs from the width-512
// kernel: every tile of 128 points is worked on by one warpgroup (thread =
// point = TMEM lane), two warpgroups per CTA share the network's 16-bit
// weights in shared memory, and two CTAs share an SM.  Per tile:
//   * L0 (K = 3), every activation and its slope, the output unit, grad f =
//     W_0^T delta_0, Eq. 2, the test f < eps and Eq. 3 (with the rigid
//     transform of Sec. 4.2) run in FP32 on CUDA cores;
//   * each hidden layer z_l = W_l h_{l-1} (Eq. 1) runs as tcgen05.mma
//     (M=128, N=64, K=16) into the tile's TMEM accumulator (64 columns),
//     A = the activation tile in shared memory (128 x 64, 128-byte swizzled
//     K-major), B = W_l (64 x 64, the same layout);
//   * the Jacobian-transpose chain g_{l-1} = W_l^T delta_l reads the same
//     copy of W_l as an MN-major B operand (no transposed copy);
//   * the slopes sigmoid(beta z) are parked in TMEM (FP16 pairs, 32 columns
//     per layer) until the reverse chain needs them.
// Precision.  One BF16 rounding of the 64-wide weights already moves f by up
// to ~2.8e-3 on these networks (and of the activations by more), against a
// target of 2e-3.  The forward products are cheap at this width, so in BF16
// they take split operands, a = a_hi + a_lo and W = W_hi + W_lo with every
// part a BF16 value, as three products A_hi W_hi + A_lo W_hi + A_hi W_lo
// (the A_lo W_lo term is below FP32 rounding of the sum), and so do the
// reverse products (deltas and W_l split alike: single BF16 operands let the
// normal of a 7-layer network drift past 1e-2 rad).  FP16 (3 more
// significand bits) takes single operands throughout.
//
// Work: tiles of 128 points, handed out in pairs (one per warpgroup); a
// grouped launch rounds every body's tile count up to even, so a pair never
// straddles two networks, and each CTA takes a contiguous range of pairs,
// reloading the weights only when its range crosses into another body.
// Every mbarrier wait is bounded (QueryParams::wait_budget); on expiry the
// kernel records kDevTimeout and returns.

#include <cudaTypedefs.h>

#include "nsdf_internal.h"
#include "softplus.cuh"
#include "tc_ptx.cuh"

namespace nsdf {
namespace {

using namespace ptx;

constexpr int kW = 64;
constexpr int kM = 128;                   // points per tile = TMEM lanes
constexpr int kTilesPerCta = 2;           // one per warpgroup
constexpr int kThreads = 128 * kTilesPerCta;
constexpr int kMaxHidden = 7;
constexpr int kWBytes = kW * kW * 2;      // one layer's 16-bit weights (8 KB)
constexpr int kABytes = kM * kW * 2;      // one A operand (16 KB)
// FP32 weights kept in shared memory: W_0 [64][3], biases [n_hidden][64],
// w_out [64], b_out
constexpr int kSmallFloats = kW * 3 + kMaxHidden * kW + kW + 4;

// Shared-memory map (bytes from a 1024-aligned base) for n_hidden = L.
struct Layout {
  int whi, wlo, a, a_stride, small, bars, slot, total;
};
__host__ __device__ inline Layout layout(int L, bool split) {
  Layout o{};
  const int nh = L - 1;
  o.whi = 0;
  o.wlo = o.whi + nh * kWBytes;
  o.a = o.wlo + (split ? nh * kWBytes : 0);
  o.a = (o.a + 1023) & ~1023;
  o.a_stride = split ? 2 * kABytes : kABytes;       // A_hi (then A_lo) per tile
  o.small = o.a + kTilesPerCta * o.a_stride;
  o.bars = o.small + kSmallFloats * 4;
  o.slot = o.bars + 8 * kTilesPerCta;
  o.total = o.slot + 16;
  return o;
}
// TMEM columns of one tile: the accumulator (64) and the parked slopes of
// layers 0 .. L-2 (32 columns of FP16 pairs each); the CTA allocates a power
// of two of at least both tiles' columns.
__host__ __device__ inline int tile_cols(int L) { return kW + (L - 1) * 32; }
__host__ __device__ inline int cta_cols(int L) {
  const int need = kTilesPerCta * tile_cols(L);
  int c = 32;
  while (c < need) c <<= 1;
  return c;
}

// Store 16 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16};\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// MN-major operand descriptor (128-byte swizzle): 64-element MN blocks `lbo`
// bytes apart, 8-row K groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc_mn(uint32_t saddr, uint32_t lbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Named barriers 1 and 2 (one per warpgroup), with immediate IDs: a barrier
// ID in a register makes the compiler reserve all 16 barriers of the CTA,
// which limits an SM to one CTA.
__device__ __forceinline__ void wg_bar(int wg) {
  if (wg == 0) asm volatile("bar.sync 1, 128;\n" ::: "memory");
  else asm volatile("bar.sync 2, 128;\n" ::: "memory");
}
// Barrier of the warpgroup that also ANDs a predicate over its 128 threads,
// so that all of them take the same path after a bounded wait.
__device__ __forceinline__ bool wg_all(int wg, bool v) {
  uint32_t res;
  if (wg == 0)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred p, 1, 128, p;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(res)
        : "r"((uint32_t)v)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred p, 2, 128, p;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(res)
        : "r"((uint32_t)v)
        : "memory");
  return res != 0;
}

template <bool kF16>
__device__ __forceinline__ float from16(uint32_t w, bool hi) {
  const uint16_t b = hi ? (uint16_t)(w >> 16) : (uint16_t)w;
  if constexpr (kF16) return __half2float(*reinterpret_cast<const __half *>(&b));
  return __uint_as_float((uint32_t)b << 16);
}

// Pack 32 FP32 values of a row into A words (and, split, the words of the
// residuals a - a_hi), then store them at columns c0..c0+31.
template <bool kF16, bool kSplit>
__device__ __forceinline__ void store_a(uint8_t *Ahi, uint8_t *Alo, int r, int c0,
                                        const float (&v)[32]) {
  uint32_t hw[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) hw[j] = pack16<kF16>(v[2 * j], v[2 * j + 1]);
  store_a_chunk(Ahi, r, c0, hw);
  if constexpr (kSplit) {
    uint32_t lw[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
      lw[j] = pack16<kF16>(v[2 * j] - from16<kF16>(hw[j], false),
                           v[2 * j + 1] - from16<kF16>(hw[j], true));
    store_a_chunk(Alo, r, c0, lw);
  }
}

template <bool kF16>
__global__ void __launch_bounds__(kThreads, 2)
    query_w64_kernel(const __grid_constant__ QueryParams prm) {
  constexpr bool kSplit = !kF16;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  const int L = prm.n_hidden, nh = L - 1;
  const Layout lay = layout(L, kSplit);
  const int tid = threadIdx.x;
  const int wg = tid >> 7, r = tid & 127, q = r >> 5, lane = tid & 31;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar = sbase + lay.bars + 8u * wg;
  volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(smem + lay.slot);
  float *sm = reinterpret_cast<float *>(smem + lay.small);
  float *sW0 = sm, *sB = sm + kW * 3, *sWo = sB + kMaxHidden * kW, *sBo = sWo + kW;
  uint8_t *Ahi = smem + lay.a + wg * lay.a_stride;
  uint8_t *Alo = Ahi + kABytes;
  const long long budget = prm.wait_budget;
  volatile int no_abort = 0;

  if (tid == 0) {
    for (int b = 0; b < kTilesPerCta; ++b) mbar_init(sbase + lay.bars + 8u * b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  const uint32_t ncols = (uint32_t)cta_cols(L);
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     sbase + lay.slot),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // this thread's TMEM row: accumulator at column 0, slopes of layer j at 64 + 32 j
  const uint32_t tb = tmem + (uint32_t)(wg * tile_cols(L)) + ((uint32_t)(32 * q) << 16);

  const bool grouped = prm.g_nets > 0;
  const int64_t tiles = grouped ? (int64_t)prm.g_tile_start[prm.g_nets] : (prm.n + kM - 1) / kM;
  const int64_t pairs = (tiles + 1) / 2;
  const int64_t p0 = pairs * blockIdx.x / gridDim.x, p1 = pairs * (blockIdx.x + 1) / gridDim.x;
  const float neg_bl2e = -prm.beta * 1.4426950408889634f, inv_beta = 1.0f / prm.beta;
  const uint32_t idesc_f = idesc_f16(kF16, kM, kW);
  const uint32_t idesc_r = idesc_f | (1u << 16);          // B (W_l read as W_l^T) MN-major
  uint32_t phase = 0;
  bool ok = true;
  int loaded = -1;
  int round = 0;      // product rounds issued by this warpgroup (for the test-only drop)

  // one round of products into the tile's accumulator, then wait for it; the
  // result is the same for every thread of the warpgroup
  auto mma_round = [&](int l, bool reverse) -> bool {
    fence_proxy_async();
    tc_fence_before();
    wg_bar(wg);
    tc_fence_after();
    if (r == 0) {
      const uint32_t a0 = smem_u32(Ahi), al = smem_u32(Alo);
      const uint32_t w0 = sbase + lay.whi + (l - 1) * kWBytes;
      const uint32_t w1 = sbase + lay.wlo + (l - 1) * kWBytes;
      const uint32_t d = tmem + (uint32_t)(wg * tile_cols(L));
#pragma unroll
      for (int ks = 0; ks < kW / 16; ++ks) {
        if (!reverse) {
          mma_f16(d, sw128_desc(a0 + 32 * ks), sw128_desc(w0 + 32 * ks), idesc_f, ks > 0 ? 1u : 0u);
          if constexpr (kSplit) {
            mma_f16(d, sw128_desc(al + 32 * ks), sw128_desc(w0 + 32 * ks), idesc_f, 1u);
            mma_f16(d, sw128_desc(a0 + 32 * ks), sw128_desc(w1 + 32 * ks), idesc_f, 1u);
          }
        } else {
          // K = the layer's outputs n: W_l rows, 16 rows = two 1024-byte groups
          mma_f16(d, sw128_desc(a0 + 32 * ks), sw128_desc_mn(w0 + 2048 * ks, 8192), idesc_r,
                  ks > 0 ? 1u : 0u);
          if constexpr (kSplit) {
            mma_f16(d, sw128_desc(al + 32 * ks), sw128_desc_mn(w0 + 2048 * ks, 8192), idesc_r, 1u);
            mma_f16(d, sw128_desc(a0 + 32 * ks), sw128_desc_mn(w1 + 2048 * ks, 8192), idesc_r, 1u);
          }
        }
      }
      if (round != prm.drop_load) mma_commit(bar);
    }
    ++round;
    const bool done = wg_all(wg, mbar_wait(bar, phase, budget, &no_abort));
    if (done) phase ^= 1u;
    tc_fence_after();
    return done;
  };

  for (int64_t pr = p0; pr < p1; ++pr) {
    // both warpgroups go on only if neither has given up
    if (!__syncthreads_and(ok ? 1 : 0)) {
      ok = false;
      break;
    }
    // ---- the network of this pair; reload its weights when it changes ----
    int k = 0;
    if (grouped) {
      int lo = 0, hi = prm.g_nets;            // tile_start[lo] <= 2 pr < tile_start[hi]
      const int32_t t0 = (int32_t)(2 * pr);
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prm.g_tile_start[mid] <= t0) lo = mid;
        else hi = mid;
      }
      k = lo;
    }
    if (k != loaded) {
      // (the barrier above: no product of either tile still reads the old weights)
      const uint16_t *w16 = grouped ? prm.g_netptrs[k].w16 : prm.fwd16;
      const uint16_t *w16lo = grouped ? prm.g_netptrs[k].w16lo : prm.fwd16_lo;
      const float *gw0 = grouped ? prm.g_netptrs[k].w0 : prm.w0;
      const float *gb = grouped ? prm.g_netptrs[k].bias : prm.bias;
      const float *gwo = grouped ? prm.g_netptrs[k].wout : prm.wout;
      const float *gbo = grouped ? prm.g_netptrs[k].bout : prm.bout;
      // 16-bit weights: row n of layer i (64 values = 8 chunks of 16 B) into
      // the 128-byte swizzle (chunk j of row n at j ^ (n % 8))
      for (int e = tid; e < nh * kW * 8; e += kThreads) {
        const int i = e / (kW * 8), n = (e / 8) % kW, j = e % 8;
        const size_t src = ((size_t)i * kW + n) * kW + 8 * j;
        const int dst = i * kWBytes + n * 128 + ((j ^ (n & 7)) * 16);
        *reinterpret_cast<uint4 *>(smem + lay.whi + dst) = __ldg(reinterpret_cast<const uint4 *>(w16 + src));
        if constexpr (kSplit)
          *reinterpret_cast<uint4 *>(smem + lay.wlo + dst) =
              __ldg(reinterpret_cast<const uint4 *>(w16lo + src));
      }
      for (int e = tid; e < kW * 3; e += kThreads) sW0[e] = __ldg(gw0 + e);
      for (int e = tid; e < L * kW; e += kThreads) sB[e] = __ldg(gb + e);
      for (int e = tid; e < kW; e += kThreads) sWo[e] = __ldg(gwo + e);
      if (tid == 0) sBo[0] = __ldg(gbo);
      fence_proxy_async();
      __syncthreads();
      loaded = k;
    }

    // ---- this warpgroup's tile and row ----
    const int64_t t = 2 * pr + wg;
    int64_t idx;
    bool valid;
    if (grouped) {
      const int64_t toff = t - prm.g_tile_start[k];
      const int64_t within = toff * kM + r;
      idx = prm.g_offsets[k] + within;
      valid = within < prm.g_counts[k];
    } else {
      idx = t * kM + r;
      valid = idx < prm.n;
    }
    float4 pw = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) pw = prm.pts[idx];
    float px = pw.x, py = pw.y, pz = pw.z;
    const float *Ti = nullptr, *R = nullptr;
    if (grouped && prm.g_T) {
      Ti = prm.g_T + (size_t)kBodyFloats * k;
      R = Ti + 12;
    } else if (!grouped && prm.has_T) {
      Ti = prm.Ti;
      R = prm.R;
    }
    if (Ti) {
      px = Ti[0] * pw.x + Ti[1] * pw.y + Ti[2] * pw.z + Ti[3];
      py = Ti[4] * pw.x + Ti[5] * pw.y + Ti[6] * pw.z + Ti[7];
      pz = Ti[8] * pw.x + Ti[9] * pw.y + Ti[10] * pw.z + Ti[11];
    }

    // ---- L0 on CUDA cores ----
#pragma unroll 1
    for (int c0 = 0; c0 < kW; c0 += 32) {
      float h[32];
      uint32_t sw[16];
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        float s2[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int c = c0 + j + u;
          const float z = fmaf(sW0[3 * c], px, fmaf(sW0[3 * c + 1], py, fmaf(sW0[3 * c + 2], pz, sB[c])));
          act_f32(z, neg_bl2e, inv_beta, h[j + u], s2[u]);
        }
        sw[j >> 1] = pack16<true>(s2[0], s2[1]);
      }
      store_a<kF16, kSplit>(Ahi, Alo, r, c0, h);
      tmem_st16(tb + kW + (c0 >> 1), sw);
    }
    tmem_wait_st();
    float f = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;

    // ---- hidden layers (forward) ----
    for (int l = 1; ok && l < L; ++l) {
      if (!mma_round(l, false)) { ok = false; break; }
      const bool last = (l == L - 1);
#pragma unroll 1
      for (int c0 = 0; c0 < kW; c0 += 32) {
        uint32_t raw[32];
        tmem_ld32_async(tb + c0, raw);
        tmem_wait_ld(raw);
        float h[32];
        uint32_t sw[16];
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
          float s2[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int c = c0 + j + u;
            act_f32(__uint_as_float(raw[j + u]) + sB[l * kW + c], neg_bl2e, inv_beta, h[j + u], s2[u]);
            if (last) {
              f = fmaf(sWo[c], h[j + u], f);
              h[j + u] = s2[u] * sWo[c];            // delta_{L-1}
            }
          }
          sw[j >> 1] = pack16<true>(s2[0], s2[1]);
        }
        if (last) {
          store_a<kF16, kSplit>(Ahi, Alo, r, c0, h);  // delta_{L-1}: the reverse chain's A
        } else {
          store_a<kF16, kSplit>(Ahi, Alo, r, c0, h);
          tmem_st16(tb + kW + 32 * l + (c0 >> 1), sw);
        }
      }
      if (!last) tmem_wait_st();
    }

    // ---- Jacobian-transpose chain: layers L-1 .. 1 ----
    for (int l = L - 1; ok && l >= 1; --l) {
      if (!mma_round(l, true)) { ok = false; break; }
#pragma unroll 1
      for (int c0 = 0; c0 < kW; c0 += 32) {
        uint32_t raw[32], sl[16];
        tmem_ld32_async(tb + c0, raw);
        tmem_ld16_async(tb + kW + 32 * (l - 1) + (c0 >> 1), sl);
        tmem_wait_ld(raw);
        tmem_wait_ld(sl);
        float dv[32];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float2 s2 = __half22float2(*reinterpret_cast<const __half2 *>(&sl[j]));
          dv[2 * j] = s2.x * __uint_as_float(raw[2 * j]);
          dv[2 * j + 1] = s2.y * __uint_as_float(raw[2 * j + 1]);
        }
        if (l > 1) {
          store_a<kF16, kSplit>(Ahi, Alo, r, c0, dv);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {         // grad f = W_0^T delta_0
            const int c = c0 + j;
            gx = fmaf(dv[j], sW0[3 * c], gx);
            gy = fmaf(dv[j], sW0[3 * c + 1], gy);
            gz = fmaf(dv[j], sW0[3 * c + 2], gz);
          }
        }
      }
    }
    if (!ok) continue;        // the barrier at the top of the loop ends both warpgroups

    // ---- Eq. 2, the test and Eq. 3 ----
    if (valid) {
      f += sBo[0];
      const float nrm = sqrtf(gx * gx + gy * gy + gz * gz);
      float nx = 0.f, ny = 0.f, nz = 0.f;
      if (nrm >= 1e-20f) { nx = gx / nrm; ny = gy / nrm; nz = gz / nrm; }
      if (!prm.collide) {
        if (prm.raw_gradient) { nx = gx; ny = gy; nz = gz; }
        prm.out_n_sdf[idx] = make_float4(nx, ny, nz, f);
      } else {
        if (R) {
          const float wx = R[0] * nx + R[1] * ny + R[2] * nz;
          const float wy = R[3] * nx + R[4] * ny + R[5] * nz;
          const float wz = R[6] * nx + R[7] * ny + R[8] * nz;
          nx = wx; ny = wy; nz = wz;
        }
        const bool hit = f < prm.eps;
        float4 p = pw;
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
  if (!ok && lane == 0) atomicExch(prm.err, kDevTimeout);
  // drain: every product of the warpgroup has completed before TMEM is freed
  // (after a timed-out round a last commit completes the pending phase)
  if (r == 0) mma_commit(bar);
  if (!wg_all(wg, mbar_wait(bar, phase, budget, &no_abort)) && lane == 0)
    atomicExch(prm.err, kDevTimeout);
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (tid < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols));
  }
}

// Dynamic shared memory of a launch: the layout, plus padding so that no
// more CTAs share an SM than their TMEM columns allow (a CTA whose
// allocation cannot be met would wait for another CTA to exit).
template <bool kF16>
int launch_smem(int L, int num_sms_unused) {
  (void)num_sms_unused;
  const int need = layout(L, !kF16).total + 1024;
  const int fit = 512 / cta_cols(L);                 // CTAs whose TMEM fits one SM
  // 233472 bytes of shared memory per SM, 1 KB reserved per CTA
  const int cap = 233472 / (fit + 1) - 1024 + 16;
  return need > cap ? need : cap;
}

// CTAs per SM: as many as the SM's registers, shared memory and TMEM
// columns hold (computed from the device's limits and the kernel's register
// count).
template <bool kF16>
int resident_ctas(int L) {
  const int smem = launch_smem<kF16>(L, 0);
  int dev = 0, smem_sm = 0, regs_sm = 0;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, query_w64_kernel<kF16>) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int by_smem = smem_sm / (smem + 1024);                 // 1 KB reserved per CTA
  const int by_regs = regs_sm / (fa.numRegs * kThreads);
  int fit = 512 / cta_cols(L);
  if (by_smem < fit) fit = by_smem;
  if (by_regs < fit) fit = by_regs;
  return fit;
}

template <bool kF16>
cudaError_t launch_t(const QueryParams &p, int num_sms, int ctas_per_sm, cudaStream_t s) {
  const int L = p.n_hidden;
  const int smem = launch_smem<kF16>(L, num_sms);
  if (smem > 232448) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(query_w64_kernel<kF16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int fit = resident_ctas<kF16>(L);
  if (fit < 1) return cudaErrorInvalidConfiguration;
  const int cps = (ctas_per_sm <= 0 || ctas_per_sm > fit) ? fit : ctas_per_sm;
  int64_t grid = (int64_t)num_sms * cps;
  if (p.g_nets == 0) {
    const int64_t pairs = ((p.n + kM - 1) / kM + 1) / 2;
    if (pairs < grid) grid = pairs;
  }
  if (grid < 1) grid = 1;
  query_w64_kernel<kF16><<<(int)grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

bool query_w64_supported(int width, int n_hidden, int skip) {
  return width == kW && n_hidden >= 2 && n_hidden <= kMaxHidden && skip <= 0;
}

int query_w64_ctas_per_sm(int n_hidden, bool fp16) {
  return fp16 ? resident_ctas<true>(n_hidden) : resident_ctas<false>(n_hidden);
}

cudaError_t launch_query_w64(const QueryParams &p, bool fp16, int num_sms, int ctas_per_sm,
                             cudaStream_t s) {
  if (!query_w64_supported(p.width, p.n_hidden, p.skip)) return cudaErrorInvalidValue;
  return fp16 ? launch_t<true>(p, num_sms, ctas_per_sm, s) : launch_t<false>(p, num_sms, ctas_per_sm, s);
}

}  // namespace nsdf
