// 16-bit tensor-core form of the fused collision query for the paper's own
// networks (Sec. 4.3): a Fourier-feature input layer gamma(p) =
// [sin(2 pi B p), cos(2 pi B p)] of m = 128 frequencies, then ReLU layers of
// width 256 and one output unit.  BF16 or FP16 operands (one template), FP32
// accumulation in TMEM.
//
// One persistent CTA per SM walks tiles of 128 points.  Per tile the whole
// query of Sec. 3.2 runs on chip:
//   * the epilogue warps evaluate gamma(p) on CUDA cores (FMA phase with its
//     integer part removed exactly, hardware sine and cosine; ff_sincos16 in
//     ff_phase.cuh) and write it as the first A operand,
//   * every layer z_l = W_l x_l (Eq. 1; layer 0 reads gamma(p)) is 16
//     tcgen05.mma (M=128, N=256, K=16; 16-bit x 16-bit -> FP32) into TMEM,
//     A = the 128 x 256 activation tile in shared memory (128-byte swizzled
//     K-major), B = 256 x 64 weight panels streamed by TMA through a 4-stage
//     ring, each panel fetched half by each CTA of a 2-CTA cluster and
//     multicast into both,
//   * the epilogue warps read z from TMEM (tcgen05.ld), add the bias, write
//     max(z, 0) back over A and keep the ReLU's slope, [z > 0], as one bit
//     per unit (4 KB per layer and tile, in a per-CTA slab that stays in L2;
//     shared memory goes to the weight ring),
//   * the last hidden layer's epilogue forms f = w_out . h in FP32 and starts
//     the reverse chain with delta = [z > 0] * w_out,
//   * the Jacobian-transpose chain of Sec. 3.2, g_{l-1} = W_l^T delta_l, runs
//     as the same products against the transposed weights, with
//     delta_{l-1} = [z_{l-1} > 0] * g_{l-1},
//   * layer 0's input gradient g_gamma goes through the feature Jacobian in
//     FP32: grad f = 2 pi sum_j (g_sin,j cos(2 pi b_j.p) - g_cos,j sin(2 pi b_j.p)) b_j,
//   * Eq. 2, the test f < eps and the contact point of Eq. 3 (with the rigid
//     transform of Sec. 4.2) in the final epilogue; float4 stores.
//
// Hand-over: TMEM holds two products (2 x 256 columns), so product g + 1
// may run while the epilogue still reads product g; the epilogue writes the
// next A operand K atom by K atom (64 columns) and announces each atom on its
// own barrier, so the next product starts on atom 0 once a quarter of the
// epilogue is done.  The weight ring fetches the next product's panels
// meanwhile.
//
// The feature tile uses a permuted column order so that each epilogue thread
// evaluates each of its phases once and uses both its sine and its cosine:
// column c = 128 g + 64 s + i holds the sine (s = 0) or cosine (s = 1) of
// frequency j = 64 g + i (ff_feature_of_column); layer 0's weights are packed
// with their columns in that order, and its transposed copy with its rows.
//
// Grouped launches (QueryParams::g_nets > 0) walk a device-built tile list in
// which every body's tiles start on an even index and come in pairs, so that
// the two CTAs of a cluster always share one network's weight panels; the
// tensor maps cover every network of the context (body k at rows
// k * n_hidden * 256), and the epilogue warps reload the small weights and
// the pose when the body changes.  The training form (kSave) also writes the
// features, every h_l and every delta_l out as 16-bit rows for the
// weight-gradient products of the fitting loss (train.cu).
//
// Warp roles (640 threads): warp 0 = TMA producer, warp 1 = MMA issuer and
// TMEM owner, warps 2, 3 idle, warps 4..19 = epilogue (warp w reads TMEM
// lanes 32*(w%4)..+31; the four warps of column group g = (w - 4) / 4 take
// columns 16 g .. 16 g + 15 of every K atom).  Every wait is bounded
// (QueryParams::wait_budget clock cycles); on expiry the kernel records
// kDevTimeout, drains what it has in flight and returns.

#include <cudaTypedefs.h>

#include "nsdf_internal.h"
#include "tc_ptx.cuh"
#include "f32x2.cuh"
#include "ff_phase.cuh"

namespace nsdf {
namespace {

using namespace ptx;

constexpr int kW = 256;                    // network width handled here
constexpr int kFreq = kW / 2;              // Fourier frequencies m
constexpr int kM = 128;                    // points per tile (MMA M, TMEM lanes)
constexpr int kN = 256;                    // MMA N: a whole layer
constexpr int kKAtom = 64;                 // K elements per 128-byte swizzle atom
constexpr int kAtoms = kW / kKAtom;        // 4 weight panels per product
// Weight-panel ring depth.  The panels stream from L2 with a latency of about
// 1.4 us, so the bytes in flight, not the tensor pipe, set the pace of a
// product: the ring takes all the shared memory the activation tile and the
// small FP32 weights leave (the ReLU bits live in a per-CTA slab in global
// memory for that reason).
constexpr int kStages = 4;
constexpr int kMaxHidden = 8;
constexpr int kCluster = 2;
constexpr int kSliceRows = kN / kCluster;
constexpr int kStageBytes = kN * kKAtom * 2;     // 32 KB weight panel
constexpr int kABytes = kM * kW * 2;             // 64 KB activation tile
constexpr int kAtomBytes = kM * kKAtom * 2;      // 16 KB: one K atom of A
// Epilogue threads per TMEM lane: each takes kGroupCols columns of every K atom.
constexpr int kColGroups = 4;
constexpr int kGroupCols = kKAtom / kColGroups;  // 16
constexpr int kEpiWarps = 4 * kColGroups;
// ReLU slope bits of one CTA's tile: 64 bits per row, group and layer
constexpr int kMaskSlabWords = (kMaxHidden - 1) * kColGroups * kM;   // uint2 entries
constexpr int kEpiWarp0 = 4;
constexpr int kThreads = 32 * (kEpiWarp0 + kEpiWarps);
constexpr float kPi = 3.14159265358979324f;

// shared-memory map (bytes from a 1024-aligned base)
constexpr int kOffA = 0;
constexpr int kOffB = kOffA + kABytes;
constexpr int kOffBias = kOffB + kStages * kStageBytes;          // float [kMaxHidden][kW]
constexpr int kOffFreq = kOffBias + kMaxHidden * kW * 4;         // float4 [kFreq]: 2 b_j
constexpr int kOffWout = kOffFreq + kFreq * 16;                  // float [kW]
constexpr int kOffExch = kOffWout + kW * 4;                      // float4 [kColGroups-1][kM]
constexpr int kOffBar = kOffExch + (kColGroups - 1) * kM * 16;
// barriers: full[kStages], empty[kStages], a_ready[kAtoms], d_full, mma_done, x_full, x_empty,
// w_free, w_ready
constexpr int kNumBars = 2 * kStages + kAtoms + 6;
constexpr int kTmemCols = 2 * kN;                 // two products in flight
constexpr int kOffTmemSlot = kOffBar + 8 * kNumBars;
constexpr int kOffAbort = kOffTmemSlot + 4;
constexpr int kSmemBytes = kOffAbort + 4;
static_assert(kSmemBytes <= 232448, "shared memory budget");
static_assert(kAtomBytes == 16384, "store_a_chunk assumes 16 KB atoms");

__device__ __forceinline__ float4 lds4(int off, int idx) {
  extern __shared__ __align__(1024) uint8_t g_smem_ff[];
  return reinterpret_cast<const float4 *>(g_smem_ff + off)[idx];
}

// Tell the MMA issuer (barrier `bar`) that this warp's writes to A, and its
// reads of TMEM, are done.
__device__ __forceinline__ void epi_arrive(uint32_t bar, int lane) {
  fence_proxy_async();
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(bar);
}

// Per-thread state of an epilogue thread for one tile.
struct Epi {
  uint8_t *A;
  uint2 *mask;          // this CTA's ReLU slope bits (global), [layer][column group][row]:
                        // atoms 0, 1 in .x, atoms 2, 3 in .y
  uint32_t t_row;       // TMEM address of lane 32*q, column 0
  uint32_t a_ready;     // barrier a_ready[0]; a_ready[k] is 8 k bytes on
  int r, ch, lane;      // tile row (= TMEM lane); column group (kGroupCols of every atom)
  float px, py, pz;     // query point in the body frame
  // training form: 16-bit rows [slot][n_pad][kW]; h_l in save_h slot l, the
  // features in slot n_hidden, delta_l in save_d slot l; this thread's row
  uint16_t *save_h, *save_d;
  int64_t n_pad, row;
  __device__ __forceinline__ uint2 &bits(int l) const { return mask[(l * kColGroups + ch) * kM + r]; }
  __device__ __forceinline__ void save(uint16_t *base, int slot, int c0, const uint32_t (&w)[kGroupCols / 2]) const {
    if (row >= n_pad) return;   // the fully masked tiles past the last one
    uint4 *dst = reinterpret_cast<uint4 *>(base + ((size_t)slot * n_pad + row) * kW + c0);
    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
  }
};

// One chunk (kGroupCols columns) of a forward epilogue: z = D + b,
// h = max(z, 0); the packed words of the next A operand go to `w` and the
// slope bits are returned.  The last layer adds w_out . h to fpart and
// writes delta = [z > 0] * w_out instead of h.
template <bool kF16, bool LAST, bool kSave = false>
__device__ __forceinline__ uint32_t fwd_chunk(int l, int c0, const uint32_t (&raw)[kGroupCols],
                                              float &fpart, uint32_t (&w)[kGroupCols / 2],
                                              uint32_t (&hx)[kGroupCols / 2]) {
  uint32_t bits = 0;
#pragma unroll
  for (int q = 0; q < kGroupCols / 4; ++q) {
    const float4 b = lds4(kOffBias, (l * kW + c0) / 4 + q);
    float4 wo = make_float4(0.f, 0.f, 0.f, 0.f);
    if (LAST) wo = lds4(kOffWout, c0 / 4 + q);
    const float wv[4] = {wo.x, wo.y, wo.z, wo.w};
    // the bias in f32x2 (scalar FP32 streams slow the products on this SM)
    const float2 z01 = f2_add(make_float2(__uint_as_float(raw[4 * q]), __uint_as_float(raw[4 * q + 1])),
                              make_float2(b.x, b.y));
    const float2 z23 = f2_add(make_float2(__uint_as_float(raw[4 * q + 2]), __uint_as_float(raw[4 * q + 3])),
                              make_float2(b.z, b.w));
    const float zv[4] = {z01.x, z01.y, z23.x, z23.y};
    float v[4], hv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float z = zv[u];
      const bool pos = z > 0.0f;
      bits |= (pos ? 1u : 0u) << (4 * q + u);
      const float h = pos ? z : 0.0f;
      hv[u] = h;
      if (LAST) {
        fpart = fmaf(wv[u], h, fpart);
        v[u] = pos ? wv[u] : 0.0f;
      } else {
        v[u] = h;
      }
    }
    w[2 * q] = pack16<kF16>(v[0], v[1]);
    w[2 * q + 1] = pack16<kF16>(v[2], v[3]);
    if (LAST && kSave) {
      hx[2 * q] = pack16<kF16>(hv[0], hv[1]);
      hx[2 * q + 1] = pack16<kF16>(hv[2], hv[3]);
    }
  }
  return bits;
}

// One chunk of a reverse epilogue: delta = [z > 0] * g.
template <bool kF16>
__device__ __forceinline__ void bwd_chunk(uint32_t bits, const uint32_t (&raw)[kGroupCols],
                                          uint32_t (&w)[kGroupCols / 2]) {
#pragma unroll
  for (int q = 0; q < kGroupCols / 2; ++q) {
    const float g0 = ((bits >> (2 * q)) & 1u) ? __uint_as_float(raw[2 * q]) : 0.0f;
    const float g1 = ((bits >> (2 * q + 1)) & 1u) ? __uint_as_float(raw[2 * q + 1]) : 0.0f;
    w[q] = pack16<kF16>(g0, g1);
  }
}

// Columns of chunk k (0..3) of this thread: kGroupCols columns of K atom k.
// All column groups work through the atoms in order, so atom k of the next
// A operand is complete, and announced on a_ready[k], after a quarter of the
// epilogue, and the next product starts on it while the rest is written.
__device__ __forceinline__ int chunk_col(const Epi &e, int k) { return kKAtom * k + kGroupCols * e.ch; }

// Forward epilogue of layer l, product in TMEM columns dcol..dcol+255 (the
// next chunk's TMEM load is issued while the current one is processed).  In
// the training form the next A operand also goes to save_h slot l (h_l), or,
// for the last layer, to save_d (delta_{L-1}) with h_{L-1} to save_h.
template <bool kF16, bool LAST, bool kSave = false>
__device__ __forceinline__ void fwd_product(const Epi &e, int l, uint32_t dcol, float &fpart) {
  const uint32_t t = e.t_row + dcol;
  uint32_t ra[kGroupCols], rb[kGroupCols], bits[4], w[kGroupCols / 2], hx[kGroupCols / 2];
  auto keep = [&](int k) {
    if constexpr (kSave) {
      if (LAST) {
        e.save(e.save_d, l, chunk_col(e, k), w);
        e.save(e.save_h, l, chunk_col(e, k), hx);
      } else {
        e.save(e.save_h, l, chunk_col(e, k), w);
      }
    }
  };
  tmem_ld16_async(t + chunk_col(e, 0), ra);
#pragma unroll
  for (int k = 0; k < 4; k += 2) {
    tmem_wait_ld(ra);
    tmem_ld16_async(t + chunk_col(e, k + 1), rb);
    bits[k] = fwd_chunk<kF16, LAST, kSave>(l, chunk_col(e, k), ra, fpart, w, hx);
    store_a_cols(e.A, e.r, chunk_col(e, k), w);
    epi_arrive(e.a_ready + 8u * k, e.lane);
    keep(k);
    tmem_wait_ld(rb);
    if (k + 2 < 4) tmem_ld16_async(t + chunk_col(e, k + 2), ra);
    bits[k + 1] = fwd_chunk<kF16, LAST, kSave>(l, chunk_col(e, k + 1), rb, fpart, w, hx);
    store_a_cols(e.A, e.r, chunk_col(e, k + 1), w);
    epi_arrive(e.a_ready + 8u * (k + 1), e.lane);
    keep(k + 1);
  }
  if (!LAST) e.bits(l) = make_uint2(bits[0] | (bits[1] << 16), bits[2] | (bits[3] << 16));
}

// Reverse epilogue of layer l >= 1: delta_{l-1} = [z_{l-1} > 0] * g_{l-1};
// m = the slope bits of layer l-1 (loaded before the product was awaited).
template <bool kF16, bool kSave = false>
__device__ __forceinline__ void bwd_product(const Epi &e, uint2 m, int l, uint32_t dcol) {
  const uint32_t t = e.t_row + dcol;
  const uint32_t bits[4] = {m.x & 0xFFFFu, m.x >> 16, m.y & 0xFFFFu, m.y >> 16};
  uint32_t ra[kGroupCols], rb[kGroupCols], w[kGroupCols / 2];
  tmem_ld16_async(t + chunk_col(e, 0), ra);
#pragma unroll
  for (int k = 0; k < 4; k += 2) {
    tmem_wait_ld(ra);
    tmem_ld16_async(t + chunk_col(e, k + 1), rb);
    bwd_chunk<kF16>(bits[k], ra, w);
    store_a_cols(e.A, e.r, chunk_col(e, k), w);
    epi_arrive(e.a_ready + 8u * k, e.lane);
    if constexpr (kSave) e.save(e.save_d, l - 1, chunk_col(e, k), w);   // delta_{l-1}
    tmem_wait_ld(rb);
    if (k + 2 < 4) tmem_ld16_async(t + chunk_col(e, k + 2), ra);
    bwd_chunk<kF16>(bits[k + 1], rb, w);
    store_a_cols(e.A, e.r, chunk_col(e, k + 1), w);
    epi_arrive(e.a_ready + 8u * (k + 1), e.lane);
    if constexpr (kSave) e.save(e.save_d, l - 1, chunk_col(e, k + 1), w);
  }
}

// gamma(p) for the thread's 2 x kGroupCols frequencies
// j = 64 blk + kGroupCols ch + i: in the permuted column order their sines
// are chunk 2 blk and their cosines chunk 2 blk + 1 of this thread.
template <bool kF16, bool kSave = false>
__device__ __forceinline__ void feature_stage(const Epi &e, int L) {
#pragma unroll 1
  for (int blk = 0; blk < 2; ++blk) {
    uint32_t sw[kGroupCols / 2], cw[kGroupCols / 2];
#pragma unroll
    for (int i = 0; i < kGroupCols; i += 2) {
      const int j = 64 * blk + kGroupCols * e.ch + i;
      const float4 b0 = lds4(kOffFreq, j), b1 = lds4(kOffFreq, j + 1);
      float s0, c0, s1, c1;
      ff_sincos16(b0.x, b0.y, b0.z, e.px, e.py, e.pz, s0, c0);
      ff_sincos16(b1.x, b1.y, b1.z, e.px, e.py, e.pz, s1, c1);
      sw[i / 2] = pack16<kF16>(s0, s1);
      cw[i / 2] = pack16<kF16>(c0, c1);
    }
    store_a_cols(e.A, e.r, chunk_col(e, 2 * blk), sw);
    epi_arrive(e.a_ready + 16u * blk, e.lane);
    store_a_cols(e.A, e.r, chunk_col(e, 2 * blk + 1), cw);
    epi_arrive(e.a_ready + 16u * blk + 8u, e.lane);
    if constexpr (kSave) {
      e.save(e.save_h, L, chunk_col(e, 2 * blk), sw);
      e.save(e.save_h, L, chunk_col(e, 2 * blk + 1), cw);
    }
  }
}

// Layer 0's reverse epilogue: g_gamma (sine and cosine parts of the thread's
// frequencies in chunks 2 blk and 2 blk + 1) through the feature Jacobian,
// accumulated into grad f / pi (the table holds 2 b_j).
__device__ __forceinline__ void feature_jacobian(const Epi &e, uint32_t dcol, float &gx, float &gy,
                                                 float &gz) {
  const uint32_t t = e.t_row + dcol;
#pragma unroll 1
  for (int blk = 0; blk < 2; ++blk) {
    uint32_t us[kGroupCols], uc[kGroupCols];
    tmem_ld16_async(t + chunk_col(e, 2 * blk), us);
    tmem_ld16_async(t + chunk_col(e, 2 * blk + 1), uc);
    tmem_wait_ld(us);
    tmem_wait_ld(uc);   // ties uc's registers to the (already complete) wait
#pragma unroll
    for (int i = 0; i < kGroupCols; ++i) {
      const int j = 64 * blk + kGroupCols * e.ch + i;
      const float4 b = lds4(kOffFreq, j);
      float sn, cs;
      ff_sincos16(b.x, b.y, b.z, e.px, e.py, e.pz, sn, cs);
      const float coef = __uint_as_float(us[i]) * cs - __uint_as_float(uc[i]) * sn;
      gx = fmaf(coef, b.x, gx);
      gy = fmaf(coef, b.y, gy);
      gz = fmaf(coef, b.z, gz);
    }
  }
}

// Tile t of a launch: its network, the index of its first point and how many
// points of that network lie from there on (<= 0: the tile is all masked).
// Grouped launches (g_nets > 0) take network k for the tiles
// g_tile_start[k] <= t < g_tile_start[k + 1]; past the last tile the lookup
// lands on a network whose points are exhausted.
struct TileRef {
  int net;
  int64_t first, valid;
};
__device__ __forceinline__ TileRef tile_ref(const QueryParams &prm, int64_t t) {
  if (prm.g_nets <= 0) return TileRef{0, t * kM, prm.n - t * kM};
  int lo = 0, hi = prm.g_nets;   // the largest k < g_nets with g_tile_start[k] <= t
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prm.g_tile_start[mid] <= t) lo = mid;
    else hi = mid;
  }
  const int64_t lt = t - prm.g_tile_start[lo];
  return TileRef{lo, prm.g_offsets[lo] + lt * kM, prm.g_counts[lo] - lt * kM};
}

// kSave: the training form, which also writes every A operand out
// (QueryParams::save_h / save_d; single-network launches only).
template <bool kF16, bool kSave = false>
__global__ void __launch_bounds__(kThreads, 1)
    query_tc16_ff_kernel(const __grid_constant__ QueryParams prm, const __grid_constant__ CUtensorMap tmap_fwd,
                         const __grid_constant__ CUtensorMap tmap_bwd) {
  extern __shared__ __align__(1024) uint8_t g_smem_ff[];
  uint8_t *smem = g_smem_ff;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if ((smem_u32(smem) & 1023u) != 0) {   // the swizzled layouts need a 1024-aligned base
    if (threadIdx.x == 0) atomicExch(prm.err, kDevTimeout);
    return;
  }
  const uint32_t sA = smem_u32(smem + kOffA), sB = smem_u32(smem + kOffB);
  const uint32_t bar0 = smem_u32(smem + kOffBar);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
  // epilogue -> MMA: K atom k of A written (and the chunks before it read from TMEM)
  const uint32_t a_ready = bar0 + 8u * (2 * kStages);
  const uint32_t d_full = a_ready + 8u * kAtoms;        // MMA -> epilogue: the product is in TMEM
  const uint32_t mma_done = d_full + 8u;
  const uint32_t x_full = mma_done + 8u;    // column groups 1.. have published their partial sums
  const uint32_t x_empty = x_full + 8u;     // column group 0 has consumed them
  // epilogue warps: done with the small weights of the previous network /
  // the next network's small weights are in shared memory
  const uint32_t w_free = x_empty + 8u;
  const uint32_t w_ready = w_free + 8u;
  volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(smem + kOffTmemSlot);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + kOffAbort);
  float4 *exch = reinterpret_cast<float4 *>(smem + kOffExch);

  const int L = prm.n_hidden;
  const int G = 2 * L;                         // products per tile
  const int64_t ntiles = prm.g_nets > 0 ? (int64_t)prm.g_tile_start[prm.g_nets] : (prm.n + kM - 1) / kM;
  const long long budget = prm.wait_budget;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), kCluster);   // freed when every CTA of the cluster consumed it
    }
    for (int k = 0; k < kAtoms; ++k) mbar_init(a_ready + 8u * k, kEpiWarps);
    mbar_init(d_full, 1);
    mbar_init(mma_done, 1);
    mbar_init(x_full, kEpiWarps - 4);   // the warps of column groups 1..
    mbar_init(x_empty, 4);              // the warps of column group 0
    mbar_init(w_free, kEpiWarps);
    mbar_init(w_ready, kEpiWarps);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fence_proxy_async();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(smem + kOffTmemSlot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();      // every CTA's barriers exist before any multicast targets them
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t crank = cluster_rank();
  const uint16_t cmask = (uint16_t)((1u << kCluster) - 1u);
  // every CTA walks the same number of tiles (the cluster's CTAs consume the
  // same weight panels in lockstep); tiles past the end are all-masked
  const int64_t iters = (ntiles + gridDim.x - 1) / gridDim.x;

  auto fail = [&]() {
    atomicExch(prm.err, kDevTimeout);
    *abort_flag = 1;
  };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, issued_parity = 0;   // per stage: a load in flight, its phase
      int64_t load_idx = 0;
      bool ok = true;
      for (int64_t it = 0; ok && it < iters; ++it) {
        const int net = tile_ref(prm, blockIdx.x + it * gridDim.x).net;
        for (int g = 0; ok && g < G; ++g) {
          const bool fwd = g < L;
          const int l = fwd ? g : G - 1 - g;            // network layer of this product
          const CUtensorMap *map = fwd ? &tmap_fwd : &tmap_bwd;
          const int row0 = (net * L + l) * kW;          // the maps cover every network
          for (int k = 0; k < kAtoms; ++k, ++load_idx) {
            if (!mbar_wait(empty_bar(stage), phase ^ 1u, budget, abort_flag)) {
              fail();
              ok = false;
              break;
            }
            if (load_idx != prm.drop_load) {
              mbar_expect_tx(full_bar(stage), kStageBytes);   // both slices land here
              tma_load_2d_mc(sB + stage * kStageBytes + crank * (kSliceRows * kKAtom * 2), map,
                             k * kKAtom, row0 + (int)crank * kSliceRows, full_bar(stage), cmask);
              issued_mask |= 1u << stage;
              issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
            }
            if (++stage == kStages) stage = 0, phase ^= 1u;
          }
        }
      }
      // drain: every issued load must land before the CTA may exit
      for (int s = 0; s < kStages; ++s) {
        if (issued_mask & (1u << s)) {
          volatile int no_abort = 0;
          if (!mbar_wait(full_bar(s), (issued_parity >> s) & 1u, budget, &no_abort)) fail();
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(kF16, kM, kN);
      // descriptors of A atom 0 and ring stage 0; atoms, stages and K steps
      // are constant offsets (addresses below 256 KB: no carry out of the
      // 14-bit address field)
      const uint64_t adesc0 = sw128_desc(sA), bdesc0 = sw128_desc(sB);
      int stage = 0;
      uint32_t phase = 0, a_phase = 0;
      bool ok = true;
      for (int64_t it = 0; ok && it < iters; ++it) {
        for (int g = 0; ok && g < G; ++g) {
          const uint32_t d = tmem + (uint32_t)(kN * (g & 1));   // products alternate buffers
          for (int k = 0; k < kAtoms; ++k) {
            if (!mbar_wait(a_ready + 8u * k, a_phase, budget, abort_flag) ||
                !mbar_wait(full_bar(stage), phase, budget, abort_flag)) {
              fail();
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t ad = adesc0 + (uint64_t)(k * (kAtomBytes >> 4));
            const uint64_t bd = bdesc0 + (uint64_t)(stage * (kStageBytes >> 4));
#pragma unroll
            for (int ks = 0; ks < kKAtom / 16; ++ks)
              mma_f16(d, ad + 2 * ks, bd + 2 * ks, idesc, (k | ks) != 0 ? 1u : 0u);
            mma_commit_mc(empty_bar(stage), cmask);
            if (++stage == kStages) stage = 0, phase ^= 1u;
          }
          if (!ok) break;
          a_phase ^= 1u;
          mma_commit(d_full);
        }
      }
      // drain: no product may still be writing TMEM when it is freed
      mma_commit(mma_done);
      volatile int no_abort = 0;
      if (!mbar_wait(mma_done, 0, budget, &no_abort)) fail();
    }
  } else if (warp >= kEpiWarp0) {
    // ---------------- epilogue warps ----------------
    const int q = warp & 3;                  // TMEM lane quarter
    const int ch = (warp - kEpiWarp0) >> 2;  // column group
    const int r = 32 * q + lane;             // row of the tile = TMEM lane
    Epi e;
    e.A = smem + kOffA;
    e.mask = reinterpret_cast<uint2 *>(prm.scratch) + (size_t)blockIdx.x * kMaskSlabWords;
    e.t_row = tmem + ((uint32_t)(32 * q) << 16);
    e.a_ready = a_ready;
    e.r = r;
    e.ch = ch;
    e.lane = lane;
    e.save_h = prm.save_h;
    e.save_d = prm.save_d;
    e.n_pad = (prm.n + kM - 1) / kM * kM;
    uint32_t d_phase = 0, x_phase = 0, w_phase = 0;
    int cur_net = -1;
    float bout = 0.f;
    bool ok = true;
    // warp-uniform, so that no TMEM load below runs with part of a warp
    auto wait_product = [&]() -> bool {
      const bool got = __all_sync(0xffffffffu, mbar_wait(d_full, d_phase, budget, abort_flag));
      d_phase ^= 1u;
      tc_fence_after();
      return got;
    };
    for (int64_t it = 0; ok && it < iters; ++it) {
      const TileRef tr = tile_ref(prm, blockIdx.x + it * gridDim.x);
      if (tr.net != cur_net) {
        // this network's biases, frequencies (2 b_j) and w_out into shared
        // memory, once every epilogue warp is done with the previous ones
        const bool grouped = prm.g_nets > 0;
        const float *bias = grouped ? prm.g_netptrs[tr.net].bias : prm.bias;
        const float *ffB = grouped ? prm.g_netptrs[tr.net].ffB : prm.ffB;
        const float *wout = grouped ? prm.g_netptrs[tr.net].wout : prm.wout;
        const float *bo = grouped ? prm.g_netptrs[tr.net].bout : prm.bout;
        __syncwarp();
        if (lane == 0) mbar_arrive(w_free);
        if (!__all_sync(0xffffffffu, mbar_wait(w_free, w_phase, budget, abort_flag))) {
          fail(); ok = false; break;
        }
        const int et = threadIdx.x - 32 * kEpiWarp0;     // 0 .. 32 kEpiWarps - 1
        float4 *dst = reinterpret_cast<float4 *>(smem + kOffBias);
        const float4 *bsrc = reinterpret_cast<const float4 *>(bias);
        for (int i = et; i < L * kW / 4; i += 32 * kEpiWarps) dst[i] = __ldg(bsrc + i);
        dst = reinterpret_cast<float4 *>(smem + kOffFreq);
        for (int i = et; i < kFreq; i += 32 * kEpiWarps)
          dst[i] = make_float4(2.f * __ldg(ffB + 3 * i), 2.f * __ldg(ffB + 3 * i + 1),
                               2.f * __ldg(ffB + 3 * i + 2), 0.f);
        dst = reinterpret_cast<float4 *>(smem + kOffWout);
        const float4 *wosrc = reinterpret_cast<const float4 *>(wout);
        for (int i = et; i < kW / 4; i += 32 * kEpiWarps) dst[i] = __ldg(wosrc + i);
        bout = __ldg(bo);
        __syncwarp();
        if (lane == 0) mbar_arrive(w_ready);
        if (!__all_sync(0xffffffffu, mbar_wait(w_ready, w_phase, budget, abort_flag))) {
          fail(); ok = false; break;
        }
        w_phase ^= 1u;
        cur_net = tr.net;
      }
      // this body's rigid pose (Sec. 4.2): T^{-1} rows 0..2 and T[:3,:3]
      const float *Ti = nullptr, *R = nullptr;
      if (prm.g_nets > 0) {
        if (prm.g_T) { Ti = prm.g_T + (size_t)kBodyFloats * tr.net; R = Ti + 12; }
      } else if (prm.has_T) {
        Ti = prm.Ti; R = prm.R;
      }
      const bool valid = r < tr.valid;
      const int64_t idx = tr.first + r;
      e.row = idx;
      float4 pw = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) pw = prm.pts[idx];
      e.px = pw.x; e.py = pw.y; e.pz = pw.z;
      if (Ti) {
        e.px = Ti[0] * pw.x + Ti[1] * pw.y + Ti[2] * pw.z + Ti[3];
        e.py = Ti[4] * pw.x + Ti[5] * pw.y + Ti[6] * pw.z + Ti[7];
        e.pz = Ti[8] * pw.x + Ti[9] * pw.y + Ti[10] * pw.z + Ti[11];
      }
      float fpart = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;

      // product g of the tile sits in TMEM columns kN * (g % 2) ..
      auto dcol = [](int g) { return (uint32_t)(kN * (g & 1)); };

      // ---- gamma(p), the first A operand ----
      feature_stage<kF16, kSave>(e, L);

      // ---- layers 0 .. L-1 (forward): product l ----
      for (int l = 0; ok && l < L; ++l) {
        if (!wait_product()) { fail(); ok = false; break; }
        if (l == L - 1) fwd_product<kF16, true, kSave>(e, l, dcol(l), fpart);
        else fwd_product<kF16, false, kSave>(e, l, dcol(l), fpart);
      }
      // ---- Jacobian-transpose chain: layers L-1 .. 1, product 2L-1-l ----
      for (int l = L - 1; ok && l >= 1; --l) {
        const uint2 m = e.bits(l - 1);    // in flight while the product is awaited
        if (!wait_product()) { fail(); ok = false; break; }
        bwd_product<kF16, kSave>(e, m, l, dcol(G - 1 - l));
      }
      if (!ok) break;
      // ---- layer 0 (product 2L-1): g_gamma through the feature Jacobian ----
      if (!wait_product()) { fail(); ok = false; break; }
      feature_jacobian(e, dcol(G - 1), gx, gy, gz);
      tc_fence_before();
      gx *= kPi; gy *= kPi; gz *= kPi;

      // ---- combine the column groups, normalise, test, project ----
      if (ch != 0) {
        if (!mbar_wait(x_empty, x_phase ^ 1u, budget, abort_flag)) { fail(); ok = false; break; }
        exch[(ch - 1) * kM + r] = make_float4(gx, gy, gz, fpart);
        __syncwarp();
        if (lane == 0) mbar_arrive(x_full);
        x_phase ^= 1u;
        continue;
      }
      if (!mbar_wait(x_full, x_phase, budget, abort_flag)) { fail(); ok = false; break; }
      x_phase ^= 1u;
#pragma unroll
      for (int g = 0; g < kColGroups - 1; ++g) {
        const float4 o = exch[g * kM + r];
        gx += o.x; gy += o.y; gz += o.z; fpart += o.w;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(x_empty);
      if (valid) {
        const float f = fpart + bout;
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
  }
  // every warp ends here: all TMEM traffic is done before the owner frees it,
  // and no CTA leaves while a cluster peer may still multicast into it
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
  }
}

// [rows x 256] 16-bit panels, boxes of 64 columns x kSliceRows rows.
bool encode_map(CUtensorMap *map, void *base, int rows, bool fp16) {
  auto fn = tensor_map_encoder();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kW, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kW * 2};
  cuuint32_t box[2] = {(cuuint32_t)kKAtom, (cuuint32_t)kSliceRows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// CTAs that can be resident at once in whole clusters.
int resident_cluster_ctas(int num_sms) {
  static int cached[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev] < num_sms ? cached[dev] : num_sms;
  cudaFuncSetAttribute(query_tc16_ff_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCluster * 256, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = kSmemBytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, query_tc16_ff_kernel<false, false>, &cfg) != cudaSuccess ||
      clusters < 1) {
    cudaGetLastError();
    clusters = num_sms / kCluster;
  }
  const int ctas = clusters * kCluster;
  if (dev >= 0 && dev < 64) cached[dev] = ctas;
  return ctas < num_sms ? ctas : num_sms;
}

template <bool kF16, bool kSave>
cudaError_t launch_t(const QueryParams &p, const NetDevice &net, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(query_tc16_ff_kernel<kF16, kSave>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  // grouped: p.n = the largest point index + 1; every network may add a
  // partial tile and a pairing tile
  const int grid = p.g_nets > 0
                       ? query_tc16_ff_grouped_grid((p.n + kM - 1) / kM + 2 * (int64_t)p.g_nets, num_sms)
                       : query_tc16_ff_grid(p.n, num_sms);
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
  e = cudaLaunchKernelEx(&cfg, query_tc16_ff_kernel<kF16, kSave>, p, net.tmap_fwd, net.tmap_bwd);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

bool query_tc16_ff_supported(int width, int n_hidden, int ff, int relu) {
  return width == kW && ff == kFreq && relu != 0 && n_hidden >= 1 && n_hidden <= kMaxHidden;
}

size_t query_tc16_ff_scratch_bytes(int grid) { return (size_t)grid * kMaskSlabWords * sizeof(uint2); }

bool make_tc16_ff_tmaps(NetDevice &net, int n_hidden, int rows_nets, bool fp16) {
  if (n_hidden < 1 || n_hidden > kMaxHidden || rows_nets < 1) return false;
  const int rows = rows_nets * n_hidden * kW;
  return encode_map(&net.tmap_fwd, net.fwd16, rows, fp16) &&
         encode_map(&net.tmap_bwd, net.bwd16, rows, fp16);
}

int query_tc16_ff_grid(int64_t n, int num_sms) {
  const int64_t tiles = (n + kM - 1) / kM;
  const int cap = resident_cluster_ctas(num_sms);
  int64_t g = tiles < cap ? tiles : cap;
  g = (g / kCluster) * kCluster;                 // whole clusters
  return (int)(g < kCluster ? kCluster : g);
}

int query_tc16_ff_grouped_grid(int64_t max_tiles, int num_sms) {
  const int cap = resident_cluster_ctas(num_sms);
  int64_t g = max_tiles < cap ? max_tiles : cap;
  g = (g / kCluster) * kCluster;
  return (int)(g < kCluster ? kCluster : g);
}

cudaError_t launch_query_tc16_ff(const QueryParams &p, const NetDevice &net, bool fp16, int num_sms,
                                 cudaStream_t s) {
  if (!query_tc16_ff_supported(p.width, p.n_hidden, p.ff, p.relu)) return cudaErrorInvalidValue;
  if (p.save_h) {
    if (p.g_nets > 0 || !p.save_d) return cudaErrorInvalidValue;
    return fp16 ? launch_t<true, true>(p, net, num_sms, s) : launch_t<false, true>(p, net, num_sms, s);
  }
  return fp16 ? launch_t<true, false>(p, net, num_sms, s) : launch_t<false, false>(p, net, num_sms, s);
}

}  // namespace nsdf
