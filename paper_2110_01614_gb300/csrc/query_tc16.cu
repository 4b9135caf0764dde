// 16-bit tensor-core form of the fused collision query (width-512 networks):
// BF16 or FP16 operands (one template), FP32 accumulation in TMEM.
//
// One persistent CTA per SM walks tiles of 128 points.  Per tile the whole
// query of Sec. 3.2 runs on chip:
//   * L0 (K = 3) on CUDA cores in the epilogue warps,
//   * each hidden layer z_l = W_l x_l (Eq. 1) as 64 tcgen05.mma
//     (M=128, N=256, K=16; 16-bit x 16-bit -> FP32) into TMEM, A = the
//     activation tile resident in shared memory (128 x 512, 128-byte
//     swizzled K-major), B = 256 x 64 weight panels streamed by TMA
//     through a 2-stage ring, each panel fetched half by each CTA of a
//     2-CTA cluster and multicast into both,
//   * the epilogue warps read z from TMEM (tcgen05.ld), add the bias (the
//     biases, W_0, the skip weights on p and w_out sit in shared memory)
//     and write softplus_beta(z) back as the next A operand, and park what
//     the reverse chain needs in a per-CTA scratch slab (FP16,
//     lane-contiguous, stored evict-first in L2): the slope sigmoid(beta z)
//     in the FP16 form, the activation itself in the BF16 form (below),
//   * the skip connection's input columns p/sqrt(2) never pass through the
//     16-bit operands: their product with W_s is added in FP32 on CUDA
//     cores, and their gradient is accumulated in FP32 from delta_s,
//   * the output unit f = w_out . h_7 is an FP32 dot in the last epilogue,
//   * the Jacobian-transpose chain (back-propagation of Sec. 3.2):
//     delta_l = sigmoid(beta z_l) * g_l, g_{l-1} = W_l^T delta_l as the same
//     tcgen05 products against the transposed weights, the skip
//     connection's 1/sqrt(2) split, and grad f = W_0^T delta_0 in FP32,
//   * Eq. 2, the test f < eps and the contact point of Eq. 3 (with the
//     rigid transform of Sec. 4.2) in the final epilogue; float4 stores.
// A training form of the same kernel (kSave) also writes every A operand out
// for the weight-gradient products of the fitting loss (train.cu).
//
// Queries run in the CTA-pair form (kPair): the two CTAs of a cluster take
// consecutive tiles, and the even CTA issues every product as M=256
// tcgen05.mma over both (cta_group::2: each CTA's A rows, each CTA's 128
// rows of the weight panel).  Each CTA then streams half a panel per
// product step (a 4-stage ring of 16 KB in the same 64 KB), and the odd
// CTA's epilogue hand-overs reach the even CTA's barriers through a relay
// thread.  The training form keeps one CTA per product (2-stage ring of
// 32 KB panels, each fetched half by each CTA and multicast).
//
// FP32 arithmetic of the epilogues (biases, the FP32 layers, the deltas and
// the running sums) is issued as f32x2 pairs: scalar FP32 FMA-pipe streams
// on the SM slow the products (softplus.cuh).
//
// BF16 operand rounding and its first-order correction.  Rounding the
// 512-wide activations to BF16's 8-bit significand at each tensor-core layer
// moves f by up to ~3.2e-3 on the body-scale network, while weight rounding
// alone moves it by ~1.5e-3.  To first order, the change of f caused by
// replacing an A operand element a by its rounded value a~ is
// (df/da) (a - a~), and df/da for every element of every A operand is exactly
// what the Jacobian-transpose chain forms: the reverse product W_l^T delta_l
// lands in TMEM as df/dA_{l-1}.  So the BF16 form parks the activation a
// itself (FP16) in the scratch slab instead of its slope, writes its BF16
// rounding (round to nearest even) as the A operand, repeats that rounding in
// the reverse epilogue by an integer operation on the FP16 encoding (the same
// value for every normal FP16 number), and there (1) derives the slope as
// sigmoid(beta z) = 1 - e^{-beta h} (h = softplus_beta(z)) and (2) adds
// sum (df/da) (a - a~) to f.  The slab keeps its size; the FP16 form (3 more
// significand bits) needs no correction and parks its slopes.

#include <cudaTypedefs.h>

#include <atomic>

#include "nsdf_debug.h"
#include "nsdf_internal.h"
#include "softplus.cuh"
#include "tc_ptx.cuh"

namespace nsdf {
namespace {

using namespace ptx;

constexpr int kW = 512;                    // network width handled here
constexpr int kM = 128;                    // points per tile (MMA M, TMEM lanes)
constexpr int kN = 256;                    // MMA N (one half of a layer)
constexpr int kKAtom = 64;                 // K elements per 128-byte swizzle atom
// Weight-panel ring depth of the one-CTA form: two 32 KB stages leave room
// for the small FP32 weights below.
constexpr int kStages = 2;
// CTA-pair form (cta_group::2): each product is one M=256 MMA chain over the
// two CTAs' tiles, issued by the even CTA; each CTA holds its 128 rows of a
// weight panel (16 KB), so the same 64 KB of ring make 4 stages.  (A fifth
// stage, made room for by reading W_0, the skip weights and w_out through L1,
// measured 0.3% faster than 4 with the same L1 reads, which cost 2%.)
constexpr int kStagesPair = 4;
// The biases of the first kMaxHidden layers, W_0, the skip layer's weights on
// p and w_out stay in shared memory (30 KB, FP32); deeper layers read their
// biases from global memory.
constexpr int kMaxHidden = 8;
// CTAs per cluster sharing every weight panel: each CTA fetches 1/kCluster of
// the panel's rows and the TMA multicasts it into all of them, so L2 streams
// each panel once per cluster instead of once per CTA.
constexpr int kCluster = 2;
constexpr int kSliceRows = 256 / kCluster;
constexpr int kStageBytes = kN * kKAtom * 2;          // 32 KB weight panel
constexpr int kStageBytesPair = kStageBytes / 2;      // 16 KB: this CTA's rows of a panel
static_assert(kStagesPair * kStageBytesPair == kStages * kStageBytes, "same ring in both forms");
constexpr int kABytes = kM * kW * 2;                  // 128 KB activation tile
constexpr int kAtomBytes = kM * kKAtom * 2;           // 16 KB: one K atom of A
constexpr int kLoadsPerLayer = (kW / kN) * (kW / kKAtom);   // 16
constexpr int kEpiWarps = 8;
constexpr int kEpiWarp0 = 4;              // epilogue = warpgroups 1 and 2
constexpr int kThreads = 32 * (kEpiWarp0 + kEpiWarps);
// Register split.  The kernel is launched with kLaunchRegs registers per
// thread (the most 384 threads can have); warpgroup 0 (producer, MMA issuer,
// two idle warps) gives registers back down to kCtlRegs and the epilogue
// warpgroups take them up to kEpiRegs.  The shares must not exceed what the
// launch holds, or the increase would wait for registers that never come;
// the host refuses to launch a build whose register count differs.
constexpr int kLaunchRegs = 168;
constexpr int kCtlRegs = 40;
constexpr int kEpiRegs = 232;
static_assert(128 * kCtlRegs + 32 * kEpiWarps * kEpiRegs <= kThreads * kLaunchRegs,
              "register split exceeds the registers of the launch");
static_assert(kThreads * kLaunchRegs <= 65536, "launch registers exceed the SM");
constexpr float kInvSqrt2 = 0.70710678118654752f;
constexpr float kSqrt2 = 1.41421356237309515f;

// shared-memory map (bytes from a 1024-aligned base)
constexpr int kOffA = 0;
constexpr int kOffB = kOffA + kABytes;
constexpr int kOffBias = kOffB + kStages * kStageBytes;   // float [kMaxHidden][kW]
constexpr int kOffW0 = kOffBias + kMaxHidden * kW * 4;     // float [kW][3]
constexpr int kOffWsk = kOffW0 + kW * 3 * 4;               // float [3][kW]: W_s[:, kW - 3 + j]
constexpr int kOffWout = kOffWsk + 3 * kW * 4;             // float [kW]
constexpr int kOffBar = kOffWout + kW * 4;
// barriers: full[stages], empty[stages], a_lo, a_hi_a, a_hi_b, d0_full,
// d1_full, lo_free_a, lo_free_b, mma_done, x_full, x_empty
constexpr int kNumBars = 2 * kStagesPair + 10;

// K atom taken at position pos (0..7) of column half nh.  Epilogue thread
// group g (0, 1) writes atoms 4h + 2g (its first two chunks) and 4h + 2g + 1
// of a half h, so atoms 4h and 4h + 2 are ready, and may be overwritten,
// before 4h + 1 and 4h + 3.  Half 0 takes atoms 0..3 (written by the previous
// epilogue's half 0), then 4, 6, 5, 7; half 1 takes 0, 2, 1, 3 (freeing
// them for this epilogue's half 0 in that order), then 4..7.
__device__ __forceinline__ int k_atom(int nh, int pos) {
  const int sw = (pos & 4) | ((pos & 1) << 1) | ((pos >> 1) & 1);
  return (nh == 0) == (pos < 4) ? pos : sw;
}
constexpr int kOffTmemSlot = kOffBar + 8 * kNumBars;
constexpr int kOffAbort = kOffTmemSlot + 4;
constexpr int kOffExch = ((kOffAbort + 4 + 15) / 16) * 16;   // float4 [kM]
constexpr int kSmemBytes = kOffExch + kM * 16;
static_assert(kSmemBytes <= 232448, "shared memory budget");

// Operand format of the 16-bit products (FP16 or BF16), and the unpacking of
// a packed pair.
template <bool kF16>
struct Op {
  static constexpr uint32_t idesc = idesc_f16(kF16, kM, kN);
  static __device__ __forceinline__ uint32_t pack(float lo, float hi) { return pack16<kF16>(lo, hi); }
  static __device__ __forceinline__ float2 unpack(uint32_t u) {
    if constexpr (kF16) {
      __half2 t = *reinterpret_cast<__half2 *>(&u);
      return __half22float2(t);
    } else {
      __nv_bfloat162 t = *reinterpret_cast<__nv_bfloat162 *>(&u);
      return __bfloat1622float2(t);
    }
  }
};

// Slopes are written once and read once, up to a tile-time later; all CTAs
// together keep about 136 MB of them in flight, more than L2 holds.  They are
// stored with an L2 evict-first policy so that they, and not the weight
// panels and biases every CTA re-reads, give way when L2 is full; each
// 128-byte line is discarded from L2 after its single read, so dead slopes
// are never written back to HBM.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void st_slope(uint4 *dst, uint4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;\n" ::"l"(dst), "r"(v.x),
               "r"(v.y), "r"(v.z), "r"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void l2_discard_line(const void *line) {
  asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(line) : "memory");
}
__device__ __forceinline__ void l2_prefetch_bulk(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"(bytes) : "memory");
}

// Two elements at once in packed FP16 (used where the result is rounded to 16
// bits anyway): u = 2^(-beta log2(e) |z|) on the MUFU in f16x2, log1p(u) =
// u P(u) with the same polynomial in HFMA2, and the slope as
// sigmoid(beta z) = (1 + tanh(beta z / 2)) / 2 with tanh in f16x2.  The
// pre-activation is rounded to FP16 first (relative 2^-11).
__device__ __forceinline__ __half2 h2_ex2(__half2 x) {
  uint32_t y, xi = *reinterpret_cast<uint32_t *>(&x);
  asm("ex2.approx.f16x2 %0, %1;\n" : "=r"(y) : "r"(xi));
  return *reinterpret_cast<__half2 *>(&y);
}
__device__ __forceinline__ __half2 h2_tanh(__half2 x) {
  uint32_t y, xi = *reinterpret_cast<uint32_t *>(&x);
  asm("tanh.approx.f16x2 %0, %1;\n" : "=r"(y) : "r"(xi));
  return *reinterpret_cast<__half2 *>(&y);
}
struct ActH2 {          // per-kernel constants of act_h2
  __half2 neg_bl2e, inv_beta, half_beta;
  __half2 neg_bl2e_s2;  // -beta log2(e) sqrt(2): slope of the layer feeding the skip
};
__device__ __forceinline__ void act_h2(float z0, float z1, const ActH2 &k, __half2 &h, __half2 &s) {
  const __half2 zh = __floats2half2_rn(z0, z1);
  const __half2 u = h2_ex2(__hmul2(__habs2(zh), k.neg_bl2e));
  __half2 p = __float2half2_rn(-2.344365580e-02f);
  p = __hfma2(p, u, __float2half2_rn(1.001397327e-01f));
  p = __hfma2(p, u, __float2half2_rn(-2.090795360e-01f));
  p = __hfma2(p, u, __float2half2_rn(3.248495807e-01f));
  p = __hfma2(p, u, __float2half2_rn(-4.993146523e-01f));
  p = __hfma2(p, u, __float2half2_rn(9.999905920e-01f));
  h = __hfma2(__hmul2(u, p), k.inv_beta, __hmax2(zh, __float2half2_rn(0.0f)));
  const __half2 half = __float2half2_rn(0.5f);
  s = __hfma2(h2_tanh(__hmul2(zh, k.half_beta)), half, half);
}
__device__ __forceinline__ uint32_t h2_bits(__half2 v) { return *reinterpret_cast<uint32_t *>(&v); }

// Two FP32 values as FP16x2 (lo -> low half), saturating at +-65504.
__device__ __forceinline__ __half2 h2_sat(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(hi), "f"(lo));
  return *reinterpret_cast<__half2 *>(&d);
}
// BF16 form: both FP16 values of a pair (non-negative, finite) rounded to
// 8 significant bits, to nearest even, on their FP16 encoding (the carry of
// the low half cannot reach the high half for such values).  For normal
// FP16 values this is the BF16 rounding that the forward epilogue applied
// to the A operand (bf16_of_h2), so the reverse epilogue gets the operand's
// residual without it; for FP16 subnormals (below 6.1e-5) the two differ by
// at most 2^-21, which the correction then carries.
__device__ __forceinline__ uint32_t rnd8_h2(uint32_t x) {
  return (x + 0x00030003u + ((x >> 3) & 0x00010001u)) & 0xfff8fff8u;
}
// The BF16 A word of an FP16 pair: each value rounded to nearest even (the
// conversion to FP32 is exact).  Converting directly instead of after
// rnd8_h2 saves four integer instructions per pair (BF16 query 7.36 ->
// 7.16 ms per 1M points).
__device__ __forceinline__ uint32_t bf16_of_h2(uint32_t a) {
  const float2 f = __half22float2(*reinterpret_cast<__half2 *>(&a));
  return pack16<false>(f.x, f.y);
}
// softplus_beta of a pair in packed FP16, without its slope (the BF16 form
// keeps the activation and derives the slope in the reverse epilogue).
__device__ __forceinline__ __half2 act_h2_h(float z0, float z1, const ActH2 &k) {
  const __half2 zh = __floats2half2_rn(z0, z1);
  const __half2 u = h2_ex2(__hmul2(__habs2(zh), k.neg_bl2e));
  __half2 p = __float2half2_rn(-2.344365580e-02f);
  p = __hfma2(p, u, __float2half2_rn(1.001397327e-01f));
  p = __hfma2(p, u, __float2half2_rn(-2.090795360e-01f));
  p = __hfma2(p, u, __float2half2_rn(3.248495807e-01f));
  p = __hfma2(p, u, __float2half2_rn(-4.993146523e-01f));
  p = __hfma2(p, u, __float2half2_rn(9.999905920e-01f));
  return __hfma2(__hmul2(u, p), k.inv_beta, __hmax2(zh, __float2half2_rn(0.0f)));
}

// The kernel's dynamic shared memory (same base as the kernel's own view).
extern __shared__ __align__(1024) uint8_t g_smem[];

// Floats idx..idx+3 of the small-weight array at byte offset `off` of shared
// memory (a plain load: the compiler may schedule it freely).
__device__ __forceinline__ float4 lds4(int off, int idx) {
  return *reinterpret_cast<const float4 *>(g_smem + off + 4 * idx);
}
// Bias floats idx..idx+3 of layer l (idx counts from layer 0).
__device__ __forceinline__ float4 bias4(const float *gbias, int l, int idx) {
  return l < kMaxHidden ? lds4(kOffBias, idx)
                        : __ldg(reinterpret_cast<const float4 *>(gbias + idx));
}
__device__ __forceinline__ float comp(const float4 &v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
__device__ __forceinline__ uint32_t comp_u(const uint4 &v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Running sums of an epilogue thread: grad f (partial) and f (partial), each
// as two partial sums (even and odd columns, accumulated in f32x2).
struct Acc {
  float2 gx = {0.f, 0.f}, gy = {0.f, 0.f}, gz = {0.f, 0.f}, f = {0.f, 0.f};
};
__device__ __forceinline__ float2 pair_of(const float4 &v, int u) {   // components u, u + 1
  return u == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w);
}
__device__ __forceinline__ float2 raw_pair(const uint32_t (&raw)[32], int i) {
  return make_float2(__uint_as_float(raw[i]), __uint_as_float(raw[i + 1]));
}

// The waits an epilogue of column half 0 passes before it overwrites A:
// part 0 (its first two chunks, atoms 0 and 2) once half 1 has read atoms
// 0 and 2, part 1 (atoms 1 and 3) once half 1 has read those.
struct Gate {
  uint32_t bar0, bar1, parity;
  long long budget;
  volatile int *abort;
  bool pending0, pending1, ok;
  __device__ __forceinline__ void pass(int part) {
    if (part ? pending1 : pending0) {
      const uint32_t bar = part ? bar1 : bar0;
      if (part) pending1 = false;
      else pending0 = false;
      ok = (mbar_try_wait<true>(bar, parity) || mbar_wait<true>(bar, parity, budget, abort)) && ok;
      tc_fence_after();
    }
  }
  __device__ __forceinline__ void pass_all() {
    pass(0);
    pass(1);
  }
};

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
  uint8_t *slab;        // this CTA's slope slab
  uint32_t t_row;       // TMEM address of lane 32*q, column 0
  int r, ch;            // tile row (= TMEM lane); which 128 columns of each half
  float neg_bl2e, inv_beta;
  float px, py, pz;     // query point in the body frame
  const float *gbias;   // [n_hidden][W] biases in global memory
  uint64_t pol;         // L2 evict-first policy for slope stores
  int lane;
  ActH2 kh;             // packed-FP16 activation constants
  // save mode (training): every A operand also goes to [n_hidden][n_pad][W]
  // 16-bit arrays, activations h_l to save_h[l], deltas to save_d[l]
  uint16_t *save_h, *save_d;
  int64_t n_pad, row;   // rows of a saved layer; this thread's row in it
  // slab words of layer l, columns 8g..8g+7 (16 B) of this row: FP16 slopes
  // (FP16 form) or FP16 activations (BF16 form)
  __device__ __forceinline__ uint4 *slope(int l, int g) const {
    return reinterpret_cast<uint4 *>(slab + (((size_t)l * (kW / 8) + g) * kM + r) * 16);
  }
};

constexpr int kNShort = kW - 3;

// Save mode: columns c0..c0+31 of this row of layer `slot` of a saved array.
// Rows past n_pad belong to the fully masked tiles that every CTA walks so
// that the cluster's CTAs stay in step; they are not saved.
__device__ __forceinline__ void save_chunk(const Epi &e, uint16_t *base, int slot, int c0,
                                           const uint32_t (&w)[16]) {
  if (e.row >= e.n_pad) return;
  uint4 *dst = reinterpret_cast<uint4 *>(base + (((size_t)slot * e.n_pad + e.row) * kW + c0));
#pragma unroll
  for (int t = 0; t < 4; ++t) dst[t] = make_uint4(w[4 * t], w[4 * t + 1], w[4 * t + 2], w[4 * t + 3]);
}

// One 32-column chunk of a forward epilogue (layers 1 .. L-1).
// The 16 packed words of the next A operand go to `hw`; the caller stores them.
// In save mode the last layer's activations h_{L-1} (its A words hold
// delta_{L-1}) go to `hx`.
template <bool kF16, bool LAST, bool AT_SKIP, bool FEEDS_SKIP, bool kSave = false>
__device__ __forceinline__ void fwd_chunk(const Epi &e, int l, int c0, const uint32_t (&raw)[32],
                                          Acc &acc, uint32_t (&hw)[16], uint32_t (&hx)[16]) {
  const int b = l * kW + c0;     // bias index
  uint32_t sw[16];               // slab words: FP16 slopes (FP16 form) / activations (BF16)
  if constexpr (!LAST && !FEEDS_SKIP) {
    // activations and slopes in packed FP16; slopes are kept as FP16 in the slab
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 bq = bias4(e.gbias, l, b + 4 * q);
      float4 s0, s1, s2;
      if (AT_SKIP) {
        s0 = lds4(kOffWsk, c0 + 4 * q);
        s1 = lds4(kOffWsk, kW + c0 + 4 * q);
        s2 = lds4(kOffWsk, 2 * kW + c0 + 4 * q);
      }
      float z[4];
#pragma unroll
      for (int u = 0; u < 4; u += 2) {    // in f32x2
        float2 zz = f2_add(raw_pair(raw, 4 * q + u), pair_of(bq, u));
        if (AT_SKIP)
          zz = f2_fma(f2_splat(kInvSqrt2),
                      f2_fma(pair_of(s0, u), f2_splat(e.px),
                             f2_fma(pair_of(s1, u), f2_splat(e.py), f2_mul(pair_of(s2, u), f2_splat(e.pz)))),
                      zz);
        z[u] = zz.x;
        z[u + 1] = zz.y;
      }
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        if constexpr (kF16) {
          __half2 h, sl;
          act_h2(z[2 * v], z[2 * v + 1], e.kh, h, sl);
          hw[2 * q + v] = h2_bits(h);
          sw[2 * q + v] = h2_bits(sl);
        } else {
          const uint32_t hb = h2_bits(act_h2_h(z[2 * v], z[2 * v + 1], e.kh));
          hw[2 * q + v] = bf16_of_h2(hb);
          sw[2 * q + v] = hb;
        }
      }
    }
    const int g0 = c0 >> 3;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      st_slope(e.slope(l, g0 + t), make_uint4(sw[4 * t], sw[4 * t + 1], sw[4 * t + 2], sw[4 * t + 3]),
               e.pol);
  } else {
    // the layer feeding the skip connection and the last layer: FP32 activation
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 bq = bias4(e.gbias, l, b + 4 * q);
      float4 wq = make_float4(0.f, 0.f, 0.f, 0.f), s0, s1, s2;
      if (LAST) wq = lds4(kOffWout, c0 + 4 * q);
      if (AT_SKIP) {
        s0 = lds4(kOffWsk, c0 + 4 * q);
        s1 = lds4(kOffWsk, kW + c0 + 4 * q);
        s2 = lds4(kOffWsk, 2 * kW + c0 + 4 * q);
      }
      float hv[4], sv[4];
#pragma unroll
      for (int u = 0; u < 4; u += 2) {    // columns u, u + 1 in f32x2
        const int c = c0 + 4 * q + u;
        float2 z = f2_add(raw_pair(raw, 4 * q + u), pair_of(bq, u));
        if (AT_SKIP)    // the skip input columns p / sqrt(2), in FP32
          z = f2_fma(f2_splat(kInvSqrt2),
                     f2_fma(pair_of(s0, u), f2_splat(e.px),
                            f2_fma(pair_of(s1, u), f2_splat(e.py), f2_mul(pair_of(s2, u), f2_splat(e.pz)))),
                     z);
        float2 h, sl;
        act_f32x2(z, e.neg_bl2e, e.inv_beta, h, sl);
        if (LAST) {
          const float2 wo = pair_of(wq, u);
          acc.f = f2_fma(wo, h, acc.f);
          if constexpr (kSave) hx[2 * q + (u >> 1)] = Op<kF16>::pack(h.x, h.y);
          h = f2_mul(sl, wo);                        // delta_{L-1}
          if (AT_SKIP) {                             // delta_s feeds the direct term
            acc.gx = f2_fma(h, f2_mul(pair_of(s0, u), f2_splat(kInvSqrt2)), acc.gx);
            acc.gy = f2_fma(h, f2_mul(pair_of(s1, u), f2_splat(kInvSqrt2)), acc.gy);
            acc.gz = f2_fma(h, f2_mul(pair_of(s2, u), f2_splat(kInvSqrt2)), acc.gz);
          }
        } else if (FEEDS_SKIP) {
          const float2 hs = f2_mul(h, f2_splat(kInvSqrt2));
          h = make_float2(c < kNShort ? hs.x : 0.0f, c + 1 < kNShort ? hs.y : 0.0f);
        }
        hv[u] = h.x; hv[u + 1] = h.y;
        sv[u] = sl.x; sv[u + 1] = sl.y;
      }
      if constexpr (!kF16 && !LAST) {
        // BF16 form: the activation as FP16 into the slab, its 8-bit rounding as A
        sw[2 * q] = h2_bits(__floats2half2_rn(hv[0], hv[1]));
        sw[2 * q + 1] = h2_bits(__floats2half2_rn(hv[2], hv[3]));
        hw[2 * q] = bf16_of_h2(sw[2 * q]);
        hw[2 * q + 1] = bf16_of_h2(sw[2 * q + 1]);
      } else {
        hw[2 * q] = Op<kF16>::pack(hv[0], hv[1]);
        hw[2 * q + 1] = Op<kF16>::pack(hv[2], hv[3]);
        sw[2 * q] = Op<true>::pack(sv[0], sv[1]);
        sw[2 * q + 1] = Op<true>::pack(sv[2], sv[3]);
      }
    }
    if constexpr (!LAST) {
      const int g0 = c0 >> 3;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        st_slope(e.slope(l, g0 + t), make_uint4(sw[4 * t], sw[4 * t + 1], sw[4 * t + 2], sw[4 * t + 3]),
                 e.pol);
    }
  }
}

// A forward epilogue over the thread's 128 columns of column half h, TMEM
// loads double-buffered; after the first two chunks it arrives on `mid`
// (when non-zero).
template <bool kF16, bool LAST, bool AT_SKIP, bool FEEDS_SKIP, bool kSave>
__device__ __forceinline__ void fwd_half(const Epi &e, int l, int h, Acc &acc, Gate &gate,
                                         uint32_t mid) {
  uint32_t ra[32], rb[32];
  const int cbase = 256 * h + 128 * e.ch;
  tmem_ld32_async(e.t_row + cbase, ra);
  // save mode: h_l (or, in the last layer, delta_{L-1} and h_{L-1})
  auto save = [&](int c0, const uint32_t (&hw)[16], const uint32_t (&hx)[16]) {
    if constexpr (kSave) {
      if (LAST) {
        save_chunk(e, e.save_d, l, c0, hw);
        save_chunk(e, e.save_h, l, c0, hx);
      } else {
        save_chunk(e, e.save_h, l, c0, hw);
      }
    }
  };
  // unrolling left to the compiler: faster than both "unroll 1" and a full
  // unroll on the 1M-point workload (7.42 / 7.49 / 7.87 ms)
  for (int cc = 0; cc < 4; cc += 2) {
    uint32_t hw[16], hx[16];
    tmem_wait_ld(ra);
    tmem_ld32_async(e.t_row + cbase + 32 * (cc + 1), rb);
    fwd_chunk<kF16, LAST, AT_SKIP, FEEDS_SKIP, kSave>(e, l, cbase + 32 * cc, ra, acc, hw, hx);
    gate.pass(cc >> 1);
    store_a_chunk(e.A, e.r, cbase + 32 * cc, hw);
    save(cbase + 32 * cc, hw, hx);
    tmem_wait_ld(rb);
    if (cc + 2 < 4) tmem_ld32_async(e.t_row + cbase + 32 * (cc + 2), ra);
    fwd_chunk<kF16, LAST, AT_SKIP, FEEDS_SKIP, kSave>(e, l, cbase + 32 * (cc + 1), rb, acc, hw, hx);
    store_a_chunk(e.A, e.r, cbase + 32 * (cc + 1), hw);
    save(cbase + 32 * (cc + 1), hw, hx);
    if (cc == 0 && mid != 0u) epi_arrive(mid, e.lane);
  }
}

// L0 (K = 3) on CUDA cores: no TMEM, same epilogue.
template <bool kF16, bool FEEDS_SKIP, bool kSave>
__device__ __forceinline__ void layer0(const Epi &e) {
#pragma unroll 1
  for (int cc = 0; cc < 8; ++cc) {
    const int c0 = 256 * e.ch + 32 * cc;
    uint32_t hw[16], sw[16];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 bq = lds4(kOffBias, c0 + 4 * q);
      const float4 w_a = lds4(kOffW0, 3 * (c0 + 4 * q));       // 12 weights of 4 columns
      const float4 w_b = lds4(kOffW0, 3 * (c0 + 4 * q) + 4);
      const float4 w_c = lds4(kOffW0, 3 * (c0 + 4 * q) + 8);
      const float w[12] = {w_a.x, w_a.y, w_a.z, w_a.w, w_b.x, w_b.y,
                           w_b.z, w_b.w, w_c.x, w_c.y, w_c.z, w_c.w};
      float hv[4], sv[4];
#pragma unroll
      for (int v = 0; v < 2; ++v) {       // columns 2v, 2v + 1 of the four, in f32x2
        const int u = 2 * v;
        const float2 z = f2_fma(make_float2(w[3 * u], w[3 * u + 3]), f2_splat(e.px),
                                f2_fma(make_float2(w[3 * u + 1], w[3 * u + 4]), f2_splat(e.py),
                                       f2_fma(make_float2(w[3 * u + 2], w[3 * u + 5]), f2_splat(e.pz),
                                              make_float2(comp(bq, u), comp(bq, u + 1)))));
        float2 h2, s2;
        act_f32x2(z, e.neg_bl2e, e.inv_beta, h2, s2);
        if (FEEDS_SKIP) {
          const float2 hs = f2_mul(h2, f2_splat(kInvSqrt2));
          const int c = c0 + 4 * q + u;
          h2 = make_float2(c < kNShort ? hs.x : 0.0f, c + 1 < kNShort ? hs.y : 0.0f);
        }
        hv[u] = h2.x; hv[u + 1] = h2.y;
        sv[u] = s2.x; sv[u + 1] = s2.y;
      }
      if constexpr (kF16) {
        hw[2 * q] = Op<kF16>::pack(hv[0], hv[1]);
        hw[2 * q + 1] = Op<kF16>::pack(hv[2], hv[3]);
        sw[2 * q] = Op<true>::pack(sv[0], sv[1]);
        sw[2 * q + 1] = Op<true>::pack(sv[2], sv[3]);
      } else {
        sw[2 * q] = h2_bits(__floats2half2_rn(hv[0], hv[1]));
        sw[2 * q + 1] = h2_bits(__floats2half2_rn(hv[2], hv[3]));
        hw[2 * q] = bf16_of_h2(sw[2 * q]);
        hw[2 * q + 1] = bf16_of_h2(sw[2 * q + 1]);
      }
    }
    store_a_chunk(e.A, e.r, c0, hw);
    if constexpr (kSave) save_chunk(e, e.save_h, 0, c0, hw);
#pragma unroll
    for (int t = 0; t < 4; ++t)
      st_slope(e.slope(0, (c0 >> 3) + t), make_uint4(sw[4 * t], sw[4 * t + 1], sw[4 * t + 2], sw[4 * t + 3]),
               e.pol);
  }
}

// One 32-column chunk of a reverse epilogue: delta_{l-1} = slope_{l-1} * g.
// The 16 packed words of the next A operand go to `dw` (unused for TO_INPUT).
// In the BF16 form the slab holds the FP16 activation a of layer l-1 (its
// A operand before rounding): the slope is sigmoid(beta z) = 1 - e^{-beta h}
// (h = a, or sqrt(2) a for the layer feeding the skip connection), and the
// chunk also adds its share of the first-order correction of f for the
// rounding of A_{l-1}: raw = W_l^T delta_l is df/dA_{l-1} (before the skip
// connection's 1/sqrt(2) split) and a - rnd8(a) the residual of the rounded
// operand.  The products are summed in packed FP16 with the residuals scaled
// by 2^10 (exact; df/dA saturates at 65504 and a non-finite chunk sum is
// dropped).
template <bool kF16, bool AT_SKIP, bool MAKES_SKIP_DELTA, bool TO_INPUT>
__device__ __forceinline__ void bwd_chunk(const Epi &e, int c0, const uint32_t (&raw)[32],
                                          const uint4 (&sl)[4], Acc &acc, uint32_t (&dw)[16]) {
  float sv_all[32];
  if constexpr (!kF16) {
    __half2 c0h = __float2half2_rn(0.0f), c1h = c0h;
    const __half2 kexp = AT_SKIP ? e.kh.neg_bl2e_s2 : e.kh.neg_bl2e;
    const __half2 one = __float2half2_rn(1.0f);
    const __half2 k1024 = __float2half2_rn(1024.0f);     // keeps the products above FP16's subnormals
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t hb = comp_u(sl[j >> 2], j & 3);      // activations of columns 2j, 2j+1
      const __half2 a = *reinterpret_cast<const __half2 *>(&hb);
      const uint32_t ab = rnd8_h2(hb);
      const __half2 r = __hmul2(__hsub2(a, *reinterpret_cast<const __half2 *>(&ab)), k1024);
      const __half2 g = h2_sat(__uint_as_float(raw[2 * j]), __uint_as_float(raw[2 * j + 1]));
      if (j & 1) c1h = __hfma2(r, g, c1h);
      else c0h = __hfma2(r, g, c0h);
      const float2 s2 = __half22float2(__hsub2(one, h2_ex2(__hmul2(a, kexp))));
      sv_all[2 * j] = s2.x;
      sv_all[2 * j + 1] = s2.y;
    }
    const float2 cs = __half22float2(__hadd2(c0h, c1h));
    const float c = cs.x + cs.y;
    if (isfinite(c)) acc.f.x = fmaf(c, 1.0f / 1024.0f, acc.f.x);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float4 s0, s1, s2, w_a, w_b, w_c;
    if (MAKES_SKIP_DELTA) {
      s0 = lds4(kOffWsk, c0 + 4 * q);
      s1 = lds4(kOffWsk, kW + c0 + 4 * q);
      s2 = lds4(kOffWsk, 2 * kW + c0 + 4 * q);
    }
    if (TO_INPUT) {
      w_a = lds4(kOffW0, 3 * (c0 + 4 * q));
      w_b = lds4(kOffW0, 3 * (c0 + 4 * q) + 4);
      w_c = lds4(kOffW0, 3 * (c0 + 4 * q) + 8);
    }
    float sv[4];
    if constexpr (kF16) {
      const uint32_t swords[2] = {comp_u(sl[q >> 1], 2 * (q & 1)), comp_u(sl[q >> 1], 2 * (q & 1) + 1)};
      const float2 sa = Op<true>::unpack(swords[0]);     // slopes are FP16 in the slab
      const float2 sb = Op<true>::unpack(swords[1]);
      sv[0] = sa.x; sv[1] = sa.y; sv[2] = sb.x; sv[3] = sb.y;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) sv[u] = sv_all[4 * q + u];
    }
    float dv[4];
#pragma unroll
    for (int u = 0; u < 4; u += 2) {    // columns u, u + 1 in f32x2
      const int c = c0 + 4 * q + u;
      float2 g = raw_pair(raw, 4 * q + u);
      if (AT_SKIP) {
        const float2 gs = f2_mul(g, f2_splat(kInvSqrt2));
        g = make_float2(c < kNShort ? gs.x : 0.0f, c + 1 < kNShort ? gs.y : 0.0f);
      }
      const float2 d = f2_mul(make_float2(sv[u], sv[u + 1]), g);
      if (MAKES_SKIP_DELTA) {                      // direct path to the input
        acc.gx = f2_fma(d, f2_mul(pair_of(s0, u), f2_splat(kInvSqrt2)), acc.gx);
        acc.gy = f2_fma(d, f2_mul(pair_of(s1, u), f2_splat(kInvSqrt2)), acc.gy);
        acc.gz = f2_fma(d, f2_mul(pair_of(s2, u), f2_splat(kInvSqrt2)), acc.gz);
      }
      if (TO_INPUT) {
        const float w[12] = {w_a.x, w_a.y, w_a.z, w_a.w, w_b.x, w_b.y,
                             w_b.z, w_b.w, w_c.x, w_c.y, w_c.z, w_c.w};
        acc.gx = f2_fma(d, make_float2(w[3 * u], w[3 * u + 3]), acc.gx);
        acc.gy = f2_fma(d, make_float2(w[3 * u + 1], w[3 * u + 4]), acc.gy);
        acc.gz = f2_fma(d, make_float2(w[3 * u + 2], w[3 * u + 5]), acc.gz);
      }
      dv[u] = d.x;
      dv[u + 1] = d.y;
    }
    dw[2 * q] = Op<kF16>::pack(dv[0], dv[1]);
    dw[2 * q + 1] = Op<kF16>::pack(dv[2], dv[3]);
  }
}

// After a chunk's slab words have been consumed, drop their L2 lines: the
// warp's 32 rows x 4 groups (columns c0..c0+31) cover 16 lines of 128 bytes,
// one per lane 0..15.
__device__ __forceinline__ void discard_chunk(const Epi &e, int l, int c0) {
  __syncwarp();
  if (e.lane < 16) {
    const int g = (c0 >> 3) + (e.lane >> 2);
    const int row0 = (e.r & ~31) + 8 * (e.lane & 3);
    const uint8_t *line = e.slab + (((size_t)l * (kW / 8) + g) * kM + row0) * 16;
    l2_discard_line(line);
  }
}

// A reverse epilogue over the thread's 128 columns of column half h: TMEM
// loads and the slopes of the next chunk are fetched while the current chunk
// is processed; after the first two chunks it arrives on `mid` (when
// non-zero).
template <bool kF16, bool AT_SKIP, bool MAKES_SKIP_DELTA, bool TO_INPUT, bool kSave>
__device__ __forceinline__ void bwd_half(const Epi &e, int l, int h, Acc &acc, Gate &gate,
                                         uint32_t mid) {
  uint32_t ra[32], rb[32];
  uint4 sa[4], sb[4];
  const int cbase = 256 * h + 128 * e.ch;
  const int g0 = cbase >> 3;
#pragma unroll
  for (int t = 0; t < 4; ++t) sa[t] = *e.slope(l - 1, g0 + t);
  tmem_ld32_async(e.t_row + cbase, ra);
#pragma unroll 1
  for (int cc = 0; cc < 4; cc += 2) {
#pragma unroll
    for (int t = 0; t < 4; ++t) sb[t] = *e.slope(l - 1, g0 + 4 * (cc + 1) + t);
    uint32_t dw[16];
    tmem_wait_ld(ra);
    tmem_ld32_async(e.t_row + cbase + 32 * (cc + 1), rb);
    bwd_chunk<kF16, AT_SKIP, MAKES_SKIP_DELTA, TO_INPUT>(e, cbase + 32 * cc, ra, sa, acc, dw);
    if (!TO_INPUT) {
      gate.pass(cc >> 1);
      store_a_chunk(e.A, e.r, cbase + 32 * cc, dw);
    }
    if constexpr (kSave) save_chunk(e, e.save_d, l - 1, cbase + 32 * cc, dw);   // delta_{l-1}
    discard_chunk(e, l - 1, cbase + 32 * cc);
    if (cc + 2 < 4) {
#pragma unroll
      for (int t = 0; t < 4; ++t) sa[t] = *e.slope(l - 1, g0 + 4 * (cc + 2) + t);
    }
    tmem_wait_ld(rb);
    if (cc + 2 < 4) tmem_ld32_async(e.t_row + cbase + 32 * (cc + 2), ra);
    bwd_chunk<kF16, AT_SKIP, MAKES_SKIP_DELTA, TO_INPUT>(e, cbase + 32 * (cc + 1), rb, sb, acc, dw);
    if (!TO_INPUT) store_a_chunk(e.A, e.r, cbase + 32 * (cc + 1), dw);
    if constexpr (kSave) save_chunk(e, e.save_d, l - 1, cbase + 32 * (cc + 1), dw);
    discard_chunk(e, l - 1, cbase + 32 * (cc + 1));
    if (cc == 0 && mid != 0u) epi_arrive(mid, e.lane);
  }
}

// kSave: the training form, which also writes every layer's A operand out
// (QueryParams::save_h / save_d) for the weight-gradient products.
// kPair: the CTA-pair form (M=256 products over the cluster's two tiles,
// issued by the even CTA; the odd CTA's hand-overs are forwarded to the even
// CTA's barriers by a relay thread).
template <bool kF16, bool kSave = false, bool kPair = false>
__global__ void __launch_bounds__(kThreads, 1)
    query_tc16_kernel(const QueryParams prm, const __grid_constant__ CUtensorMap tmap_fwd,
                      const __grid_constant__ CUtensorMap tmap_bwd) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = smem_raw;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if ((smem_u32(smem) & 1023u) != 0) {   // the swizzled layouts need a 1024-aligned base
    if (threadIdx.x == 0) atomicExch(prm.err, kDevTimeout);
    return;
  }
  uint8_t *A = smem + kOffA;
  const uint32_t sA = smem_u32(A), sB = smem_u32(smem + kOffB);
  const uint32_t bar0 = smem_u32(smem + kOffBar);
  constexpr int S = kPair ? kStagesPair : kStages;          // ring stages
  constexpr int SB = kPair ? kStageBytesPair : kStageBytes;  // bytes of a stage in this CTA
  const uint32_t crank = cluster_rank();
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
  // epilogue -> MMA: A atoms 0..3 written (and TMEM half 0 read); atoms 4, 6;
  // atoms 5, 7 (and TMEM half 1 read)
  const uint32_t a_lo = bar0 + 8u * (2 * S);
  const uint32_t a_hi_a = a_lo + 8u;
  const uint32_t a_hi_b = a_hi_a + 8u;
  // MMA -> epilogue: column half 0 / 1 of the product in TMEM; half 1 has
  // read A atoms 0, 2 / atoms 1, 3
  const uint32_t d0_full = a_hi_b + 8u;
  const uint32_t d1_full = d0_full + 8u;
  const uint32_t lo_free_a = d1_full + 8u;
  const uint32_t lo_free_b = lo_free_a + 8u;
  const uint32_t mma_done = lo_free_b + 8u;
  const uint32_t x_full = mma_done + 8u;    // column-half 1 has published its partial sums
  const uint32_t x_empty = x_full + 8u;     // column-half 0 has consumed them
  volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(smem + kOffTmemSlot);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + kOffAbort);
  float4 *exch = reinterpret_cast<float4 *>(smem + kOffExch);

  const int L = prm.n_hidden;
  const int G = 2 * (L - 1);                   // tensor-core layers per tile
  const int64_t ntiles = (prm.n + kM - 1) / kM;
  const long long budget = prm.wait_budget;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), 1);
      // freed when every CTA of the cluster consumed it (pair: the even CTA's
      // products read both CTAs' stages; its commit reaches both)
      mbar_init(empty_bar(s), kPair ? 1 : kCluster);
    }
    // pair: the even CTA's gates also count the odd CTA's relayed arrival
    const uint32_t gate_count = kEpiWarps + ((kPair && crank == 0) ? 1 : 0);
    mbar_init(a_lo, gate_count);
    mbar_init(a_hi_a, gate_count);
    mbar_init(a_hi_b, gate_count);
    mbar_init(d0_full, 1);
    mbar_init(d1_full, 1);
    mbar_init(lo_free_a, 1);
    mbar_init(lo_free_b, 1);
    mbar_init(mma_done, 1);
    mbar_init(x_full, kEpiWarps / 2);
    mbar_init(x_empty, kEpiWarps / 2);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fence_proxy_async();
  }
  {
    // the small FP32 weights, once per CTA
    float4 *dst = reinterpret_cast<float4 *>(smem + kOffBias);
    const float4 *bsrc = reinterpret_cast<const float4 *>(prm.bias);
    const int nb = (L < kMaxHidden ? L : kMaxHidden) * kW / 4;
    for (int i = threadIdx.x; i < nb; i += kThreads) dst[i] = __ldg(bsrc + i);
    dst = reinterpret_cast<float4 *>(smem + kOffW0);
    const float4 *w0src = reinterpret_cast<const float4 *>(prm.w0);
    for (int i = threadIdx.x; i < kW * 3 / 4; i += kThreads) dst[i] = __ldg(w0src + i);
    // W_s[:, nshort + j] (j = 0..2): the skip layer's weights on p, from the
    // transposed copy (row k = nshort + j holds W_s[n][k] over n)
    dst = reinterpret_cast<float4 *>(smem + kOffWsk);
    const float4 *wssrc = reinterpret_cast<const float4 *>(
        prm.fwd_t + ((size_t)(prm.skip > 0 ? prm.skip - 1 : 0) * kW + (kW - 3)) * kW);
    for (int i = threadIdx.x; i < 3 * kW / 4; i += kThreads)
      dst[i] = prm.skip > 0 ? __ldg(wssrc + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    dst = reinterpret_cast<float4 *>(smem + kOffWout);
    const float4 *wosrc = reinterpret_cast<const float4 *>(prm.wout);
    for (int i = threadIdx.x; i < kW / 4; i += kThreads) dst[i] = __ldg(wosrc + i);
  }
  if (warp == 1) {
    if constexpr (kPair) {   // one warp of each CTA of the pair allocates collectively
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                       smem_u32(smem + kOffTmemSlot)),
                   "r"(kW));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;\n");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                       smem_u32(smem + kOffTmemSlot)),
                   "r"(kW));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();      // every CTA's barriers exist before any multicast targets them
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint16_t cmask = (uint16_t)((1u << kCluster) - 1u);
  // every CTA walks the same number of tiles (the cluster's CTAs consume the
  // same weight panels in lockstep); tiles past the end are all-masked
  const int64_t iters = (ntiles + gridDim.x - 1) / gridDim.x;

  auto fail = [&]() {
    atomicExch(prm.err, kDevTimeout);
    *abort_flag = 1;
  };

  // every warp ends here: all TMEM traffic is done before the owner frees it,
  // and no CTA leaves while a cluster peer may still multicast into it.  Each
  // role calls it from its own register region.
  auto finish = [&](bool tmem_owner) {
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    if (tmem_owner) {
      tc_fence_after();
      if constexpr (kPair)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kW));
      else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kW));
    }
  };

  if (warp < kEpiWarp0) {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(kCtlRegs));
  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, issued_parity = 0;   // per stage: a load in flight, its phase
      int64_t load_idx = 0;
      bool ok = true;
      for (int64_t it = 0; ok && it < iters; ++it) {
        for (int li = 0; ok && li < G; ++li) {
          const bool fwd = li < L - 1;
          const int l = fwd ? li + 1 : G - li;           // network layer of this product
          const CUtensorMap *map = fwd ? &tmap_fwd : &tmap_bwd;
          const int rowbase = (l - 1) * kW;
          for (int ld = 0; ld < kLoadsPerLayer; ++ld, ++load_idx) {
            if (!mbar_wait<true>(empty_bar(stage), phase ^ 1u, budget, abort_flag)) {
              fail();
              ok = false;
              break;
            }
            const int nh = ld / (kW / kKAtom), kb = k_atom(nh, ld % (kW / kKAtom));
            if (load_idx != prm.drop_load) {
              if constexpr (kPair) {
                // this CTA's 128 rows of the panel; both halves count on the
                // even CTA's barrier, which expects them both
                if (crank == 0) mbar_expect_tx(full_bar(stage), 2 * SB);
                tma_load_2d_pair(sB + stage * SB, map, kb * kKAtom,
                                 rowbase + nh * kN + (int)crank * kSliceRows,
                                 map_to_rank(full_bar(stage), 0));
              } else {
                mbar_expect_tx(full_bar(stage), kStageBytes);   // all slices land here
                tma_load_2d_mc(sB + stage * kStageBytes + crank * (kSliceRows * kKAtom * 2), map,
                               kb * kKAtom, rowbase + nh * kN + (int)crank * kSliceRows,
                               full_bar(stage), cmask);
              }
              issued_mask |= 1u << stage;
              issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
            }
            if (++stage == S) stage = 0, phase ^= 1u;
          }
        }
      }
      // drain: every issued load must land before the CTA may exit (pair: the
      // even CTA's barriers count both CTAs' halves)
      if (!kPair || crank == 0) {
        for (int s = 0; s < S; ++s) {
          if (issued_mask & (1u << s)) {
            volatile int no_abort = 0;
            if (!mbar_wait<true>(full_bar(s), (issued_parity >> s) & 1u, budget, &no_abort)) fail();
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && (!kPair || crank == 0)) {
      // ---------------- MMA issuer (pair form: the even CTA) ----------------
      // descriptors of A atom 0 and ring stage 0; atoms, stages and K steps
      // are constant offsets (addresses below 256 KB: no carry out of the
      // 14-bit address field)
      const uint64_t adesc0 = sw128_desc(sA), bdesc0 = sw128_desc(sB);
      constexpr uint32_t idesc = kPair ? idesc_f16(kF16, 2 * kM, kN) : Op<kF16>::idesc;
      auto commit_both = [&](uint32_t bar) {     // pair form: reaches both CTAs
        if constexpr (kPair) mma_commit_pair_mc(bar, cmask);
        else mma_commit(bar);
      };
      int stage = 0;
      uint32_t phase = 0, a_phase = 0;
      bool ok = true;
      for (int64_t it = 0; ok && it < iters; ++it) {
        for (int li = 0; ok && li < G; ++li) {
          for (int ld = 0; ld < kLoadsPerLayer; ++ld) {
            const int nh = ld / (kW / kKAtom), pos = ld % (kW / kKAtom), kb = k_atom(nh, pos);
            // half 0 needs A atoms 0..3 (and TMEM half 0 read) before it
            // starts, atoms 4, 6 and then 5, 7 (and TMEM half 1 read) later
            if (nh == 0 && (pos == 0 || pos == 4 || pos == 6)) {
              const uint32_t bar = pos == 0 ? a_lo : (pos == 4 ? a_hi_a : a_hi_b);
              const bool got = kPair ? mbar_wait_cluster(bar, a_phase, budget, abort_flag)
                                     : mbar_wait<true>(bar, a_phase, budget, abort_flag);
              if (!got) {
                fail();
                ok = false;
                break;
              }
              tc_fence_after();
            }
            if (!mbar_wait<true>(full_bar(stage), phase, budget, abort_flag)) {
              fail();
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(nh * kN);
            const uint64_t ad = adesc0 + (uint64_t)(kb * (kAtomBytes >> 4));
            const uint64_t bd = bdesc0 + (uint64_t)(stage * (SB >> 4));
#pragma unroll
            for (int ks = 0; ks < kKAtom / 16; ++ks) {
              const uint32_t acc = (pos | ks) != 0 ? 1u : 0u;
              if constexpr (kPair) mma_f16_pair(d, ad + 2 * ks, bd + 2 * ks, idesc, acc);
              else mma_f16(d, ad + 2 * ks, bd + 2 * ks, idesc, acc);
            }
            if constexpr (kPair) mma_commit_pair_mc(empty_bar(stage), cmask);
            else mma_commit_mc(empty_bar(stage), cmask);
            if (++stage == S) stage = 0, phase ^= 1u;
            if (nh == 0 && pos == 7) commit_both(d0_full);
            else if (nh == 1 && pos == 1) commit_both(lo_free_a);
            else if (nh == 1 && pos == 3) commit_both(lo_free_b);
          }
          if (!ok) break;
          a_phase ^= 1u;
          commit_both(d1_full);
        }
      }
      // drain: no product may still be writing TMEM when it is freed
      if constexpr (kPair) mma_commit_pair(mma_done);
      else mma_commit(mma_done);
      volatile int no_abort = 0;
      if (!mbar_wait<true>(mma_done, 0, budget, &no_abort)) fail();
    } else if (kPair && lane == 0) {
      // ---------------- relay (pair form: the odd CTA) ----------------
      // forwards each completed phase of this CTA's epilogue gates to the
      // even CTA's gates, in the order the products consume them
      const uint32_t remote[3] = {map_to_rank(a_lo, 0), map_to_rank(a_hi_a, 0),
                                  map_to_rank(a_hi_b, 0)};
      const uint32_t local[3] = {a_lo, a_hi_a, a_hi_b};
      uint32_t a_phase = 0;
      bool ok = true;
      for (int64_t it = 0; ok && it < iters; ++it) {
        for (int li = 0; ok && li < G; ++li) {
          for (int g = 0; g < 3; ++g) {
            if (!mbar_wait<true>(local[g], a_phase, budget, abort_flag)) {
              fail();
              ok = false;
              break;
            }
            mbar_arrive_remote(remote[g]);
          }
          a_phase ^= 1u;
        }
      }
    }
  }
  finish(warp == 1);
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(kEpiRegs));
    // ---------------- epilogue warps ----------------
    const int q = warp & 3;                  // TMEM lane quarter
    const int ch = (warp - kEpiWarp0) >> 2;  // first or last 128 columns of each half
    const int r = 32 * q + lane;             // row of the tile = TMEM lane
    const int skip = prm.skip;
    Epi e;
    e.A = A;
    e.slab = reinterpret_cast<uint8_t *>(prm.scratch) +
             (size_t)blockIdx.x * (size_t)(L - 1) * kW * kM * 2;
    e.t_row = tmem + ((uint32_t)(32 * q) << 16);
    e.r = r;
    e.ch = ch;
    e.neg_bl2e = -prm.beta * 1.4426950408889634f;
    e.inv_beta = 1.0f / prm.beta;
    e.gbias = prm.bias;
    e.save_h = prm.save_h;
    e.save_d = prm.save_d;
    e.n_pad = ntiles * kM;
    e.pol = l2_evict_first_policy();
    e.kh.neg_bl2e = __float2half2_rn(-prm.beta * 1.4426950408889634f);
    e.kh.inv_beta = __float2half2_rn(1.0f / prm.beta);
    e.kh.half_beta = __float2half2_rn(0.5f * prm.beta);
    e.kh.neg_bl2e_s2 = __float2half2_rn(-prm.beta * 1.4426950408889634f * kSqrt2);
    e.lane = lane;
    const bool prefetcher = (warp == kEpiWarp0 && lane == 0);
    uint32_t d_phase = 0, x_phase = 0;
    bool ok = true;
    auto arrive = [&](uint32_t bar) { epi_arrive(bar, lane); };
    // start of column half h of a product: its products are in TMEM; half 0
    // gets the gates it must pass before it overwrites A's columns 0..255
    auto begin_half = [&](int h, Gate &gate) -> bool {
      gate = Gate{lo_free_a, lo_free_b, d_phase, budget, abort_flag, h == 0, h == 0, true};
      if (!mbar_wait<true>(h == 0 ? d0_full : d1_full, d_phase, budget, abort_flag)) return false;
      tc_fence_after();
      return true;
    };
    for (int64_t it = 0; ok && it < iters; ++it) {
      // pair form: the cluster's two CTAs take consecutive tiles (rows 0..127
      // and 128..255 of each M=256 product)
      const int64_t tile = kPair ? ((int64_t)(blockIdx.x >> 1) + it * (gridDim.x >> 1)) * 2 + crank
                                 : blockIdx.x + it * gridDim.x;
      const int64_t idx = tile * kM + r;
      e.row = idx;
      float4 pw = make_float4(0.f, 0.f, 0.f, 0.f);
      if (idx < prm.n) pw = prm.pts[idx];
      e.px = pw.x; e.py = pw.y; e.pz = pw.z;
      if (prm.has_T) {
        const float *t = prm.Ti;
        e.px = t[0] * pw.x + t[1] * pw.y + t[2] * pw.z + t[3];
        e.py = t[4] * pw.x + t[5] * pw.y + t[6] * pw.z + t[7];
        e.pz = t[8] * pw.x + t[9] * pw.y + t[10] * pw.z + t[11];
      }
      Acc acc;

      // ---- L0 on CUDA cores ----
      if (skip == 1) layer0<kF16, true, kSave>(e);
      else layer0<kF16, false, kSave>(e);
      arrive(a_lo);
      arrive(a_hi_a);
      arrive(a_hi_b);

      // ---- hidden layers L1 .. L{L-1} (forward) ----
      for (int l = 1; ok && l < L; ++l) {
        const bool last = (l == L - 1), at = (l == skip), feeds = (l == skip - 1);
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          Gate gate;
          if (!begin_half(h, gate)) { fail(); ok = false; break; }
          const uint32_t mid = h == 1 ? a_hi_a : 0u;
          if (last) {
            if (at) fwd_half<kF16, true, true, false, kSave>(e, l, h, acc, gate, mid);
            else fwd_half<kF16, true, false, false, kSave>(e, l, h, acc, gate, mid);
          } else if (at) {
            fwd_half<kF16, false, true, false, kSave>(e, l, h, acc, gate, mid);
          } else if (feeds) {
            fwd_half<kF16, false, false, true, kSave>(e, l, h, acc, gate, mid);
          } else {
            fwd_half<kF16, false, false, false, kSave>(e, l, h, acc, gate, mid);
          }
          gate.pass_all();
          if (!gate.ok) { fail(); ok = false; break; }
          arrive(h == 0 ? a_lo : a_hi_b);
        }
        d_phase ^= 1u;
      }

      // ---- Jacobian-transpose chain: layers L-1 .. 1 ----
      for (int l = L - 1; ok && l >= 1; --l) {
        // bring this layer's slopes (128 KB of this CTA) into L2 while its products run
        if (prefetcher) l2_prefetch_bulk(e.slab + (size_t)(l - 1) * kW * kM * 2, kW * kM * 2);
        const bool at = (l == skip), makes = (l - 1 == skip), to_input = (l == 1);
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          Gate gate;
          if (!begin_half(h, gate)) { fail(); ok = false; break; }
          const uint32_t mid = h == 1 ? a_hi_a : 0u;
          if (to_input) {
            if (at) bwd_half<kF16, true, false, true, kSave>(e, l, h, acc, gate, 0u);
            else bwd_half<kF16, false, false, true, kSave>(e, l, h, acc, gate, 0u);
          } else if (at) {
            bwd_half<kF16, true, false, false, kSave>(e, l, h, acc, gate, mid);
          } else if (makes) {
            bwd_half<kF16, false, true, false, kSave>(e, l, h, acc, gate, mid);
          } else {
            bwd_half<kF16, false, false, false, kSave>(e, l, h, acc, gate, mid);
          }
          gate.pass_all();
          if (!gate.ok) { fail(); ok = false; break; }
          // the last product of the tile feeds no A: the next tile's L0 writes it
          if (!to_input) arrive(h == 0 ? a_lo : a_hi_b);
          else tc_fence_before();
        }
        d_phase ^= 1u;
      }
      if (!ok) break;
      float gx = acc.gx.x + acc.gx.y, gy = acc.gy.x + acc.gy.y, gz = acc.gz.x + acc.gz.y;
      float fpart = acc.f.x + acc.f.y;

      // ---- a7-a9: combine the two column halves, normalise, test, project ----
      if (ch == 1) {
        if (!mbar_wait<true>(x_empty, x_phase ^ 1u, budget, abort_flag)) { fail(); ok = false; break; }
        exch[r] = make_float4(gx, gy, gz, fpart);
        __syncwarp();
        if (lane == 0) mbar_arrive(x_full);
        x_phase ^= 1u;
        continue;
      }
      if (!mbar_wait<true>(x_full, x_phase, budget, abort_flag)) { fail(); ok = false; break; }
      x_phase ^= 1u;
      const float4 o = exch[r];
      __syncwarp();
      if (lane == 0) mbar_arrive(x_empty);
      if (idx < prm.n) {
        gx += o.x; gy += o.y; gz += o.z;
        const float f = fpart + o.w + __ldg(prm.bout);
        const float nrm = sqrtf(gx * gx + gy * gy + gz * gz);
        float nx = 0.f, ny = 0.f, nz = 0.f;
        if (nrm >= 1e-20f) { nx = gx / nrm; ny = gy / nrm; nz = gz / nrm; }
        if (!prm.collide) {
          if (prm.raw_gradient) { nx = gx; ny = gy; nz = gz; }
          prm.out_n_sdf[idx] = make_float4(nx, ny, nz, f);
        } else {
          if (prm.has_T) {
            const float *R = prm.R;
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
    finish(false);
  }
}

bool encode_panel_map(CUtensorMap *map, void *base, int rows, bool fp16) {
  auto fn = tensor_map_encoder();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kW, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kW * 2};
  cuuint32_t box[2] = {(cuuint32_t)kKAtom, (cuuint32_t)kSliceRows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool query_tc16_supported(int width, int n_hidden, int skip) {
  (void)skip;
  return width == kW && n_hidden >= 2;
}

bool make_tc16_tmaps(NetDevice &net, int width, int n_hidden, bool fp16) {
  if (!query_tc16_supported(width, n_hidden, 0)) return false;
  const int rows = (n_hidden - 1) * kW;
  return encode_panel_map(&net.tmap_fwd, net.fwd16, rows, fp16) &&
         encode_panel_map(&net.tmap_bwd, net.bwd16, rows, fp16);
}

// CTAs of this kernel that can be resident at once in whole clusters (a GPC
// with an odd number of free SMs cannot host a full cluster on all of them).
static int resident_cluster_ctas(int num_sms) {
  static int cached[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev] < num_sms ? cached[dev] : num_sms;
  cudaFuncSetAttribute(query_tc16_kernel<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
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
  if (cudaOccupancyMaxActiveClusters(&clusters, query_tc16_kernel<false, false, true>, &cfg) != cudaSuccess ||
      clusters < 1) {
    cudaGetLastError();
    clusters = num_sms / kCluster;
  }
  const int ctas = clusters * kCluster;
  if (dev >= 0 && dev < 64) cached[dev] = ctas;
  return ctas < num_sms ? ctas : num_sms;
}

int query_tc16_min_grid() { return kCluster; }

int query_tc16_grid(int width, int64_t n, int num_sms) {
  (void)width;
  const int64_t tiles = (n + kM - 1) / kM;
  const int cap = resident_cluster_ctas(num_sms);
  int64_t g = tiles < cap ? tiles : cap;
  g = (g / kCluster) * kCluster;                 // whole clusters
  return (int)(g < kCluster ? kCluster : g);
}



size_t query_tc16_scratch_bytes(int width, int n_hidden, int grid, bool fp16) {
  (void)width;
  (void)fp16;
  // one 16-bit word per element: the slope (FP16 form) or the activation (BF16 form)
  return (size_t)grid * (size_t)(n_hidden - 1) * kW * kM * 2;
}

template <bool kF16, bool kSave, bool kPair>
cudaError_t launch_t(const QueryParams &p, const NetDevice &net, int num_sms, cudaStream_t s) {
  auto kern = query_tc16_kernel<kF16, kSave, kPair>;
  // the register split inside the kernel is only valid for this count
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  if (fa.numRegs != kLaunchRegs) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  const int grid = query_tc16_grid(p.width, p.n, num_sms);
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
  e = cudaLaunchKernelEx(&cfg, kern, p, net.tmap_fwd, net.tmap_bwd);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Queries and the training form both run as CTA pairs unless the one-CTA
// form is selected (nsdf_debug_tc16_one_cta).
std::atomic<int> g_one_cta{0};

cudaError_t launch_query_tc16_net(const QueryParams &p, const NetDevice &net, bool fp16,
                                  int num_sms, cudaStream_t s) {
  if (g_one_cta.load(std::memory_order_relaxed)) {
    if (p.save_h)
      return fp16 ? launch_t<true, true, false>(p, net, num_sms, s)
                  : launch_t<false, true, false>(p, net, num_sms, s);
    return fp16 ? launch_t<true, false, false>(p, net, num_sms, s)
                : launch_t<false, false, false>(p, net, num_sms, s);
  }
  if (p.save_h)
    return fp16 ? launch_t<true, true, true>(p, net, num_sms, s)
                : launch_t<false, true, true>(p, net, num_sms, s);
  return fp16 ? launch_t<true, false, true>(p, net, num_sms, s)
              : launch_t<false, false, true>(p, net, num_sms, s);
}

}  // namespace nsdf

extern "C" nsdf_status nsdf_debug_tc16_one_cta(int enable) {
  nsdf::g_one_cta.store(enable ? 1 : 0, std::memory_order_relaxed);
  return NSDF_OK;
}
