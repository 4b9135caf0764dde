/*
 * nsdf.h - C ABI of the neural signed-distance collision library.
 *
 * The library answers collision queries against a body represented by a
 * signed-distance network f: R^3 -> R (Eq. 1 of Bertiche, Madadi & Escalera,
 * "Neural Implicit Surfaces for Efficient and Accurate Collisions in
 * Physically Based Simulations").  For every query point p it evaluates
 * f(p), the input gradient grad f(p) by back-propagation and the surface
 * normal N = grad f / ||grad f|| (Eq. 2); a point collides when f(p) < eps
 * (Sec. 3.2) and is then moved to its contact point p + (eps - f(p)) N
 * (Eq. 3 with the naive solve of Sec. 3.2).  A body placed by a rigid
 * transform T is queried at T^{-1} p and its normal rotated by T[:3,:3]
 * (Sec. 4.2).
 *
 * Conventions shared by every entry point:
 *  - Points are float4 records (x, y, z, w), 16-byte aligned, n of them
 *    contiguous; w is ignored on input and copied through to projected
 *    points.  Pointers that are not 16-byte aligned give NSDF_ERR_MISALIGNED.
 *  - Buffers are owned by the caller.  Unless an entry point says otherwise
 *    they are device pointers; the context owns only its weight copies,
 *    its scratch and its error word.
 *  - Calls are asynchronous on the given stream (NULL = legacy default
 *    stream).  n == 0 is a successful no-op.  Nothing is thrown across the
 *    ABI: every failure is a status code.
 *  - Errors raised inside a kernel (a bounded wait that ran out) are
 *    recorded in the context's error word and reported by
 *    nsdf_sync_status().
 *  - A context is used by one stream at a time; use one context per
 *    concurrent stream.
 */
#ifndef NSDF_H
#define NSDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nsdf_ctx nsdf_ctx;

/* Same object as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *nsdf_stream;

typedef enum {
  NSDF_OK = 0,
  NSDF_ERR_INVALID_ARG = 1,  /* bad pointer, size, shape or index            */
  NSDF_ERR_MISALIGNED = 2,   /* point / output pointer not 16-byte aligned   */
  NSDF_ERR_NOT_LOADED = 3,   /* query before nsdf_load_weights for that net  */
  NSDF_ERR_OOM = 4,          /* device allocation failed                     */
  NSDF_ERR_CUDA = 5,         /* a CUDA runtime call failed                   */
  NSDF_ERR_UNSUPPORTED = 6,  /* shape / precision this build has no kernel for */
  NSDF_ERR_TIMEOUT = 7,      /* a bounded wait inside a kernel ran out        */
  NSDF_ERR_TOO_LARGE = 8     /* exceeds the fixed scratch of nsdf_collide_noalloc */
} nsdf_status;

typedef enum {
  NSDF_FP32 = 0,  /* FP32 CUDA-core arithmetic throughout                      */
  NSDF_BF16 = 1,  /* hidden-layer products on BF16 tensor cores, FP32 accumulate */
  NSDF_FP16 = 2   /* hidden-layer products on FP16 tensor cores, FP32 accumulate:
                     same speed as BF16, 3 more significand bits; activations and
                     weights must stay within FP16 range (|x| < 65504)         */
} nsdf_precision;

/* Hidden-layer activation (nsdf_arch.activation). */
typedef enum {
  NSDF_ACT_SOFTPLUS = 0, /* softplus_beta(z) = log(1 + exp(beta z)) / beta */
  NSDF_ACT_RELU = 1      /* max(z, 0); its slope is taken as 0 at z = 0     */
} nsdf_activation;

/*
 * Network shape (Eq. 1): n_hidden layers L0..L{n_hidden-1} of `width` units
 * with the activation `activation`, then a linear output unit.  With
 * skip_layer = s > 0, layer L{s-1} has width - in_dim units and L{s} reads
 * [h_{s-1}, p] / sqrt(2).  in_dim must be 3; beta > 0 is the softplus
 * sharpness (ignored by ReLU).  ff_freqs = m > 0 puts the Fourier-feature
 * layer of the paper's networks (Sec. 4.3) in front: L0 reads
 * gamma(p) = [sin(2 pi B p), cos(2 pi B p)] (2m values, sines first), with
 * the frequency matrix B [m x 3] stored at the start of the weight blob;
 * this needs 2m == width and no skip layer.
 */
typedef struct {
  int in_dim;
  int width;
  int n_hidden;
  int skip_layer; /* -1: no skip */
  float beta;
  int activation; /* nsdf_activation */
  int ff_freqs;   /* 0: the network reads p itself */
} nsdf_arch;

/* nsdf_query flag: return grad f instead of the unit normal. */
#define NSDF_RAW_GRADIENT 1u

/*
 * Number of floats in a packed weight blob for `arch`: B [ff_freqs x 3]
 * (when ff_freqs > 0), then for each layer in order, W row-major [out x in]
 * then b[out].  Returns 0 for an invalid arch.
 */
size_t nsdf_num_params(const nsdf_arch *arch);

/*
 * Create a context for n_nets networks of the same shape on the current
 * device.  Synchronous.  Fails with NSDF_ERR_UNSUPPORTED when no kernel of
 * this build handles (arch, prec): FP32 takes widths 32, 64, 128, 256 and
 * 512 with either activation and Fourier features; BF16 and FP16 take
 * softplus networks of width 512 with at least two hidden layers and no
 * Fourier features, softplus networks of width 64 with 2 to 7 hidden layers
 * and no skip layer or Fourier features (their forward products take split
 * BF16 operands, hi + lo, in the BF16 form: one BF16 rounding of 64-wide
 * weights alone moves f by up to ~3e-3), and the Fourier-feature ReLU
 * networks of Sec. 4.3 of width 256 (ff_freqs = 128) with 1 to 8 layers and
 * no skip layer.  In the
 * 16-bit forms a ReLU slope is decided on the 16-bit network's own
 * pre-activations: near z = 0 it can differ from an FP32 or exact
 * evaluation, and with it the normal.
 */
nsdf_status nsdf_create(const nsdf_arch *arch, nsdf_precision prec, int n_nets,
                        nsdf_ctx **out);

/* Free the context and everything it owns.  Synchronises the device. */
nsdf_status nsdf_destroy(nsdf_ctx *ctx);

/*
 * Load the packed FP32 blob `w` (n_floats == nsdf_num_params) of network
 * `net`.  The library keeps its own converted copies (transposed, padded,
 * 16-bit where the precision asks); the caller keeps `w`.  w_is_device
 * selects whether `w` is a device or a host pointer; with a host pointer the
 * call returns after the copy has been taken.
 */
nsdf_status nsdf_load_weights(nsdf_ctx *ctx, int net, const float *w,
                              size_t n_floats, int w_is_device,
                              nsdf_stream stream);

/*
 * Eq. 1-2 for network 0: out_n_sdf[i] = (N_x, N_y, N_z, f(p_i)) with N the
 * unit normal (grad f if flags has NSDF_RAW_GRADIENT).  Where
 * ||grad f|| < 1e-20 the normal is the zero vector.
 */
nsdf_status nsdf_query(nsdf_ctx *ctx, const float *pts, int64_t n,
                       float *out_n_sdf, uint32_t flags, nsdf_stream stream);

/*
 * Collision test and naive solve (Sec. 3.2, Eq. 3, Sec. 4.2) for network 0.
 *   T: NULL, or a 4x4 row-major rigid transform placing the body (host
 *      memory, read during the call).
 *   out_pts[i]   = p_i + (eps - f) N_world if f < eps, else p_i (w copied)
 *   out_n_sdf[i] = (N_world, f)   (nullable)
 *   out_hit[i]   = f < eps        (nullable, one byte per point)
 * pts / out_pts / out_n_sdf / out_hit may all be device pointers, or all be
 * host pointers: with host pointers the library streams chunks through its
 * own device buffers (copies overlapped with compute) and returns once the
 * results are in host memory.  out_pts may alias pts.
 */
nsdf_status nsdf_collide(nsdf_ctx *ctx, const float *pts, int64_t n, float eps,
                         const float *T, float *out_pts, float *out_n_sdf,
                         uint8_t *out_hit, nsdf_stream stream);

/*
 * nsdf_collide without any allocation, for callers that cannot allocate
 * device memory when they query: a simulator running inside a fixed memory
 * budget, code that records its GPU work into a CUDA graph or calls from a
 * real-time callback (where cudaMalloc would synchronise or is forbidden),
 * or a host that forbids the library from growing after set-up.  The paper
 * has no counterpart; this is a property of the library, not of the method.
 *
 * Same arguments and results as nsdf_collide (device pointers only).  The
 * kernels' scratch comes from one fixed 32 MiB device array that every GPU
 * loading the library holds until exit; the launch uses as many CTAs as
 * whole per-CTA scratch slabs fit in it, so wide networks run on fewer SMs.
 * A network whose scratch for one CTA exceeds the array is rejected with
 * NSDF_ERR_TOO_LARGE.  pts, out_pts, out_n_sdf and out_hit must be device
 * (or managed) memory; a host array is rejected with NSDF_ERR_INVALID_ARG
 * before any launch, as is a non-finite eps.  No cudaMalloc, cudaFree or
 * allocating library call is made.  The first call on each device resolves
 * the array's device address (cudaGetSymbolAddress) and should come before
 * any stream capture; the address is kept for the life of the process, so,
 * like every context, it does not survive a device reset (cudaDeviceReset).
 * All calls share the array: calls that may overlap on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.
 */
nsdf_status nsdf_collide_noalloc(nsdf_ctx *ctx, const float *pts, int64_t n,
                                 float eps, const float *T, float *out_pts,
                                 float *out_n_sdf, uint8_t *out_hit,
                                 nsdf_stream stream);

/*
 * Gradients of L = sum_i g_sdf[i] f(p_i) + g_grad[i] . grad f(p_i) for
 * network 0 (training of Sec. 3.1; collision penalties).  g_grad is float4
 * per point (w ignored) and nullable (= 0).  g_weights (nullable) receives
 * dL/dtheta in blob layout (overwritten, FP32, nsdf_num_params floats);
 * g_pts (nullable) receives dL/dp_i as float4 (w = 0).  Layer activations
 * are recomputed, not stored.  FP32 arithmetic for either precision.  Every
 * array is DEVICE memory (host memory: NSDF_ERR_INVALID_ARG, nothing is
 * launched).
 */
nsdf_status nsdf_backward(nsdf_ctx *ctx, const float *pts, int64_t n,
                          const float *g_sdf, const float *g_grad,
                          float *g_weights, float *g_pts, nsdf_stream stream);

/*
 * Gradient of the L1 fitting loss of Sec. 3.1, L = (1/n) sum_i |f(p_i) - d_i|
 * (training points p_i, float4 [n], w ignored; exact signed distances d_i,
 * float [n]; both DEVICE), for network 0 of a 16-bit context (tensor cores).
 * g_weights (device, nsdf_num_params floats, blob layout) is overwritten with
 * dL/dtheta; loss (device float, nullable) receives L.  The derivative of
 * |f - d| is taken as sign(f - d), 0 at equality.  The hidden-layer weight
 * gradients are products over the points of the kernel's 16-bit deltas and
 * activations on the tensor cores with FP32 accumulation (the library's own
 * tcgen05 kernel, widths 256 and 512); the other sums are FP32 and
 * reduced in a fixed order, so repeated calls give identical results.  Uses
 * about 2 n_hidden x width x 2 bytes of device memory per point, allocated on
 * the first call and when n grows.  Fourier-feature ReLU contexts (Sec. 4.3)
 * take the same route through their own tensor-core kernel; their
 * frequencies B are not trained (random Fourier features) and receive 0.
 * FP32 contexts: NSDF_ERR_UNSUPPORTED (use nsdf_backward); n = 0 or a host
 * array: NSDF_ERR_INVALID_ARG.
 */
nsdf_status nsdf_l1_grad(nsdf_ctx *ctx, const float *pts, int64_t n,
                         const float *targets, float *g_weights, float *loss,
                         nsdf_stream stream);

/*
 * Many bodies in one launch: network k answers points
 * pts[offsets[k] .. offsets[k] + counts[k]) for k < n_nets of the context,
 * with the collision solve of nsdf_collide (no transform).  offsets and
 * counts are DEVICE int64 arrays: the work list is built on the device, so a
 * CUDA graph that captured this call replays correctly with new counts.
 * max_total (at most 2^34) bounds offsets[k] + counts[k] (a violating entry
 * is skipped and reported by nsdf_sync_status as NSDF_ERR_INVALID_ARG) and
 * sizes the launch.
 * out_n_sdf nullable; points outside every range are left untouched.  pts,
 * out_pts and out_n_sdf are DEVICE memory too (a host array, or host
 * offsets / counts: NSDF_ERR_INVALID_ARG, nothing is launched).
 * Arithmetic: FP32 contexts run the FP32 fused kernel; 16-bit width-64
 * softplus and Fourier-feature ReLU contexts run the tensor-core kernel of
 * their shape and precision with the same results per point as
 * nsdf_collide.  The
 * first call with a given max_total may allocate scratch: make it before
 * capturing the call into a graph.
 */
nsdf_status nsdf_query_grouped(nsdf_ctx *ctx, const float *pts,
                               const int64_t *offsets, const int64_t *counts,
                               int64_t max_total, float eps, float *out_pts,
                               float *out_n_sdf, nsdf_stream stream);

/*
 * nsdf_query_grouped for a scene of posed bodies (Sec. 4.2 per body): body k
 * is placed by the rigid transform T[16k .. 16k+15], a row-major 4x4 in
 * DEVICE memory (float, 4-byte aligned; the last row is not read).  Its
 * points are queried at T_k^{-1} p and its normals rotated by T_k[:3,:3], as
 * in nsdf_collide.  The poses are read (and inverted, in FP64, on the device)
 * by every call, so a captured CUDA graph replays with updated poses.  A
 * singular T_k is replaced by the identity and reported by nsdf_sync_status
 * as NSDF_ERR_INVALID_ARG.  Other arguments and errors as nsdf_query_grouped;
 * T == NULL is NSDF_ERR_INVALID_ARG.  This batching form has no counterpart
 * in the paper, which places one body.
 */
nsdf_status nsdf_query_grouped_T(nsdf_ctx *ctx, const float *pts,
                                 const int64_t *offsets, const int64_t *counts,
                                 int64_t max_total, float eps, const float *T,
                                 float *out_pts, float *out_n_sdf,
                                 nsdf_stream stream);

/*
 * Autotuner of the grouped launch: times every tile shape (4 or 8 points per
 * thread) and every CTAs-per-SM count that fits on this exact problem
 * (3 timed launches each, CUDA events), keeps the fastest in the context for
 * later nsdf_query_grouped calls and writes it to chosen[0] (points per
 * thread) and chosen[1] (CTAs per SM) when chosen is not NULL.  16-bit
 * Fourier-feature contexts have one grouped shape (a 128-point tile per
 * CTA, one CTA per SM, on tensor cores): the problem runs once and chosen
 * receives {0, 1}.  16-bit width-64 contexts (two 128-point tiles per CTA
 * on tensor cores) time every CTAs-per-SM count that fits and report
 * {0, CTAs per SM}.  Runs the
 * problem several times (outputs are overwritten with correct results) and
 * synchronises `stream`; do not call it during stream capture.
 */
nsdf_status nsdf_autotune_grouped(nsdf_ctx *ctx, const float *pts,
                                  const int64_t *offsets, const int64_t *counts,
                                  int64_t max_total, float eps, float *out_pts,
                                  float *out_n_sdf, nsdf_stream stream,
                                  int *chosen);

/* Set the grouped launch configuration directly (e.g. from a saved tuning):
 * points_per_thread 4 or 8 (FP32 contexts; 16-bit contexts, whose kernels
 * have one tile shape, also accept 0), ctas_per_sm >= 0 (0: as many as fit). */
nsdf_status nsdf_set_grouped_config(nsdf_ctx *ctx, int points_per_thread,
                                    int ctas_per_sm);

/*
 * Voxel SDF baseline, the comparison system of Sec. 4.3 (Table 1): the
 * signed distance sampled on a regular grid of n^3 nodes over the box
 * [lo, hi] (lo, hi: 3 floats each, HOST memory), node (i, j, k) at
 * lo + (i, j, k) (hi - lo) / (n - 1) stored at grid[i + n (j + n k)]
 * (float, DEVICE, n^3 values; n = 256 is 64 MB).
 *
 * nsdf_voxel_build fills the grid with the exact signed distance of every
 * node to a watertight mesh (the brute force of nsdf_mesh_sdf; same mesh
 * arguments, DEVICE pointers).  n in [2, 2048].
 *
 * nsdf_voxel_collide answers the collision query of nsdf_collide from the
 * grid: sdf by trilinear interpolation of the node values, normal = the
 * normalised gradient of that interpolant (Eq. 2 applied to it), hit =
 * sdf < eps and the contact point of Eq. 3.  A point outside the box takes
 * the value at its nearest point of the box plus its distance to the box,
 * and that distance's gradient is added to the normal's.  pts, out_pts,
 * out_n_sdf (float4, 16-byte aligned) and out_hit are DEVICE memory (host
 * memory: NSDF_ERR_INVALID_ARG); out_n_sdf and out_hit nullable; out_pts
 * may alias pts.  Asynchronous on `stream`.
 */
nsdf_status nsdf_voxel_build(const float *verts, int64_t n_verts,
                             const int32_t *faces, int64_t n_faces, int n,
                             const float *lo, const float *hi, float *grid,
                             nsdf_stream stream);
nsdf_status nsdf_voxel_collide(const float *grid, int n, const float *lo,
                               const float *hi, const float *pts, int64_t n_pts,
                               float eps, float *out_pts, float *out_n_sdf,
                               uint8_t *out_hit, nsdf_stream stream);

/*
 * Ground-truth signed distance to a watertight triangle mesh by brute force
 * (the targets of Sec. 3.1): out_sdf[i] = +-min_t dist(p_i, triangle t),
 * negative where the generalized winding number exceeds 1/2 (interior
 * negative, Sec. 3.2).  verts: float [n_verts*3]; faces: int32 [n_faces*3],
 * counter-clockwise seen from outside; pts float4; all device pointers (a
 * host array: NSDF_ERR_INVALID_ARG, nothing is launched).
 * The winding number is accumulated in FP32 and recomputed in FP64 for
 * points with |w - 1/2| < 0.25 or distance < 1e-3.
 */
nsdf_status nsdf_mesh_sdf(const float *verts, int64_t n_verts,
                          const int32_t *faces, int64_t n_faces,
                          const float *pts, int64_t n, float *out_sdf,
                          nsdf_stream stream);

/*
 * One explicit Verlet step of a rectangular quad cloth (Sec. 4.1) on an
 * nx-by-ny grid (float4 positions, row-major, row = z index): structural and
 * shear springs with rest lengths from the grid spacings hx (along rows) and
 * hz (between rows), unit mass, Hooke constant k_over_m, gravity (0, -g, 0):
 *   x_new = 2 x - x_prev + dt^2 a(x).
 * nx <= 2^30, ny <= 65535.
 * Writes x_new into x_prev's buffer (the caller swaps the two).  x and
 * x_prev_inout are DEVICE memory (host memory: NSDF_ERR_INVALID_ARG).  The
 * collision solve is a separate nsdf_collide call on the result.
 */
nsdf_status nsdf_cloth_step(const float *x, float *x_prev_inout, int nx,
                            int ny, float hx, float hz, float k_over_m,
                            float g, float dt, nsdf_stream stream);

/*
 * Synchronise `stream`, then report (and clear) an error recorded by a
 * kernel of this context: NSDF_ERR_TIMEOUT when a bounded wait ran out.
 */
nsdf_status nsdf_sync_status(nsdf_ctx *ctx, nsdf_stream stream);

/* Static, human-readable name of a status code. */
const char *nsdf_status_string(nsdf_status s);

#ifdef __cplusplus
}
#endif

#endif /* NSDF_H */
