/*
 * nsdf_debug.h - test-only controls of the nsdf library's failure path.
 *
 * The tensor-core query kernel hands work between its producer, MMA and
 * epilogue warps through mbarriers.  Every wait is bounded: after
 * `wait_budget_cycles` SM clock cycles without progress the kernel records a
 * timeout in the context's error word, lets the copies and products it has
 * in flight finish, frees its tensor memory and returns;
 * nsdf_sync_status() then reports NSDF_ERR_TIMEOUT and the context stays
 * usable.  Nothing in the paper corresponds to this; it exists so that a
 * test can exercise the timeout path without faulting or hanging a GPU.
 */
#ifndef NSDF_DEBUG_H
#define NSDF_DEBUG_H

#include "nsdf.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * drop_load >= 0: the producer skips that weight-panel load (counted from 0
 * within one launch), so the consumer's wait for it runs out.  -1 restores
 * normal operation.  wait_budget_cycles > 0 bounds every mbarrier wait
 * (default 4e9 cycles, about two seconds).  Applies to later launches of
 * this context's BF16 query; host-side only, no device work.
 */
nsdf_status nsdf_debug_inject(nsdf_ctx *ctx, int drop_load, long long wait_budget_cycles);

/*
 * Caps the bytes of nsdf_collide_noalloc's fixed device array that later
 * calls may use (process-wide; 0 restores the whole array).  With the whole
 * array no network the library accepts is rejected, so this lets a test
 * reach the NSDF_ERR_TOO_LARGE reject, which returns before any launch.
 * Host-side only.
 */
nsdf_status nsdf_debug_noalloc_limit(size_t bytes);

/*
 * Measures the FP32 FMA throughput of the current GPU (the peak against
 * which the FP32 form's arithmetic is reported): independent FMA chains on
 * every SM, timed with CUDA events on `stream`, best of three launches;
 * writes TFLOP/s (2 FLOP per FMA) to *tflops.  Synchronises `stream`.
 */
nsdf_status nsdf_debug_fp32_fma_peak(double *tflops, nsdf_stream stream);

/*
 * Selects how later launches of the width-512 tensor-core kernel issue their
 * products (process-wide): 1 = one CTA per 128-point tile (M=128 products, a
 * 2-stage ring of 32 KB weight panels), 0 = the default CTA pairs (M=256
 * products over a 2-CTA cluster's two tiles).  Both compute the same values;
 * this lets a test and a timing compare them.  Host-side only.
 */
nsdf_status nsdf_debug_tc16_one_cta(int enable);

#ifdef __cplusplus
}
#endif

#endif /* NSDF_DEBUG_H */
