/*
 * ttc_debug.h -- testing hooks of libttc (not needed by applications).
 */
#ifndef TTC_DEBUG_H_
#define TTC_DEBUG_H_

#include "ttc.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Host-side check of a schedule, without a GPU: runs the exact index
 * arithmetic of the kernels for candidate `candidate` of `plan` (every tile or
 * row chunk, every thread) and verifies that (1) every A and B access lies
 * inside the (sub-)tensors' byte ranges, (2) every element of B's sub-tensor
 * is written exactly once, (3) the element written at each B position is the
 * A element that Eq. 1 (section 1) maps there under the permutation and the
 * outer sizes as given to ttc_plan, (4) shared-memory positions stay inside
 * the tile buffer, each written once and read once, and (5) the FP8 amax
 * pre-pass visits every element of A's sub-tensor once.  Cost is linear in
 * the number of elements.  candidate = -1 - j checks instead the batched
 * body's schedule j (ttc_batch_*, ttc_server_*): j = 0 is the one it runs by
 * default, j = 1, 2, ... the further candidates ttc_batch_autotune may
 * choose; a j beyond the plan's batch candidates returns TTC_ERR_INVALID_ARG
 * with "no such batch candidate".  Returns TTC_OK or TTC_ERR_INVALID_ARG
 * with a description of the first violation in msg (NUL-terminated, msglen
 * bytes).
 */
ttc_status ttc_debug_verify_schedule(ttc_plan_t plan, int candidate, char* msg, int msglen);

/*
 * Text description of candidate `candidate` of `plan`: its kernel, tile
 * groups and extents, lane layout, grid order (fastest first) and the cost
 * model's estimate, written NUL-terminated into buf (buflen bytes).
 * TTC_ERR_INVALID_ARG for a bad plan, candidate or buffer.
 */
ttc_status ttc_debug_describe_candidate(ttc_plan_t plan, int candidate, char* buf, int buflen);

/*
 * The slot tables tile_slots_kernel reads for candidate `candidate` of
 * `plan` (layout: TileParams::slots in csrc/ttc_internal.h), copied into
 * out[0..count) as int32 values; *needed receives the table's length.
 * TTC_ERR_INVALID_ARG if the candidate does not use slot tables or count is
 * too small.
 */
ttc_status ttc_debug_slot_tables(ttc_plan_t plan, int candidate, int32_t* out, int64_t count, int64_t* needed);

/*
 * Server failure detection without a GPU fault: set the watchdog (seconds;
 * default 30) after which a server gives up an epoch whose completion it has
 * not seen, and submit a request that is a single-thread kernel staying busy
 * for `microseconds` (0..10 s, bounded by the device timer) on a stream of
 * the large class.  A delay longer than the watchdog makes the request
 * complete with TTC_ERR_TIMEOUT and retires its stream; the kernel itself
 * still ends on its own.
 */
ttc_status ttc_debug_server_set_watchdog(ttc_server_t server, double seconds);
ttc_status ttc_debug_server_submit_delay(ttc_server_t server, int64_t microseconds, int64_t* ticket);

/*
 * Failure detection of the packed GEMM's bounded waits without a GPU fault:
 * with skip != 0 the plan's next executions issue no tensor-core MMA and
 * commit nothing, so every mbarrier wait runs out (after 2^12 polls under
 * this hook); the kernel records the error word, frees its tensor memory and
 * returns without writing C, and ttc_packed_gemm_check reports
 * TTC_ERR_TIMEOUT (once).  skip = 0 restores normal executions.
 */
ttc_status ttc_debug_packed_gemm_skip_mma(ttc_packed_gemm_t g, int skip);

/*
 * The packed GEMM runs its warp-specialised kernel (Bm copied by TMA, the
 * pack by warps of its own, a ring of stages) when the pack reads A 16 bytes
 * at a time (k dense in A, A 16-byte aligned); with classic != 0 it runs the
 * kernel whose threads stage both operands through registers instead (what
 * it runs otherwise), so that tests can compare the two on the same
 * operands.  classic = 0 restores the choice.
 */
ttc_status ttc_debug_packed_gemm_classic(ttc_packed_gemm_t g, int classic);

/*
 * A timed comparison for the BF16 contraction: with use != 0 the
 * contraction's GEMM on the same K-major BF16 operands runs on cuBLAS
 * instead of this library's tensor-core kernel (use = 0 restores it).  No
 * effect on the FP32 and FP64 modes.
 */
ttc_status ttc_debug_contraction_use_cublas(ttc_contraction_t c, int use);

/*
 * The tile shape of the BF16 contraction's tensor-core GEMM: variant 0 lets
 * the library pick (the default); 1, 4 and 5 force one CTA per 128 x 256,
 * 128 x 192 or 128 x 128 output tile; 2, 6 and 3 a pair of CTAs on
 * neighbouring SMs per 256 x 256, 256 x 192 or 256 x 128 tile; -1 leaves the
 * setting as it is.  Other values return TTC_ERR_INVALID_ARG.
 * *last_used (if not NULL) receives the shape the last execution ran (1..6;
 * 0 before the first).  A pair shape falls back to 1 when K = 0 or the
 * device runs no CTA pairs.
 */
ttc_status ttc_debug_contraction_gemm_variant(ttc_contraction_t c, int variant, int* last_used);

#ifdef __cplusplus
}
#endif
#endif /* TTC_DEBUG_H_ */
