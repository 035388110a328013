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
 * the number of elements.  candidate = -1 checks the schedule the batched
 * body (ttc_batch_*, ttc_server_*) runs for the plan instead.  Returns TTC_OK
 * or TTC_ERR_INVALID_ARG with a description of the first violation in msg
 * (NUL-terminated, msglen bytes).
 */
ttc_status ttc_debug_verify_schedule(ttc_plan_t plan, int candidate, char* msg, int msglen);

/*
 * Text description of candidate `candidate` of `plan`: its kernel, tile
 * groups and extents, lane layout, grid order (fastest first) and the cost
 * model's estimate, written NUL-terminated into buf (buflen bytes).
 * TTC_ERR_INVALID_ARG for a bad plan, candidate or buffer.
 */
ttc_status ttc_debug_describe_candidate(ttc_plan_t plan, int candidate, char* buf, int buflen);

#ifdef __cplusplus
}
#endif
#endif /* TTC_DEBUG_H_ */
