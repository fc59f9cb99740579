/*
 * fpparse_test.h -- test hooks of libfpparse (not part of the parsing API).
 *
 * They let a test drive the library's device-side error paths without a GPU
 * fault: every wait in the kernels is bounded, and a hook can make one wait
 * run out on purpose, so that the error path, and the recovery of the next
 * call, can be checked.
 */
#ifndef FPPARSE_TEST_H
#define FPPARSE_TEST_H

#include "fpparse.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * fp_test_arm_stalled_lookback -- arm the next fp_parse_f64, fp_parse_f32 or
 * fp_parse_ex call on `stream` (one call only).  That call hands out its
 * chunk tickets from 1 instead of 0, so chunk 0 is never parsed and never
 * publishes its field count; the decoupled look-back of the chunks after it
 * (Section 4's field index, here a cross-chunk scan) waits for that word,
 * which nothing ever writes.  Each device wait of that call gives up after
 * wait_limit_ns nanoseconds (1 .. 2e9; the default limit of every other call
 * is 2 s), records FP_ERR_TIMEOUT in the stream's error word (read with
 * fp_get_error) and lets the kernel finish; that call's results and count
 * are void.  Later calls on the stream are unaffected.
 *   stream          the stream whose next call is armed (its per-stream
 *                   scratch is created if needed: cudaMalloc)
 *   wait_limit_ns   the armed call's wait limit
 * Returns FP_ERR_ARG for a limit outside 1 .. 2e9, FP_ERR_CUDA if the
 * scratch cannot be allocated, else FP_OK.
 */
FP_API fp_err_t fp_test_arm_stalled_lookback(struct CUstream_st *stream, uint64_t wait_limit_ns);

#ifdef __cplusplus
}
#endif
#endif /* FPPARSE_TEST_H */
