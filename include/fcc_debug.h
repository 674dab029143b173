/*
 * fcc_debug.h -- test hooks for the failure paths of the library.  The paper
 * has no counterpart; these exist so that tests can drive the error exits of
 * the kernels and of plan creation without faulting a GPU: every device-side
 * wait in the FP32 kernels (the folded-form kernel, its batched form, the
 * split-form kernel, and the per-pair kernel of the smoothed path) is a bounded loop
 * that, when it runs out, latches FCC_ERR_TIMEOUT in the plan's error word and
 * lets the kernel finish once its own copies have landed.
 *
 * The hooks are process-wide and not thread-safe; they are meant for tests.
 */
#ifndef FCC_DEBUG_GB300_H
#define FCC_DEBUG_GB300_H

#include "fcc.h"

#ifdef __cplusplus
extern "C" {
#endif

enum {
    /* Bound of every device-side wait of the FP32 kernels launched from now on,
     * in SM clock cycles (value >= 1000); 0 restores the default (2e9, about 1 s). */
    FCC_DEBUG_WAIT_CYCLES = 0,
    /* The next `value` FP32 launches withhold the first bulk copy of one warp
     * group (block 0, group 0; in the per-pair kernel block 0's first frame), so
     * that group's first wait runs out: the launch finishes and fcc_plan_sync
     * reports FCC_ERR_TIMEOUT.  Only launches that stage with bulk copies (an
     * even number of microphones) are affected. */
    FCC_DEBUG_WITHHOLD_COPY = 1,
    /* The next `value` device allocations made while creating a plan, or the
     * staging of fcc_tdoa_host / fcc_tdoa_pcm_host on their first call, fail as
     * if the device were out of memory (the call returns FCC_ERR_OOM and keeps
     * nothing of what it had allocated). */
    FCC_DEBUG_FAIL_ALLOC = 2
};

/* Set one hook.  Errors: INVALID_ARG (unknown hook, value out of range). */
fcc_status_t fcc_debug_set(int hook, long long value);

#ifdef __cplusplus
}
#endif
#endif /* FCC_DEBUG_GB300_H */
