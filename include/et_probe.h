/*
 * et_probe.h -- measurement aid of libet, not part of the paper's method:
 * the 32-bit integer issue throughput of the device.  The tube-count kernel
 * (tube tests of Section 2, Fig. 4b) is bound by integer arithmetic, so this
 * measured rate is the denominator its roofline is compared with beside the
 * nominal one (SMs x 128 lanes x clock).
 *
 * et_probe_int_throughput runs three kernels over the whole device (8 blocks
 * of 256 threads per SM, 8 independent dependency chains per thread):
 *   out[0] "alu": per step a 32-bit xor and an add (the integer ALU pipe),
 *   out[1] "mad": per step a 32-bit multiply-add whose factors are both the
 *          chain value (IMAD),
 *   out[2] "mix": per step a xor, an add and a multiply-add, the ALU : IMAD
 *          ratio of the exact tube test,
 * and stores the operations per second of each, from the CUDA-event time of
 * one launch after a warm-up launch, on the context's stream.  The call is
 * synchronous and takes about 0.1 s.
 *
 * Arguments: ctx from et_ctx_create; out points to 3 doubles (caller-owned).
 * Errors: ET_ERR_INVALID_ARG for a NULL ctx or out, ET_ERR_CUDA when a launch
 * or an event fails (out is then left unchanged).
 */
#ifndef ET_PROBE_H
#define ET_PROBE_H

#include "et.h"

#ifdef __cplusplus
extern "C" {
#endif

et_status et_probe_int_throughput(et_ctx *ctx, double out[3]);

#ifdef __cplusplus
}
#endif

#endif /* ET_PROBE_H */
