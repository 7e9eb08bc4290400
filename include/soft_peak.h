/* soft_peak.h -- issue-rate peaks of the arithmetic pipes, measured on the
 * current device, used as the roofline denominators of the shot kernels.
 *
 * The paper has no counterpart (it reports no roofline). The FP64 path's
 * binding pipe is the FP64 one, whose rate on this part has no measured
 * figure elsewhere; the FP32 and integer rates put the lane-op roof (SMs x
 * 128 lanes x clock) next to a measurement.
 */
#ifndef SOFT_PEAK_H
#define SOFT_PEAK_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Instruction kinds: FP64 fused multiply-add (2 flops each), FP32 fused
 * multiply-add (2 flops each), 32-bit three-input logic op (1 op each). */
enum { SOFT_PEAK_FP64_FMA = 0, SOFT_PEAK_FP32_FMA = 1, SOFT_PEAK_INT32_LOGIC = 2 };

/* Run a kernel of independent chains of one instruction kind on every SM of
 * the current device (4 blocks of 256 threads per SM), asynchronously on
 * `stream` (NULL = the legacy default stream), and wait for it. Two warm-up
 * launches, then the fastest of five timed by CUDA events on that stream.
 *   ops_per_s: receives flops/s (FMA kinds) or ops/s (logic) of that launch.
 *   ms_per_launch (may be NULL): its duration in milliseconds.
 * The rate follows the SM clock, which this call does not set: sample the
 * clock while it runs to know what it was measured at. Errors: SOFT_E_ARG
 * (unknown kind, NULL ops_per_s), SOFT_E_CUDA. */
int soft_peak_pipe_rate(int32_t kind, void *stream, double *ops_per_s, double *ms_per_launch);

#ifdef __cplusplus
}
#endif
#endif
