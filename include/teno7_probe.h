/*
 * teno7_probe.h -- measured arithmetic peaks of the current CUDA device, the
 * denominators of the ALU roofline that the TENO7-ext stage kernels are
 * reported against; and a self-test of the checked build's index check.  The paper has no counterpart: it reports no
 * performance figures.  Part of libteno7 (links against teno7.h's status
 * codes).
 */
#ifndef TENO7_PROBE_H
#define TENO7_PROBE_H

#include "teno7.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { T7_PROBE_F32 = 0, T7_PROBE_F32X2 = 1, T7_PROBE_F64 = 2 };

/* FMA throughput of the device in TFLOP/s (2 flop per fused multiply-add; no
 * counterpart in the paper, which reports no performance figures):
 * every SM filled with CTAs of 256 threads, each running 8 independent
 * chains of 16 x iters FMAs (kind T7_PROBE_F32: scalar FP32; T7_PROBE_F32X2:
 * packed f32x2 FMAs, two per instruction; T7_PROBE_F64: FP64), one warm-up
 * launch, then the fastest of `repeats` launches timed with CUDA events on
 * `stream` (a cudaStream_t; NULL = legacy default stream).
 *   tflops  host, receives the rate; ms (host, nullable) the launch time.
 * Allocates and frees a small device buffer (the results' sink).
 * Synchronises.  T7_EINVAL for a bad kind or count, T7_ECUDA / T7_ENOMEM if a
 * CUDA call fails. */
t7_status t7_probe_fma(int kind, int iters, int repeats, void *stream, double *tflops, float *ms);

/* Self-test of the index check of the checked build (see teno7.h; no
 * counterpart in the paper): one
 * device thread passes index i through the check against [lo, hi) on a
 * private control block, as every kernel does for the indices it forms.
 *   index_out          host, receives the index an access would use: i, or,
 *                      in the checked build with i outside [lo, hi), lo
 *   flagged_out        host, receives 1 if the check latched the failure
 *                      with index i (checked build, i outside), else 0
 *   checked_build_out  host, receives 1 for the checked build, 0 otherwise
 * No memory is addressed by i.  Synchronises (legacy default stream).
 * T7_EINVAL for a null pointer or lo >= hi, T7_ENOMEM / T7_ECUDA if a CUDA
 * call fails. */
t7_status t7_probe_index_check(int i, int lo, int hi, int *index_out, int *flagged_out, int *checked_build_out);

#ifdef __cplusplus
}
#endif
#endif /* TENO7_PROBE_H */
