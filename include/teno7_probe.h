/*
 * teno7_probe.h -- measured arithmetic peaks of the current CUDA device, the
 * denominators of the ALU roofline that the TENO7-ext stage kernels are
 * reported against.  The paper has no counterpart: it reports no
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

/* FMA throughput of the device in TFLOP/s (2 flop per fused multiply-add):
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

#ifdef __cplusplus
}
#endif
#endif /* TENO7_PROBE_H */
