/*
 * ptn_peaks.h -- measured arithmetic peaks of the current GPU, the denominators of the
 * benchmark's roofline fractions.  The paper has no counterpart: this is measurement
 * infrastructure, built as its own library (libptn_peaks.so), not part of the solver.
 */
#ifndef PTN_PEAKS_H
#define PTN_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* Throughput of fused multiply-adds on the current device, in TFLOP/s (2 flops per FMA):
 * fp64 = 0 measures the FP32 pipe, 1 the FP64 pipe.  A grid of blocks_per_sm x SM-count
 * blocks of 256 threads runs `iters` rounds of 8 independent FMA chains per thread; the
 * second of two launches is timed with CUDA events on the legacy default stream, which
 * the call synchronises.  Writes *tflops and *ms (either may be NULL) and returns 0, or
 * returns the negative cudaError_t of the first failing call (-1 for invalid arguments:
 * fp64 outside {0, 1}, blocks_per_sm < 1 or iters < 1). */
int ptn_peak_fma(int fp64, int blocks_per_sm, int iters, double* tflops, double* ms);

#ifdef __cplusplus
}
#endif
#endif /* PTN_PEAKS_H */
