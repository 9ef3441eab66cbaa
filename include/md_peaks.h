/*
 * md_peaks.h -- pipe-throughput microbenchmarks used as roofline denominators
 * of the pair kernels.  The paper has no counterpart: its kernels ran on a
 * Kepler GPU whose peaks it does not state; these measure the sm_103a pipes
 * that the FP32 pair path (Sec. 3.2) and the FP64 state updates depend on.
 */
#ifndef MD_PEAKS_H
#define MD_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* Measure, on the current CUDA device, per-SM per-clock throughputs.
 * out[0] = SM count; then for k = 0..8, out[1+2k] = operations per SM per clock
 * and out[2+2k] = the SM clock (MHz) seen during that test, for
 *   k=0 FP32 FMA (scalar fmaf), k=1 FP32 FMA issued as packed f32x2 (2 per
 *   instruction), k=2 rsqrt.approx, k=3 rcp.approx, k=4 sin.approx,
 *   k=5 lg2.approx + ex2.approx (2 per iteration), k=6 FP64 FMA,
 *   k=7 FP32->FP64->FP32 conversions (2 per iteration), k=8 FP32 FMA with half
 *   the chains packed f32x2 and half scalar (1.5 per iteration on average).
 * nout must be >= 19.  Returns 0 on success, nonzero on a CUDA failure.
 * Takes about a second; allocates and frees its own small device buffers. */
int mdp_pipe_rates(double *out, int nout);

#ifdef __cplusplus
}
#endif
#endif
