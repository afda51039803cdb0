/*
 * rtlbfs_measure.h -- measurement support: the arithmetic rates that the
 * rooflines of the step kernels are stated against.  Not a step of the
 * paper's method; the paper reports no GPU figures (arXiv 2202.13449 times
 * serial CPU programs only, Section 4.4, Table 6).
 *
 * The step kernels are bound by plain FP32 (or FP64) arithmetic, not by
 * tensor cores, so their roofline denominator is the rate at which the SMs
 * retire fused multiply-adds.  This call measures that rate on the current
 * device instead of deriving it from unit counts and a nominal clock.
 */
#ifndef RTLBFS_MEASURE_H
#define RTLBFS_MEASURE_H

#ifdef __cplusplus
extern "C" {
#endif

#define RTLBFS_RATE_FP32 0  /* scalar FP32 FMA (FFMA) */
#define RTLBFS_RATE_FP32X2 1 /* packed FP32x2 FMA (two FMAs per instruction) */
#define RTLBFS_RATE_FP64 2  /* FP64 FMA */

/*
 * FMA rate of the current device for the given kind: a kernel of
 * independent FMA chains (8 per thread, no memory traffic in the loop)
 * over every SM at full occupancy, `reps` inner iterations per chain,
 * timed with CUDA events on the legacy default stream after one untimed
 * launch.  Writes FMAs per second (each FFMA2 counts as 2) to *fma_per_s
 * and the timed launch's duration in milliseconds to *ms.  Host pointers,
 * caller-owned.  Allocates 4 bytes of device memory for the kernel's sink
 * and frees it.  RTLBFS_ERR_ARG for an unknown kind, reps < 1 or null
 * pointers; RTLBFS_ERR_CUDA if a CUDA call fails.
 */
int rtlbfs_fma_rate(int kind, int reps, double* fma_per_s, double* ms);

#ifdef __cplusplus
}
#endif

#endif
