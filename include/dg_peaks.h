/*
 * dg_peaks.h -- ALU throughput microbenchmarks (libdgpeaks.so) that give the roofline denominators of the RHS
 * kernels. The flux-differencing volume term (Sec. 2.1-2.3, Eq. fluxdiff-SBP-opDsplit) is bound by floating-
 * point arithmetic, and the two-point flux needs divisions and logarithms (Sec. 3.1, Algorithms 2-3), so the
 * device's rates for these operations bound the kernel.
 *
 * Kinds: 0 fp64 FMA, 1 fp32 FMA, 2 fp64 division, 3 fp64 log, 4 fp32 logf, 5 fp32 lg2.approx (special-function
 * unit), 6 fp32 rcp.approx, 7 fp32 division, 8 fp64 reciprocal (round to nearest).
 * Runs on the current device; allocates and frees a small device buffer; synchronizes the device.
 */
#ifndef DG_PEAKS_H
#define DG_PEAKS_H
#ifdef __cplusplus
extern "C" {
#endif

/* number of benchmark kinds */
int dgpk_num_kinds(void);

/* Measures kind `kind`: *ops_per_s receives operations per second (an FMA counts as one operation), *seconds
   (may be NULL) the duration of the timed launch, which is grown to at least min_seconds. Returns 0 or a
   cudaError_t value. */
int dgpk_measure(int kind, double min_seconds, double* ops_per_s, double* seconds);

#ifdef __cplusplus
}
#endif
#endif
