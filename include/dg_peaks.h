/*
 * dg_peaks.h -- ALU throughput microbenchmarks (libdgpeaks.so) that give the roofline denominators of the RHS
 * kernels. The flux-differencing volume term (Sec. 2.1-2.3, Eq. fluxdiff-SBP-opDsplit) is bound by floating-
 * point arithmetic, and the two-point flux needs divisions and logarithms (Sec. 3.1, Algorithms 2-3), so the
 * device's rates for these operations bound the kernel.
 *
 * Kinds: 0 fp64 FMA, 1 fp32 FMA, 2 fp64 division, 3 fp64 log, 4 fp32 logf, 5 fp32 lg2.approx (special-function
 * unit), 6 fp32 rcp.approx, 7 fp32 division, 8 fp64 reciprocal (round to nearest), 9 the RHS kernels' fp64
 * logarithm (log_f64), 10 fp64 exp, 11 fp64 sqrt, 12 the RHS kernels' fp64 square root (sqrt_f64).
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

/* Arithmetic self-test of the RHS kernels' device code (the same source as libdg): for i < n, on device arrays,
   L[i] = {{a1[i], b1[i]}}_log by Algorithm 2 and Li[i] = 1/{{a2[i], b2[i]}}_log by Algorithm 3 (Sec. 3.1), from the
   single reciprocal the flux kernels share, and r[i] = the kernels' reciprocal of a1[i]. precision 0: FP64;
   1: FP32 (inputs rounded to float). Inputs must be positive. Synchronizes the device; returns 0 or a
   cudaError_t value. */
int dgpk_eval_logmeans(long long n, int precision, const double* a1, const double* b1, const double* a2,
                       const double* b2, double* L, double* Li, double* r);

/* Self-test of the integer-pipe IEEE conversions the FP32 flux mode uses (binary64 -> binary32 round to nearest
   even with flush to zero below the normal range; binary32 -> binary64 exact) against the hardware conversions:
   f_int/f_hw receive the float bit patterns of d2f_int(x) and __double2float_rn(x), d_int/d_hw the widenings of that
   float. Device arrays of n elements; synchronizes; returns 0 or a cudaError_t value. */
int dgpk_eval_convert(long long n, const double* x, unsigned* f_int, unsigned* f_hw, double* d_int, double* d_hw);

/* Self-test of the two-float split that the FP32 flux mode's reference pressure uses (integer pipe): hi = the
   round-to-nearest float of x[i], lo = the float of x[i] - hi (to within 2^-22 of itself), and rel = x[i] - ref[i]
   in FP32 from the two splits (energy_rel). Device arrays of n elements; synchronizes; returns 0 or a cudaError_t
   value. */
int dgpk_eval_split(long long n, const double* x, const double* ref, float* hi, float* lo, float* rel);

/* Self-test of the RHS kernels' FP64 natural logarithm (Cody and Waite's argument reduction with an atanh series;
   used by the logarithmic means and the entropy projection) against CUDA's log: log_own/log_ref receive
   log_f64(x[i]) / log(x[i]). Device arrays of n elements; synchronizes; returns 0 or a cudaError_t value. */
int dgpk_eval_log(long long n, const double* x, double* log_own, double* log_ref);

/* Self-test of the RHS kernels' FP64 square root (Goldschmidt's iteration from rsqrt.approx; the LLF wave speeds)
   against CUDA's sqrt: own/ref receive sqrt_f64(x[i]) / sqrt(x[i]). Device arrays; synchronizes; returns 0 or a
   cudaError_t value. */
int dgpk_eval_sqrt(long long n, const double* x, double* own, double* ref);

/* Self-test of the LLF wave speed's square root (an FP32 root refined by one FP64 Newton step, about 46 bits;
   sqrt_f64 outside [2^-100, 2^100]): out receives sqrt_wave_f64(x[i]). Device arrays; synchronizes; returns 0 or a
   cudaError_t value. */
int dgpk_eval_sqrt_wave(long long n, const double* x, double* out);

#ifdef __cplusplus
}
#endif
#endif
