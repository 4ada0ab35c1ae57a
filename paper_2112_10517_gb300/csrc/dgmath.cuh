// Device arithmetic of the two-point flux: reciprocals, the logarithmic mean and its inverse (Sec. 3.1,
// Algorithms 2 and 3), per-node quantities and Ranocha's flux (Sec. 3.2, Eq. flux_ranocha).
// Shared by the RHS kernels (libdg) and by the arithmetic self-test entry of libdgpeaks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_internal.h"

namespace dgk {

// ---------------------------------------------------------------------------------------------------
// Precision traits. On GB300 an FP64 FMA issues at 2 per clock per SM; a correctly rounded FP64 reciprocal
// costs about 7 FMA slots, a division 10 and a logarithm 37 (measured with libdgpeaks), so the FP64 kernels
// avoid them where the mathematics allows.
// ---------------------------------------------------------------------------------------------------
// ---------------------------------------------------------------------------------------------------
// FP64 natural logarithm for the flux and entropy arithmetic (Cody and Waite's argument reduction with a short
// series): within 2 ulp of the C library's and CUDA's log, at 1.2x the throughput of CUDA's log on GB300.
//
// log_f64(x), x positive: x = 2^k m with m in [sqrt(1/2), sqrt(2)); log m = 2 atanh(t), t = (m - 1)/(m + 1),
// |t| <= 0.1716, summed as 2 sum_{j=0..9} t^(2j+1)/(2j+1) (truncation below 2.4e-17 relative); k ln 2 with ln 2
// split into a head with the low 21 mantissa bits cleared (k head is exact for |k| < 2^21) and the tail.
// Subnormal x are scaled by 2^54 first; x <= 0 or NaN gives NaN, +inf gives +inf.
// ---------------------------------------------------------------------------------------------------
__device__ __forceinline__ double rcp_newton_f64(double s) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(s));
  double e = fma(-s, r, 1.0);
  r = fma(r, e, r);
  e = fma(-s, r, 1.0);
  return fma(r, e, r);
}

__device__ __forceinline__ double log_f64(double x) {
  constexpr double kLn2Head = 0.6931471803691238;      // 0x3FE62E42FEE00000
  constexpr double kLn2Tail = 1.9082149292705877e-10;  // ln 2 - head
  constexpr double kTwo52p31 = 4503601774854144.0;     // 2^52 + 2^31: int -> double through the low word
  if (!(x >= 2.2250738585072014e-308) || x == __longlong_as_double(0x7FF0000000000000LL)) {
    if (x == __longlong_as_double(0x7FF0000000000000LL)) return x;
    if (!(x > 0.0)) return __longlong_as_double(0x7FF8000000000000LL);
  }
  int adj = 0;
  if (x < 2.2250738585072014e-308) {  // subnormal
    x *= 18014398509481984.0;         // 2^54
    adj = -54;
  }
  const int hi = __double2hiint(x), lo = __double2loint(x);
  // m in [sqrt(1/2), sqrt(2)): mantissas above that of sqrt(2) (high word 0x3FF6A09E) take exponent -1
  const int mh = hi & 0x000FFFFF;
  const int big = mh > 0x6A09E ? 1 : 0;
  const int k = ((hi >> 20) & 0x7FF) - 1023 + big + adj;
  const double m = __hiloint2double((mh | 0x3FF00000) - (big << 20), lo);
  const double t = (m - 1.0) * rcp_newton_f64(m + 1.0);
  const double z = t * t;
  double P = 2.0 / 19.0;
  P = fma(P, z, 2.0 / 17.0);
  P = fma(P, z, 2.0 / 15.0);
  P = fma(P, z, 2.0 / 13.0);
  P = fma(P, z, 2.0 / 11.0);
  P = fma(P, z, 2.0 / 9.0);
  P = fma(P, z, 2.0 / 7.0);
  P = fma(P, z, 2.0 / 5.0);
  P = fma(P, z, 2.0 / 3.0);
  const double logm = fma(t * z, P, t + t);  // 2t + t z P(z)
  const double kd = __hiloint2double(0x43300000, k ^ (int)0x80000000) - kTwo52p31;  // (double)k, exact
  return fma(kd, kLn2Head, fma(kd, kLn2Tail, logm));
}

// Sign and order tests of doubles on the integer pipe (on GB300 FP64 compares, absolute values and minima/maxima
// issue on the FP64 pipe, which the kernels saturate): a double's bit pattern read as a signed 64-bit integer
// orders like the value for non-negative values, and +inf is 0x7FF0000000000000 with the NaNs above it.
//   pos_f64(x):   0 < x <= +inf (false for NaN and zero), as x > 0
//   posfin_f64(x): 0 < x < +inf
//   abs_f64(x):   |x| by clearing the sign bit of the high word
//   maxnn_f64(a, b): max(a, b) for non-negative a, b (b when equal)
__device__ __forceinline__ bool pos_f64(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7FF0000000000000LL;
}
__device__ __forceinline__ bool posfin_f64(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7FF0000000000000LL;
}
__device__ __forceinline__ double abs_f64(double x) {
  return __hiloint2double(__double2hiint(x) & 0x7FFFFFFF, __double2loint(x));
}
__device__ __forceinline__ double maxnn_f64(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b) ? a : b;
}

// sqrt x for positive normal x by Goldschmidt's iteration for the square root: from r ~ 1/sqrt(x)
// (rsqrt.approx.ftz.f64), g = x r ~ sqrt(x) and h = r/2 are refined together by e = 1/2 - g h,
// g <- g + g e, h <- h + h e, which doubles the number of correct bits per step; two steps reach the rounding
// limit (about 1 ulp). x = 0 gives 0; other non-positive or non-finite x give NaN or inf.
__device__ __forceinline__ double sqrt_f64(double x) {
  if (!posfin_f64(x)) return x == 0.0 ? x : (x > 0.0 ? x : __longlong_as_double(0x7FF8000000000000LL));
  double r;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double g = x * r, h = 0.5 * r;
  double e = fma(-g, h, 0.5);
  g = fma(g, e, g);
  h = fma(h, e, h);
  e = fma(-g, h, 0.5);
  return fma(g, e, g);
}

template <typename T>
struct Num;

template <>
struct Num<double> {
  // 1/s by one third-order step of the reciprocal iteration, r <- r (1 + e + e^2) with e = 1 - s r, started
  // from the hardware approximation rcp.approx.ftz.f64 (which reads the top 32 bits of s: relative error
  // delta about 2^-20). With r = (1 + delta)/s, e = -delta and the step gives (1 + delta^3)/s, so one step
  // (3 FMA) reaches the rounding limit where two Newton-Raphson steps (which square delta: 4 FMA) did: within
  // 0.5 ulp + |delta|^3 of 1/s. Valid for normal positive and negative s; s = 0 gives a non-finite result.
  __device__ static __forceinline__ double rcp(double s) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(s));
    const double e = fma(-s, r, 1.0);
    return fma(r, fma(e, e, e), r);
  }
  __device__ static __forceinline__ double log(double x) { return log_f64(x); }
  __device__ static __forceinline__ double log1p(double x) { return ::log1p(x); }
  __device__ static __forceinline__ double sqrt(double x) { return sqrt_f64(x); }
  __device__ static __forceinline__ double abs(double x) { return abs_f64(x); }
  __device__ static __forceinline__ bool pos(double x) { return pos_f64(x); }
  __device__ static __forceinline__ double maxnn(double a, double b) { return maxnn_f64(a, b); }
  // u < 1e-4, the threshold of the series branch of Algorithms 2 and 3 for 64-bit floats (Sec. 3.1), tested on
  // the high 32 bits of u >= 0 (an integer comparison): the effective threshold is the largest double whose
  // high word is below that of 1e-4, 1e-4 to within a relative 1e-6; both branches are accurate there.
  // values within this ratio give u = ((r - 1)/(r + 1))^2 <= 8.9e-5: the series branch with margin
  __device__ static __forceinline__ double series_range() { return 1.019; }
  __device__ static __forceinline__ bool series(double u) {
    return __double2hiint(u) < 0x3F1A36E2;  // high word of 1e-4 = 0x3F1A36E2EB1C432D
  }
};

template <>
struct Num<float> {
  // rcp.approx.ftz.f32 and one Newton-Raphson step (FP32 flux mode)
  __device__ static __forceinline__ float rcp(float s) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(s));
    return fmaf(r, fmaf(-s, r, 1.0f), r);
  }
  __device__ static __forceinline__ float log(float x) { return ::logf(x); }
  __device__ static __forceinline__ float log1p(float x) { return ::log1pf(x); }
  __device__ static __forceinline__ float sqrt(float x) { return ::sqrtf(x); }
  __device__ static __forceinline__ float abs(float x) { return ::fabsf(x); }
  __device__ static __forceinline__ bool pos(float x) { return x > 0.0f; }
  __device__ static __forceinline__ float maxnn(float a, float b) { return a > b ? a : b; }
  // The paper states the threshold for 64-bit floats only. In FP32 the truncated series is accurate to about
  // 0.03 u^4 relative and the log branch loses about eps32/(2 sqrt(u)); 1e-2 keeps both near 1 ulp.
  // values within this ratio give u <= 7.6e-3: the series branch with margin
  __device__ static __forceinline__ float series_range() { return 1.19f; }
  __device__ static __forceinline__ bool series(float u) { return u < 1e-2f; }
};

// ---------------------------------------------------------------------------------------------------
// IEEE format conversions on the integer pipe. On GB300 a hardware FP64<->FP32 conversion issues on the FP64
// pipe (2 per clock per SM), which the FP32 flux mode would otherwise saturate converting every state value.
//   d2f_int: binary64 -> binary32, round to nearest even; results below the smallest normal float flush to
//            signed zero (the FP32 mode's flush-to-zero); infinities and NaN are not preserved.
//   f2d_int: binary32 -> binary64, exact for normal floats and zero (subnormals flush to zero).
// ---------------------------------------------------------------------------------------------------
__device__ __forceinline__ float d2f_int(double x) {
  // on the two 32-bit halves: a 64-bit mask of the sign bit may be turned into an FP64 absolute value
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const unsigned mhi = hi & 0x7FFFFFFFu;
  // keep 23 of the 52 mantissa bits: adding 2^28 - 1 plus the lowest kept bit (bit 29 of the low word) rounds to
  // nearest, ties to even; the carry into the high word, and out of the mantissa into the exponent, is exact
  const unsigned add = 0x0FFFFFFFu + ((lo >> 29) & 1u);
  const unsigned rlo = lo + add;
  const unsigned rhi = mhi + (rlo < add ? 1u : 0u);
  const int e = (int)(rhi >> 20) - 1023 + 127;
  const unsigned m = ((rhi & 0xFFFFFu) << 3) | (rlo >> 29);
  return __uint_as_float(e <= 0 ? sign : (sign | ((unsigned)e << 23) | m));
}

__device__ __forceinline__ double f2d_int(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned em = b & 0x7FFFFFFFu;
  const unsigned hi = em < 0x00800000u ? sign : (sign | ((em >> 3) + ((1023u - 127u) << 20)));
  const unsigned lo = em < 0x00800000u ? 0u : (em << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// The rounding remainder of d2f_int, on the integer pipe: for x in the normal FP32 range and hi = d2f_int(x),
// lo = x - hi to within 2^-22 of itself, so that hi + lo equals x to about 2^-46 relative. The 29 mantissa bits that
// d2f_int drops, less 2^29 where it rounded up, give x - hi in units of 2^(e-52) (e the exponent of x); their top 23
// bits convert exactly to a float (the 1.5 * 2^23 bias trick) and a power of two scales them. lo is 0 where that
// scale leaves the float range (|x| below about 2^-80 or above 2^170) and where hi flushed to zero.
__device__ __forceinline__ float split_lo_f64(double x, float hi) {
  const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
  const int L = (int)(l & 0x1FFFFFFFu);
  const bool up = L > 0x10000000 || (L == 0x10000000 && ((l >> 29) & 1u));  // d2f_int's round-to-nearest-even
  int r = up ? L - 0x20000000 : L;                                          // in [-2^28, 2^28]
  if (h & 0x80000000u) r = -r;
  const float fr = __int_as_float(0x4B400000 + (r >> 6)) - 12582912.0f;  // r / 64, exact
  const int se = (int)((h >> 20) & 0x7FFu) - 1023 + 81;                 // FP32 biased exponent of 2^(e-46)
  return (se >= 1 && se <= 254 && hi != 0.0f) ? fr * __int_as_float(se << 23) : 0.0f;
}

// The energy of a state in the flux precision, relative to a reference (FP32 mode with a reference pressure):
// E - E_ref with E_ref = eh + el, from the FP64 state value E without FP64 instructions. With E and E_ref within a
// factor 2 the difference of the leading floats is exact (Sterbenz), so the result carries the rounding of the small
// difference, not that of E (|E| 2^-24). eh = el = 0 gives d2f_int(E) itself (no reference).
template <typename T>
__device__ __forceinline__ T energy_rel(double E, float eh, float el) {
  if constexpr (sizeof(T) == 8) {
    return E;
  } else {
    const float hi = d2f_int(E);
    if (eh == 0.0f && el == 0.0f) return hi;
    return (hi - eh) + (split_lo_f64(E, hi) - el);
  }
}

// sqrt x to about 46 bits, for the local Lax-Friedrichs wave speed: the correctly rounded FP32 root g of x and
// h ~ 1/(2g) in FP32 (integer-pipe conversions), then one Newton (Heron) step in FP64, g + h (x - g^2), which
// squares the relative error of g (2^-24 -> 2^-48; h's own error adds about 2^-47). Two FP64 operations instead
// of the seven of sqrt_f64; x outside [2^-100, 2^100] (beyond the FP32 seed's range) takes sqrt_f64.
__device__ __forceinline__ double sqrt_wave_f64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  if (hi - 0x39B00000u >= 0x0C800000u) return sqrt_f64(x);  // not in [2^-100, 2^100): sign, 0, NaN, inf, range
  const float xf = d2f_int(x);
  const float gf = sqrtf(xf);
  const double g = f2d_int(gf);
  const double h = f2d_int(__fdividef(0.5f, gf));
  return fma(fma(-g, g, x), h, g);
}

// FP32 value of a double x in [0, 1) from its high word alone: the exponent and 20 of the 52 mantissa bits
// (truncated, relative error below 2^-20); x below 2^-100 gives 0. Four integer operations.
__device__ __forceinline__ float d2f_hi(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  return hi < 0x39B00000u ? 0.0f : __uint_as_float((hi - 0x38000000u) << 3);
}

// The innermost coefficient c2 + c3 u of the log means' series (u < 1e-4 on the FP64 series branch). It
// multiplies u^2 <= 1e-8 and its u-term is at most 5e-5 of c2, so FP32 arithmetic on a truncated u changes the
// mean by well under 1 ulp, and the FP64 pipe (1/64 of the FP32 rate on GB300) is spared one FMA per mean.
template <typename T>
__device__ __forceinline__ T series_inner(T u, float c2, float c3) {
  if constexpr (sizeof(T) == 8)
    return f2d_int(fmaf(d2f_hi(u), c3, c2));
  else
    return c2 + u * c3;
}

// state value (FP64 in memory) in the flux precision T; a float is already in the FP32 flux precision
template <typename T>
__device__ __forceinline__ T to_flux(double x);
template <typename T>
__device__ __forceinline__ T to_flux(float x) { return (T)x; }
template <>
__device__ __forceinline__ double to_flux<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_flux<float>(double x) { return d2f_int(x); }

// FP64 means of values within a ratio of about 1.22 (1e-4 <= u < 1e-2, u tested on its high word, the threshold
// the double 0x3F847AE100000000 just below 1e-2): the two series of log_means continued to u^7, whose truncation
// is then below 6e-18 relative, in 7 FMA and one product each instead of a logarithm (about 37 FMA slots) and a
// division. f/atanh(f) = 1/sum_k u^k/(2k+1) = 1 - u/3 - 4u^2/45 - 44u^3/945 - 428u^4/14175 - 10196u^5/467775
// - 10719068u^6/638512875 - 25865068u^7/1915538625 - ... (half of it for L), and 2 atanh(f)/f = sum_k 2u^k/(2k+1).
__device__ __forceinline__ bool wide_series_f64(double u) { return __double2hiint(u) < 0x3F847AE1; }
__device__ __forceinline__ double wide_L_f64(double s, double u) {
  double P = -12932534.0 / 1915538625.0 / 2.0;
  P = fma(P, u, -5359534.0 / 638512875.0);
  P = fma(P, u, -5098.0 / 467775.0);
  P = fma(P, u, -214.0 / 14175.0);
  P = fma(P, u, -22.0 / 945.0);
  P = fma(P, u, -2.0 / 45.0);
  P = fma(P, u, -1.0 / 6.0);
  return s * fma(P, u, 0.5);
}
template <typename T>
__device__ __forceinline__ bool wide_series(T u) {
  if constexpr (sizeof(T) == 8) return wide_series_f64(u);
  else return false;
}
template <typename T>
__device__ __forceinline__ T wide_L(T s, T u) {
  if constexpr (sizeof(T) == 8) return wide_L_f64(s, u);
  else return s;  // not reached (wide_series is false in FP32)
}
__device__ __forceinline__ double wide_Li_f64(double r, double u);
template <typename T>
__device__ __forceinline__ T wide_Li(T r, T u) {
  if constexpr (sizeof(T) == 8) return wide_Li_f64(r, u);
  else return r;  // not reached
}
__device__ __forceinline__ double wide_Li_f64(double r, double u) {
  double P = 2.0 / 15.0;
  P = fma(P, u, 2.0 / 13.0);
  P = fma(P, u, 2.0 / 11.0);
  P = fma(P, u, 2.0 / 9.0);
  P = fma(P, u, 2.0 / 7.0);
  P = fma(P, u, 2.0 / 5.0);
  P = fma(P, u, 2.0 / 3.0);
  return r * fma(P, u, 2.0);
}

// ---------------------------------------------------------------------------------------------------
// The two logarithmic means of Ranocha's flux from ONE reciprocal (Sec. 3.1 and 3.2):
//   L  = {{a}}_log                for (a1, b1)                (Algorithm 2)
//   Li = 1/{{c}}_log              for (a2, b2)                (Algorithm 3)
// With s = a + b and f = (b - a)/s, u = f^2 equals the u of Algorithms 2 and 3 (their numerator and
// denominator are (b - a)^2 and (b + a)^2). R = 1/(s1 s2) gives 1/s1 = s2 R and 1/s2 = s1 R.
// Series branches: L = s1 (1/2 - u/6 - 2u^2/45 - 22u^3/945), the polynomial form of 1/log of Sec. 3.1
// (a multiplication instead of a division), and Li = (2 + 2u/3 + 2u^2/5 + 2u^3/7)/s2 (Algorithm 3); the innermost
// coefficients (of u^2) in FP32 for FP64 means (series_inner).
// WIDE (FP64): between u = 1e-4 and 1e-2 the same series to u^7 (wide_L_f64, wide_Li_f64). The volume terms' beta
// form takes it; the product form (the interface kernel, which it measured 2 % slower on the Taylor-Green vortex,
// whose pairs never need it) keeps the paper's two branches.
// Log branches: L = (b - a)/log(b/a), Li = log(b/a)/(b - a), as in Algorithms 2 and 3.
// ---------------------------------------------------------------------------------------------------
template <typename T, bool WIDE = true>
__device__ __forceinline__ void log_means(T a1, T b1, T a2, T b2, T& L, T& Li) {
  const T s1 = a1 + b1, d1 = b1 - a1;
  const T s2 = a2 + b2, d2 = b2 - a2;
  const T R = Num<T>::rcp(s1 * s2);
  const T r1 = s2 * R, r2 = s1 * R;
  const T f1 = d1 * r1, f2 = d2 * r2;
  const T u1 = f1 * f1, u2 = f2 * f2;
  if (Num<T>::series(u1))
    L = s1 * (T(0.5) + u1 * (T(-1.0 / 6.0) + u1 * series_inner<T>(u1, float(-2.0 / 45.0), float(-22.0 / 945.0))));
  else if (WIDE && wide_series<T>(u1))
    L = wide_L<T>(s1, u1);
  else
    L = d1 / Num<T>::log(b1 / a1);
  if (Num<T>::series(u2))
    Li = r2 * (T(2.0) + u2 * (T(2.0 / 3.0) + u2 * series_inner<T>(u2, float(2.0 / 5.0), float(2.0 / 7.0))));
  else if (WIDE && wide_series<T>(u2))
    Li = wide_Li<T>(r2, u2);
  else
    Li = Num<T>::log(b2 / a2) / d2;
}

// ---------------------------------------------------------------------------------------------------
// Per-node quantities for the pair flux (Sec. 7.1: computed once per node, not once per pair):
//   q = (rho, v_1..v_d, pp = 2p, pg = 2p/(gamma - 1))                            NQ = d + 3 values
// from conserved u; returns false for rho <= 0, p <= 0 or NaN.
// FP32 mode with a reference pressure (shift pp0 = 2 p_ref != 0): the state's energy arrives as E - p_ref/(gamma-1)
// (energy_rel), and q[PP] holds pp - pp0 = 2 (p - p_ref), the form the momentum equations' pressure terms take
// (a constant pressure contributes nothing to them: its volume and surface terms cancel by the discrete metric
// identities). The flux recovers pp = q[PP] + pp0 where it needs the pressure itself; q[PG] is unshifted.
// ---------------------------------------------------------------------------------------------------
template <int ND>
struct NodeQ {
  static constexpr int NQ = ND + 3;
  static constexpr int RHO = 0, V = 1, PP = ND + 1, PG = ND + 2;
};

// The same with 1/rho given (ir), for callers that share one reciprocal between two states; uc is the state in
// FP64 (U = double) or already in the flux precision (U = T, with the energy relative to the reference, if any).
template <int ND, typename T, typename U>
__device__ __forceinline__ bool node_quantities_ir(const U* uc, T ir, T gm1, T two_over_gm1, T* q, T pp0 = T(0)) {
  const T rho = to_flux<T>(uc[0]);
  T ke = T(0);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const T m = to_flux<T>(uc[1 + j]);
    const T v = m * ir;
    q[1 + j] = v;
    ke += m * v;
  }
  const T p = gm1 * (to_flux<T>(uc[ND + 1]) - T(0.5) * ke);
  const T pt = sizeof(T) == 8 ? p : p + T(0.5) * pp0;  // the pressure itself (pp0 = 0: p)
  q[0] = rho;
  q[NodeQ<ND>::PP] = p + p;
  q[NodeQ<ND>::PG] = pt * two_over_gm1;
  return Num<T>::pos(rho) && Num<T>::pos(pt);
}

// From the FP64 state; sh (FP32 mode) the reference pressure's split energy and pp0 (all zero: none).
// beta: q[PG] holds beta = rho/p instead of pg (the volume terms of Ranocha's flux, ranocha_flux8 with BETA).
template <int ND, typename T>
__device__ __forceinline__ bool node_quantities(const double* uc, T gm1, T two_over_gm1, T* q, T* ir_out = nullptr,
                                                float sh_eh = 0.0f, float sh_el = 0.0f, float sh_pp = 0.0f,
                                                bool beta = false) {
  const T rho = to_flux<T>(uc[0]);
  const T ir = Num<T>::rcp(rho);
  if (ir_out) *ir_out = ir;  // 1/rho, for callers that need it again (the LLF wave speed)
  T ke = T(0);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const T m = to_flux<T>(uc[1 + j]);
    const T v = m * ir;
    q[1 + j] = v;
    ke += m * v;
  }
  const T p = gm1 * (energy_rel<T>(uc[ND + 1], sh_eh, sh_el) - T(0.5) * ke);
  const T pt = sizeof(T) == 8 ? p : p + T(0.5) * T(sh_pp);  // the pressure itself (no shift: p)
  q[0] = rho;
  q[NodeQ<ND>::PP] = p + p;
  q[NodeQ<ND>::PG] = beta ? rho * Num<T>::rcp(pt) : pt * two_over_gm1;
  return Num<T>::pos(rho) && Num<T>::pos(pt);
}

// ---------------------------------------------------------------------------------------------------
// Variants of the two means for the ablation of Sec. 3.1 and Sec. 7.2 (volume terms only):
//   LM_SHARED_RCP  log_means above: no division; one reciprocal shared by u1, u2 and the inverse mean's series,
//                  the mean's series in the polynomial 1/log form (a product);
//   LM_ALG         Algorithm 2 (mean) and Algorithm 3 (inverse mean) as stated: u by a division, the series
//                  branches by a division, the log branches as log(b/a) with two divisions;
//   LM_ALG_POLY    the same with the polynomial 1/log form of the mean's series branch (Sec. 3.1), i.e. one
//                  division fewer there;
//   LM_PRELOG      LM_SHARED_RCP with logarithms computed once per node instead of once per pair (Sec. 7.2): the
//                  log branches take log(b/a) as a difference of the per-node values.
// ---------------------------------------------------------------------------------------------------
// (the LM_* codes are defined in dg_internal.h)

template <typename T, int LM>
__device__ __forceinline__ void log_means_alg(T a1, T b1, T a2, T b2, T& L, T& Li) {
  const T u1 = (a1 * (a1 - T(2) * b1) + b1 * b1) / (a1 * (a1 + T(2) * b1) + b1 * b1);
  const T u2 = (a2 * (a2 - T(2) * b2) + b2 * b2) / (a2 * (a2 + T(2) * b2) + b2 * b2);
  if (Num<T>::series(u1)) {
    if (LM == LM_ALG_POLY)
      L = (a1 + b1) * (T(0.5) + u1 * (T(-1.0 / 6.0) + u1 * (T(-2.0 / 45.0) + u1 * T(-22.0 / 945.0))));
    else
      L = (a1 + b1) / (T(2.0) + u1 * (T(2.0 / 3.0) + u1 * (T(2.0 / 5.0) + u1 * T(2.0 / 7.0))));
  } else {
    L = (b1 - a1) / Num<T>::log(b1 / a1);
  }
  if (Num<T>::series(u2))
    Li = (T(2.0) + u2 * (T(2.0 / 3.0) + u2 * (T(2.0 / 5.0) + u2 * T(2.0 / 7.0)))) / (a2 + b2);
  else
    Li = Num<T>::log(b2 / a2) / (b2 - a2);
}

// LM_PRELOG: as log_means, with l1 = log(b1 / a1) and l2 = log(b2 / a2) taken from per-node logarithms (la, lb:
// the two nodes' [LR, LB] values, ls apart in shared memory, read only in the log branches); the log branches
// become L = d1 / l1 and Li = l2 / d2, each by the shared reciprocal routine (Num::rcp).
template <typename T>
__device__ __forceinline__ void log_means_prelog(T a1, T b1, T a2, T b2, const T* la, const T* lb, int ls, T& L,
                                                 T& Li) {
  const T s1 = a1 + b1, d1 = b1 - a1;
  const T s2 = a2 + b2, d2 = b2 - a2;
  const T R = Num<T>::rcp(s1 * s2);
  const T r1 = s2 * R, r2 = s1 * R;
  const T f1 = d1 * r1, f2 = d2 * r2;
  const T u1 = f1 * f1, u2 = f2 * f2;
  if (Num<T>::series(u1))
    L = s1 * (T(0.5) + u1 * (T(-1.0 / 6.0) + u1 * series_inner<T>(u1, float(-2.0 / 45.0), float(-22.0 / 945.0))));
  else
    L = d1 * Num<T>::rcp(lb[0] - la[0]);
  if (Num<T>::series(u2))
    Li = r2 * (T(2.0) + u2 * (T(2.0 / 3.0) + u2 * series_inner<T>(u2, float(2.0 / 5.0), float(2.0 / 7.0))));
  else
    Li = (lb[ls] - la[ls]) * Num<T>::rcp(d2);
}

// Per-node logarithms for LM_PRELOG, relative to the element's first node (rho0, pp0): LR = log(rho/rho0),
// LB = log(rho/pp) - log(rho0/pp0). Differences of these are the logarithms of ratios the paper's per-node
// log(rho), log(p) give (the reference cancels), without the cancellation of two large logarithms: each value is
// log1p of a small relative change, so a difference carries the rounding of the change, not of log(rho).
template <int ND, typename T>
__device__ __forceinline__ void node_logs(const T* q, T rho0, T pp0, T& lr, T& lb) {
  using Q = NodeQ<ND>;
  lr = Num<T>::log1p((q[Q::RHO] - rho0) * Num<T>::rcp(rho0));
  const T lp = Num<T>::log1p((q[Q::PP] - pp0) * Num<T>::rcp(pp0));
  lb = lr - lp;
}

// The per-node logarithms of LM_PRELOG, passed to the flux: node a's and node b's LR values, LB ls further on.
template <typename T>
struct LogRef {
  const T* la;
  const T* lb;
  int ls;
};

// ppa, ppb: the two nodes' 2p (unshifted)
template <int ND, typename T, int LM>
__device__ __forceinline__ void ranocha_means(const T* a, const T* b, T ppa, T ppb, T& L, T& Li,
                                              const LogRef<T>& lg) {
  using Q = NodeQ<ND>;
  const T a2 = a[Q::RHO] * ppb, b2 = b[Q::RHO] * ppa;
  if constexpr (LM == LM_PRELOG)
    log_means_prelog<T>(a[Q::RHO], b[Q::RHO], a2, b2, lg.la, lg.lb, lg.ls, L, Li);
  else if constexpr (LM == LM_ALG || LM == LM_ALG_POLY)
    log_means_alg<T, LM>(a[Q::RHO], b[Q::RHO], a2, b2, L, Li);
  else
    log_means<T, false>(a[Q::RHO], b[Q::RHO], a2, b2, L, Li);
}

// ---------------------------------------------------------------------------------------------------
// Ranocha's EC/KEP/PEP flux in directional form (Eq. flux_ranocha), scaled by 8:
//   F = 8 f(u_a, u_b, n2/2),  n2 = Ja^n_a + Ja^n_b (twice the averaged contravariant vector, Sec. 2.3).
// With A = v_a.n2, B = v_b.n2, L = {{rho}}_log, Li = 1/{{rho_a pp_b, rho_b pp_a}}_log, Q = L (A + B):
//   F_rho  = 2 Q                                          (8 {{rho}}_log {{v.n}})
//   F_rhov = Q (v_a + v_b) + (pp_a + pp_b) n2             (8 (f_rho {{v}} + {{p}} n))
//   F_rhoe = Q (v_a.v_b + pg_a pp_b Li) + pp_a B + pp_b A (8 (f_rho (v_a.v_b/2 + 1/({{rho/p}}_log (gamma-1)))
//                                                             + ((p; v.n))))
// using 1/{{rho/p}}_log = p_a p_b / {{rho_a p_b, rho_b p_a}}_log (Sec. 3.2) and the homogeneity of the mean.
// ---------------------------------------------------------------------------------------------------
// HALF0: return F_rho / 2 (= Q; the volume sums take it with doubled coefficients, which is exact and saves the
// addition Q + Q per pair).
// pp0 (FP32 mode with a reference pressure): the nodes' q[PP] hold pp - pp0; the momentum flux takes the shifted sum,
// everything else the pressure itself (pp0 = 0 and FP64: unshifted values, the same arithmetic as without it).
template <typename T>
__device__ __forceinline__ T unshift_pp(T pp, T pp0) {
  if constexpr (sizeof(T) == 8)
    return pp;
  else
    return pp + pp0;
}

// BETA (the volume terms, default log mean): the nodes' q[PG] hold beta = rho/p, the inverse mean is taken of beta
// directly, Li = 1/{{beta}}_log, and the energy flux's 1/({{rho/p}}_log (gamma-1)) term is c2 Li with
// c2 = 2/(gamma-1) (pg_a pp_b / {{rho_a pp_b, rho_b pp_a}}_log = 2/((gamma-1) {{beta}}_log by the homogeneity of the
// mean): the two products rho_a pp_b, rho_b pp_a and one product of the energy flux per pair become one reciprocal
// per node.
template <int ND, typename T, int LM = LM_SHARED_RCP, bool HALF0 = false, bool BETA = false>
__device__ __forceinline__ void ranocha_flux8(const T* a, const T* b, const T* n2, T* F,
                                              const LogRef<T>& lg = LogRef<T>{nullptr, nullptr, 0}, T pp0 = T(0),
                                              T c2 = T(0)) {
  using Q = NodeQ<ND>;
  static_assert(!BETA || LM == LM_SHARED_RCP, "the beta form serves the default log mean");
  T A = a[1] * n2[0], B = b[1] * n2[0], vv = a[1] * b[1];
#pragma unroll
  for (int j = 1; j < ND; ++j) {
    A += a[1 + j] * n2[j];
    B += b[1 + j] * n2[j];
    vv += a[1 + j] * b[1 + j];
  }
  const T ppa = unshift_pp(a[Q::PP], pp0), ppb = unshift_pp(b[Q::PP], pp0);
  T L, Li;
  if constexpr (BETA)
    log_means<T>(a[Q::RHO], b[Q::RHO], a[Q::PG], b[Q::PG], L, Li);
  else
    ranocha_means<ND, T, LM>(a, b, ppa, ppb, L, Li, lg);
  const T q = L * (A + B);
  const T ps = a[Q::PP] + b[Q::PP];
  F[0] = HALF0 ? q : q + q;
#pragma unroll
  for (int j = 0; j < ND; ++j) F[1 + j] = q * (a[1 + j] + b[1 + j]) + ps * n2[j];
  if constexpr (BETA)
    F[ND + 1] = q * (vv + c2 * Li) + (ppa * B + ppb * A);
  else
    F[ND + 1] = q * (vv + a[Q::PG] * ppb * Li) + (ppa * B + ppb * A);
}

// ---------------------------------------------------------------------------------------------------
// Flux of Shima et al. (Sec. 3.2, Eq. flux_shima_etal; kinetic energy and pressure equilibrium preserving, the
// paper's "cheap" flux), scaled by 8 like ranocha_flux8. With A = v_a.n2, B = v_b.n2, q = (rho_a + rho_b)(A + B):
//   F_rho  = q                                              (8 {{rho}} {{v.n}})
//   F_rhov = q (v_a + v_b)/2 + (pp_a + pp_b) n2              (8 (f_rho {{v}} + {{p}} n))
//   F_rhoe = q v_a.v_b/2 + (pg_a + pg_b)(A + B)/2 + pp_a B + pp_b A
//                                                          (8 (f_rho ((v;v))/2 + {{p}}{{v.n}}/(gamma-1) + ((p; v.n))))
// ---------------------------------------------------------------------------------------------------
template <int ND, typename T, bool HALF0 = false>
__device__ __forceinline__ void shima_flux8(const T* a, const T* b, const T* n2, T* F, T pp0 = T(0)) {
  using Q = NodeQ<ND>;
  T A = a[1] * n2[0], B = b[1] * n2[0], vv = a[1] * b[1];
#pragma unroll
  for (int j = 1; j < ND; ++j) {
    A += a[1 + j] * n2[j];
    B += b[1 + j] * n2[j];
    vv += a[1 + j] * b[1 + j];
  }
  const T AB = A + B;
  const T q = (a[Q::RHO] + b[Q::RHO]) * AB;
  const T hq = T(0.5) * q;
  const T ps = a[Q::PP] + b[Q::PP];
  F[0] = HALF0 ? hq : q;
#pragma unroll
  for (int j = 0; j < ND; ++j) F[1 + j] = hq * (a[1 + j] + b[1 + j]) + ps * n2[j];
  F[ND + 1] = hq * vv + T(0.5) * (a[Q::PG] + b[Q::PG]) * AB + (unshift_pp(a[Q::PP], pp0) * B +
                                                               unshift_pp(b[Q::PP], pp0) * A);
}

// ---------------------------------------------------------------------------------------------------
// The same fluxes on a Cartesian (affine, axis-aligned) element: the averaged contravariant vector of direction n
// has the single component n2n = 2 Ja^n_n along axis n, so v.n2 is one product and the pressure acts on one
// momentum component (van, vbn: the velocity components along n).
// ---------------------------------------------------------------------------------------------------
template <int ND, typename T, int FLUX, int LM = LM_SHARED_RCP, bool HALF0 = false, bool BETA = false>
__device__ __forceinline__ void pair_flux8_cart(const T* a, const T* b, T van, T vbn, T n2n, int n, T* F,
                                                const LogRef<T>& lg = LogRef<T>{nullptr, nullptr, 0}, T pp0 = T(0),
                                                T c2 = T(0)) {
  using Q = NodeQ<ND>;
  const T A = van * n2n, B = vbn * n2n;
  T vv = a[1] * b[1];
#pragma unroll
  for (int j = 1; j < ND; ++j) vv += a[1 + j] * b[1 + j];
  const T pn = (a[Q::PP] + b[Q::PP]) * n2n;
  const T ppa = unshift_pp(a[Q::PP], pp0), ppb = unshift_pp(b[Q::PP], pp0);
  T qv, e;
  if (FLUX == 0) {
    T L, Li;
    if constexpr (BETA)
      log_means<T>(a[Q::RHO], b[Q::RHO], a[Q::PG], b[Q::PG], L, Li);
    else
      ranocha_means<ND, T, LM>(a, b, ppa, ppb, L, Li, lg);
    const T q = L * (A + B);
    F[0] = HALF0 ? q : q + q;
    qv = q;
    if constexpr (BETA)
      e = q * (vv + c2 * Li);
    else
      e = q * (vv + a[Q::PG] * ppb * Li);
  } else {
    const T AB = A + B;
    const T q = (a[Q::RHO] + b[Q::RHO]) * AB;
    qv = T(0.5) * q;
    F[0] = HALF0 ? qv : q;
    e = qv * vv + T(0.5) * (a[Q::PG] + b[Q::PG]) * AB;
  }
#pragma unroll
  for (int j = 0; j < ND; ++j) F[1 + j] = qv * (a[1 + j] + b[1 + j]) + (j == n ? pn : T(0));
  F[ND + 1] = e + (ppa * B + ppb * A);
}

template <int ND, typename T, int FLUX, int LM = LM_SHARED_RCP, bool HALF0 = false, bool BETA = false>
__device__ __forceinline__ void pair_flux8(const T* a, const T* b, const T* n2, T* F,
                                           const LogRef<T>& lg = LogRef<T>{nullptr, nullptr, 0}, T pp0 = T(0),
                                           T c2 = T(0)) {
  if (FLUX == 0)
    ranocha_flux8<ND, T, LM, HALF0, BETA>(a, b, n2, F, lg, pp0, c2);
  else
    shima_flux8<ND, T, HALF0>(a, b, n2, F, pp0);
}

}  // namespace dgk

namespace dgk {

// ---------------------------------------------------------------------------------------------------
// Adjoint (reverse-mode derivative) arithmetic for dg_vjp.
// ---------------------------------------------------------------------------------------------------

// The two means of log_means and their exact partial derivatives. Series branches (u small):
//   L  = s P(u),  P = 1/2 - u/6 - 2u^2/45 - 22u^3/945,  dL/da = P - 4 (b/s) f P'(u),  dL/db = P + 4 (a/s) f P'(u)
//   Li = Q(u)/s,  Q = 2 + 2u/3 + 2u^2/5 + 2u^3/7,      dLi/da = -(Q + 4 (b/s) f Q'(u))/s^2,
//                                                      dLi/db = -(Q - 4 (a/s) f Q'(u))/s^2
// with s = a + b, f = (b - a)/s, u = f^2 (du/da = -4 b f/s^2, du/db = 4 a f/s^2). P' and Q' carry the next
// series term (856/14175 and 8/9) so that the derivatives are as accurate as the values.
// Log branches with l = log(b/a), d = b - a:  dL/da = (d/a - l)/l^2, dL/db = (l - d/b)/l^2,
//                                             dLi/da = (l - d/a)/d^2, dLi/db = (d/b - l)/d^2.
template <typename T>
__device__ __forceinline__ void log_means_grad(T a1, T b1, T a2, T b2, T& L, T& Li, T& dLa, T& dLb, T& dLia,
                                               T& dLib) {
  const T s1 = a1 + b1, d1 = b1 - a1;
  const T s2 = a2 + b2, d2 = b2 - a2;
  const T R = Num<T>::rcp(s1 * s2);
  const T r1 = s2 * R, r2 = s1 * R;
  const T f1 = d1 * r1, f2 = d2 * r2;
  const T u1 = f1 * f1, u2 = f2 * f2;
  if (Num<T>::series(u1)) {
    const T P = T(0.5) + u1 * (T(-1.0 / 6.0) + u1 * (T(-2.0 / 45.0) + u1 * T(-22.0 / 945.0)));
    const T dP = T(-1.0 / 6.0) + u1 * (T(-4.0 / 45.0) + u1 * (T(-66.0 / 945.0) + u1 * T(-856.0 / 14175.0)));
    L = s1 * P;
    const T g = T(4.0) * f1 * r1 * dP;  // 4 f P'/s
    dLa = P - b1 * g;
    dLb = P + a1 * g;
  } else {
    const T l = Num<T>::log(b1 / a1);
    const T il = T(1) / l;
    L = d1 * il;
    dLa = (d1 / a1 - l) * il * il;
    dLb = (l - d1 / b1) * il * il;
  }
  if (Num<T>::series(u2)) {
    const T Qv = T(2.0) + u2 * (T(2.0 / 3.0) + u2 * (T(2.0 / 5.0) + u2 * T(2.0 / 7.0)));
    const T dQ = T(2.0 / 3.0) + u2 * (T(4.0 / 5.0) + u2 * (T(6.0 / 7.0) + u2 * T(8.0 / 9.0)));
    Li = r2 * Qv;
    const T g = T(4.0) * f2 * r2 * dQ;  // 4 f Q'/s
    const T r22 = r2 * r2;
    dLia = -(Qv + b2 * g) * r22;
    dLib = -(Qv - a2 * g) * r22;
  } else {
    const T l = Num<T>::log(b2 / a2);
    const T id = T(1) / d2;
    Li = l * id;
    dLia = (l - d2 / a2) * id * id;
    dLib = (d2 / b2 - l) * id * id;
  }
}

// Adjoint of ranocha_flux8: given Fb = dJ/dF for F = ranocha_flux8(a, b, n2), adds dJ/da to abar and dJ/db to
// bbar (node quantities; n2 is geometry and has no adjoint here).
template <int ND, typename T>
__device__ __forceinline__ void ranocha_flux8_adjoint(const T* a, const T* b, const T* n2, const T* Fb, T* abar,
                                                      T* bbar) {
  using Q = NodeQ<ND>;
  T A = a[1] * n2[0], B = b[1] * n2[0], vv = a[1] * b[1];
#pragma unroll
  for (int j = 1; j < ND; ++j) {
    A += a[1 + j] * n2[j];
    B += b[1 + j] * n2[j];
    vv += a[1 + j] * b[1 + j];
  }
  T L, Li, dLa, dLb, dLix, dLiy;
  log_means_grad<T>(a[Q::RHO], b[Q::RHO], a[Q::RHO] * b[Q::PP], b[Q::RHO] * a[Q::PP], L, Li, dLa, dLb, dLix, dLiy);
  const T q = L * (A + B);
  const T t = a[Q::PG] * b[Q::PP] * Li;
  const T Fe = Fb[ND + 1];
  T qb = T(2) * Fb[0] + Fe * (vv + t);
  T psb = T(0);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    qb += Fb[1 + j] * (a[1 + j] + b[1 + j]);
    psb += Fb[1 + j] * n2[j];
  }
  const T vvb = Fe * q, tb = Fe * q;
  const T Ab = Fe * b[Q::PP] + qb * L;
  const T Bb = Fe * a[Q::PP] + qb * L;
  const T Lb = qb * (A + B);
  const T Lib = tb * a[Q::PG] * b[Q::PP];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    abar[1 + j] += Fb[1 + j] * q + vvb * b[1 + j] + Ab * n2[j];
    bbar[1 + j] += Fb[1 + j] * q + vvb * a[1 + j] + Bb * n2[j];
  }
  abar[Q::PG] += tb * b[Q::PP] * Li;
  bbar[Q::PP] += tb * a[Q::PG] * Li + Fe * A + psb;
  abar[Q::PP] += Fe * B + psb;
  const T x2b = Lib * dLix, y2b = Lib * dLiy;  // x2 = rho_a pp_b, y2 = rho_b pp_a
  abar[Q::RHO] += Lb * dLa + x2b * b[Q::PP];
  bbar[Q::RHO] += Lb * dLb + y2b * a[Q::PP];
  bbar[Q::PP] += x2b * a[Q::RHO];
  abar[Q::PP] += y2b * b[Q::RHO];
}

// Adjoint of node_quantities: ubar = (dq/du)^T qbar for q = (rho, v = m/rho, pp = 2p, pg = 2p/(gamma-1)),
// p = (gamma - 1)(E - |m|^2/(2 rho)).
template <int ND, typename T>
__device__ __forceinline__ void node_quantities_adjoint(const double* uc, T gm1, T two_over_gm1, const T* qbar,
                                                        T* ubar) {
  using Q = NodeQ<ND>;
  const T rho = (T)uc[0];
  const T ir = Num<T>::rcp(rho);
  const T pb = T(2) * qbar[Q::PP] + two_over_gm1 * qbar[Q::PG];
  T rb = qbar[Q::RHO], v2 = T(0);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const T v = (T)uc[1 + j] * ir;
    v2 += v * v;
    rb -= qbar[1 + j] * v * ir;
    ubar[1 + j] = qbar[1 + j] * ir - pb * gm1 * v;
  }
  ubar[0] = rb + pb * gm1 * T(0.5) * v2;
  ubar[ND + 1] = pb * gm1;
}

}  // namespace dgk
