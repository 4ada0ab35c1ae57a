// ALU throughput microbenchmarks for the roofline denominators of the RHS kernels.
//
// The volume term of flux-differencing DGSEM (Sec. 2.1-2.3, Eq. fluxdiff-SBP-opDsplit) is bound by
// floating-point arithmetic, not by memory, so its roofline needs the device's FP64 and FP32 FMA rates
// and the rates of the special operations the two-point flux uses (division, logarithm; Sec. 3.1).
// Each kernel runs many independent dependency chains per thread so that the pipe, not latency, limits it.
// Exported with a C ABI (plain pointers and sizes); the caller reads ops/second.

#include <cuda_runtime.h>
#include <stdint.h>

#include "dgmath.cuh"

namespace {

constexpr int kChains = 8;

enum Kind : int {
  K_DFMA = 0,      // fp64 fused multiply-add (2 flop)
  K_FFMA = 1,      // fp32 fused multiply-add (2 flop)
  K_DDIV = 2,      // fp64 IEEE division a/b
  K_DLOG = 3,      // fp64 log()
  K_FLOG = 4,      // fp32 logf()
  K_MUFU_LG2 = 5,  // fp32 lg2.approx (special-function unit)
  K_MUFU_RCP = 6,  // fp32 rcp.approx (special-function unit)
  K_FDIV = 7,      // fp32 IEEE division
  K_DRCP = 8,      // fp64 reciprocal, round to nearest
  K_DLOG_OWN = 9,  // fp64 log_f64 of the RHS kernels
  K_DEXP = 10,     // fp64 exp()
  K_DSQRT = 11,    // fp64 sqrt()
  K_DSQRT_OWN = 12,  // fp64 sqrt_f64 of the RHS kernels
  K_NKINDS = 13
};

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float r;
  asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <int KIND>
__global__ void chain_kernel(double* sink, int iters, double seed) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double d[kChains];
  float f[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    d[c] = 1.0 + 1e-3 * (double)((tid + c) & 15);
    f[c] = 1.0f + 1e-3f * (float)((tid + c) & 15);
  }
  const double b = 0.999999 * seed, a = 1e-7 * seed;
  const float bf = (float)b, af = (float)a;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if (KIND == K_DFMA) d[c] = fma(d[c], b, a);
      if (KIND == K_FFMA) {
        f[c] = fmaf(f[c], bf, af);
        f[c + 0] = fmaf(f[c], bf, af);  // two per chain step keep fp32 issue dense
      }
      if (KIND == K_DDIV) d[c] = 2.0 + b / d[c];
      if (KIND == K_DLOG) d[c] = 1.0 + log(d[c] + b);
      if (KIND == K_FLOG) f[c] = 1.0f + logf(f[c] + bf);
      if (KIND == K_MUFU_LG2) f[c] = lg2_approx(f[c] + bf);
      if (KIND == K_MUFU_RCP) f[c] = rcp_approx(f[c] + af);
      if (KIND == K_FDIV) f[c] = 2.0f + bf / f[c];
      if (KIND == K_DRCP) d[c] = 2.0 + __drcp_rn(d[c]);
      if (KIND == K_DLOG_OWN) d[c] = 1.0 + dgk::log_f64(d[c] + b);
      if (KIND == K_DEXP) d[c] = exp(0.5 - d[c] * a);
      if (KIND == K_DSQRT) d[c] = 0.5 + sqrt(d[c] + b);
      if (KIND == K_DSQRT_OWN) d[c] = 0.5 + dgk::sqrt_f64(d[c] + b);
    }
  }
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += d[c] + (double)f[c];
  if (acc == seed * 12345.678) sink[tid] = acc;  // never true for the seeds used; keeps the chains live
}

// operations counted per chain step (FFMA does two dependent FMAs per chain step)
__host__ int ops_per_step(int kind) { return kind == K_FFMA ? 2 : 1; }

template <int KIND>
cudaError_t launch(int blocks, int threads, double* sink, int iters, cudaStream_t s) {
  chain_kernel<KIND><<<blocks, threads, 0, s>>>(sink, iters, 1.0);
  return cudaGetLastError();
}

cudaError_t launch_kind(int kind, int blocks, int threads, double* sink, int iters, cudaStream_t s) {
  switch (kind) {
    case K_DFMA: return launch<K_DFMA>(blocks, threads, sink, iters, s);
    case K_FFMA: return launch<K_FFMA>(blocks, threads, sink, iters, s);
    case K_DDIV: return launch<K_DDIV>(blocks, threads, sink, iters, s);
    case K_DLOG: return launch<K_DLOG>(blocks, threads, sink, iters, s);
    case K_FLOG: return launch<K_FLOG>(blocks, threads, sink, iters, s);
    case K_MUFU_LG2: return launch<K_MUFU_LG2>(blocks, threads, sink, iters, s);
    case K_MUFU_RCP: return launch<K_MUFU_RCP>(blocks, threads, sink, iters, s);
    case K_FDIV: return launch<K_FDIV>(blocks, threads, sink, iters, s);
    case K_DRCP: return launch<K_DRCP>(blocks, threads, sink, iters, s);
    case K_DLOG_OWN: return launch<K_DLOG_OWN>(blocks, threads, sink, iters, s);
    case K_DEXP: return launch<K_DEXP>(blocks, threads, sink, iters, s);
    case K_DSQRT: return launch<K_DSQRT>(blocks, threads, sink, iters, s);
    case K_DSQRT_OWN: return launch<K_DSQRT_OWN>(blocks, threads, sink, iters, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
__global__ void logmeans_kernel(long long n, const double* a1, const double* b1, const double* a2, const double* b2,
                                double* L, double* Li, double* r) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T l, li;
  dgk::log_means<T>((T)a1[i], (T)b1[i], (T)a2[i], (T)b2[i], l, li);
  L[i] = (double)l;
  Li[i] = (double)li;
  r[i] = (double)dgk::Num<T>::rcp((T)a1[i]);
}

__global__ void convert_kernel(long long n, const double* x, unsigned* f_int, unsigned* f_hw, double* d_int,
                               double* d_hw) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float hw = __double2float_rn(x[i]);
  f_int[i] = __float_as_uint(dgk::d2f_int(x[i]));
  f_hw[i] = __float_as_uint(hw);
  d_int[i] = dgk::f2d_int(hw);
  d_hw[i] = (double)hw;
}

__global__ void split_kernel(long long n, const double* x, const double* ref, float* hi, float* lo, float* rel) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float h = dgk::d2f_int(x[i]);
  hi[i] = h;
  lo[i] = dgk::split_lo_f64(x[i], h);
  const float rh = dgk::d2f_int(ref[i]);
  rel[i] = dgk::energy_rel<float>(x[i], rh, dgk::split_lo_f64(ref[i], rh));
}

__global__ void log_kernel(long long n, const double* x, double* log_own, double* log_ref) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  log_own[i] = dgk::log_f64(x[i]);
  log_ref[i] = log(x[i]);
}

__global__ void sqrt_kernel(long long n, const double* x, double* own, double* ref) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  own[i] = dgk::sqrt_f64(x[i]);
  ref[i] = sqrt(x[i]);
}

}  // namespace

extern "C" {

__global__ void sqrt_wave_kernel(long long n, const double* x, double* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = dgk::sqrt_wave_f64(x[i]);
}

int dgpk_eval_sqrt_wave(long long n, const double* x, double* out) {
  if (n <= 0) return 0;
  sqrt_wave_kernel<<<(unsigned)((n + 255) / 256), 256>>>(n, x, out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}

// Self-test of the RHS kernels' FP64 square root against CUDA's sqrt: own/ref = sqrt_f64(x[i]) / sqrt(x[i]).
int dgpk_eval_sqrt(long long n, const double* x, double* own, double* ref) {
  if (n <= 0) return 0;
  sqrt_kernel<<<(unsigned)((n + 255) / 256), 256>>>(n, x, own, ref);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}

// Self-test of the RHS kernels' FP64 logarithm against CUDA's log: for i < n, log_own/log_ref = log_f64(x[i]) /
// log(x[i]). Device arrays; synchronizes; returns 0 or a cudaError_t value.
int dgpk_eval_log(long long n, const double* x, double* log_own, double* log_ref) {
  if (n <= 0) return 0;
  log_kernel<<<(unsigned)((n + 255) / 256), 256>>>(n, x, log_own, log_ref);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}

// Self-test of the integer-pipe format conversions of the RHS kernels against the hardware conversions: for
// i < n, f_int[i] / f_hw[i] = bits of d2f_int(x[i]) / __double2float_rn(x[i]); d_int[i] / d_hw[i] = f2d_int and
// the hardware widening of that float. Device arrays; synchronizes; returns 0 or a cudaError_t value.
int dgpk_eval_split(long long n, const double* x, const double* ref, float* hi, float* lo, float* rel) {
  if (n <= 0) return 0;
  split_kernel<<<(unsigned)((n + 255) / 256), 256>>>(n, x, ref, hi, lo, rel);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}

int dgpk_eval_convert(long long n, const double* x, unsigned* f_int, unsigned* f_hw, double* d_int, double* d_hw) {
  if (n <= 0) return 0;
  convert_kernel<<<(unsigned)((n + 255) / 256), 256>>>(n, x, f_int, f_hw, d_int, d_hw);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}

// Evaluates the RHS kernels' device arithmetic on n inputs (device arrays): L = {{a1, b1}}_log (Algorithm 2),
// Li = 1/{{a2, b2}}_log (Algorithm 3), both from the single shared reciprocal, and r = the reciprocal of a1,
// in FP64 (precision 0) or FP32 (precision 1; inputs rounded to float, results widened). Queues on the legacy
// default stream and synchronizes. Returns 0 or a cudaError_t value.
int dgpk_eval_logmeans(long long n, int precision, const double* a1, const double* b1, const double* a2,
                       const double* b2, double* L, double* Li, double* r) {
  if (n <= 0) return 0;
  const int threads = 256;
  const long long blocks = (n + threads - 1) / threads;
  if (precision == 1)
    logmeans_kernel<float><<<(unsigned)blocks, threads>>>(n, a1, b1, a2, b2, L, Li, r);
  else
    logmeans_kernel<double><<<(unsigned)blocks, threads>>>(n, a1, b1, a2, b2, L, Li, r);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}


// Number of benchmark kinds; kind ids are listed in include/dg_peaks.h.
int dgpk_num_kinds(void) { return K_NKINDS; }

// Runs benchmark `kind` on the current device and returns operations per second in *ops_per_s
// (an FMA counts as one operation; multiply by 2 for flop/s). The iteration count is grown until one
// launch takes at least `min_seconds`. Returns 0 on success, else a cudaError_t value.
int dgpk_measure(int kind, double min_seconds, double* ops_per_s, double* seconds) {
  if (kind < 0 || kind >= K_NKINDS || !ops_per_s) return (int)cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int threads = 256, blocks = sms * 8;
  double* sink = nullptr;
  e = cudaMalloc(&sink, sizeof(double) * (size_t)threads * blocks);
  if (e != cudaSuccess) return (int)e;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  int iters = 64;
  float ms = 0.f;
  // warm-up launch
  e = launch_kind(kind, blocks, threads, sink, iters, 0);
  for (int attempt = 0; attempt < 24 && e == cudaSuccess; ++attempt) {
    cudaEventRecord(t0, 0);
    e = launch_kind(kind, blocks, threads, sink, iters, 0);
    cudaEventRecord(t1, 0);
    if (e != cudaSuccess) break;
    e = cudaEventSynchronize(t1);
    if (e != cudaSuccess) break;
    cudaEventElapsedTime(&ms, t0, t1);
    if (ms * 1e-3 >= min_seconds || iters > (1 << 26)) break;
    const double grow = ms > 0.5f ? (min_seconds * 1e3 / ms) * 1.2 : 16.0;
    iters = (int)(iters * (grow > 16.0 ? 16.0 : (grow < 2.0 ? 2.0 : grow)));
  }
  if (e == cudaSuccess) {
    const double ops = (double)blocks * threads * kChains * (double)iters * ops_per_step(kind);
    *ops_per_s = ops / (ms * 1e-3);
    if (seconds) *seconds = ms * 1e-3;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(sink);
  return (int)e;
}

}  // extern "C"
