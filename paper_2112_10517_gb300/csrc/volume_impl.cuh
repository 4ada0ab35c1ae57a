// Volume-kernel launchers. volume_inst.cu instantiates launch_volume_n for one dimension, one flux precision and a
// range of node counts per object file (compiled several times with different -D settings, in parallel).
#pragma once

#include "kernels.cuh"
#include "volume_pipe.cuh"

namespace dgk {
namespace volume_detail {


// Threads per CTA the element tile aims at (elements per CTA = this / threads per element), by flux precision;
// compile-time tuning parameters. Measured at 16^3 and 32^3, p = 3 (3D): FP64 best at 192 (two CTAs of six warps
// per SM, bound by the FP64 pipe), FP32 at 96 (finer tiles and smaller shared-memory footprint for the
// memory-latency-bound kernel); tiles that leave a partial warp (144, 240) lose 10-20%.
#ifndef DG_VOLUME_TARGET_THREADS_F64
#define DG_VOLUME_TARGET_THREADS_F64 192
#endif
#ifndef DG_VOLUME_TARGET_THREADS_F32
#define DG_VOLUME_TARGET_THREADS_F32 96
#endif

template <int ND, int N, typename T>
constexpr int elems_per_block() {
  constexpr int target = sizeof(T) == 8 ? DG_VOLUME_TARGET_THREADS_F64 : DG_VOLUME_TARGET_THREADS_F32;
  return Geo<ND, N>::TPE >= target ? 1 : target / Geo<ND, N>::TPE;
}

// Threads per CTA of the pipelined kernel (FP32, FP64), and the fewest tiles per resident CTA for which
// DG_STAGING_AUTO uses it (compile-time tuning parameters, as above). With one tile per CTA nothing overlaps.
// Measured on the RK4 step (volume kernel, pipelined vs per-tile, FP32 / FP64): p = 3 at 16^3 (2.2 tiles per CTA in
// FP32, 3.4 in FP64) -15 % / -10 %, at 32^3 -34 % / -9 %; at about 2M DOF p = 1 -13 % / -14 %, p = 2 +25 % / -15 %,
// p = 4 -16 % / -7 %, p = 5 -27 % / -6 %, p = 6 -8 % / -9 %, p = 7 0 % / -11 %.
#ifndef DG_VOLUME_PIPE_TARGET_THREADS
#define DG_VOLUME_PIPE_TARGET_THREADS 96
#endif
#ifndef DG_VOLUME_PIPE_TARGET_THREADS_F64
#define DG_VOLUME_PIPE_TARGET_THREADS_F64 192
#endif
#ifndef DG_VOLUME_PIPE_MIN_TILES_PER_CTA
#define DG_VOLUME_PIPE_MIN_TILES_PER_CTA 2
#endif
// Tiles from a counter in the pipelined volume kernel (MeshTileSource), per precision. Measured on dg_rhs, p = 3,
// 16 x 16 x k elements (volume kernel, us, round-robin -> counter): FP64 k = 12: 138.6 -> 131.0, 16: 159.9 -> 163.7,
// 17: 182.2 -> 174.0, 19: 182.3 -> 185.8, 20: 202.8 -> 195.7, 32: 313.3 -> 305.3, where the launcher's prediction
// picks the faster in each of the ten sizes measured; FP32 (half tiles of one element) 16: 18.5 -> 22.6, 32:
// 28.8 -> 33.0, slower at every size but k = 12: FP32 keeps round-robin.
#ifndef DG_VOLUME_DYNAMIC_TILES_F64
#define DG_VOLUME_DYNAMIC_TILES_F64 1
#endif
#ifndef DG_VOLUME_DYNAMIC_TILES
#define DG_VOLUME_DYNAMIC_TILES 0
#endif

template <int N, typename T>
OpTable<N, T> op_table() {
  OpTable<N, T> op;
  const RefTables& t = ref_tables(N - 1);
  for (int i = 0; i < N * N; ++i) {
    op.Dt8[i] = (T)(0.125 * t.Dt[i]);
    op.D0[i] = (T)(0.25 * t.Dt[i]);
  }
  op.winv = (T)(1.0 / t.w[0]);
  op.lift8 = (T)(0.125 / t.w[0]);
  return op;
}

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// The pipelined kernel (volume_pipe.cuh) where it applies: the default log mean, shared memory within the opt-in
// limit, for even N 16-byte-aligned arrays (bulk copies), and (var.pipe == 1) enough tiles per resident CTA, or
// (var.pipe == 2) any mesh. Returns cudaErrorNotSupported where it does not apply (the caller then launches the
// per-tile kernel).
template <int ND, int N, typename T, int EPI, int LMK>
cudaError_t launch_volume_pipe(MeshDims md, const double* u, const T* Ja, const double* invJ, const T* face,
                               double* du, double gamma, int* flag, cudaStream_t s, const Epilogue& epi,
                               const Variant& var) {
  if constexpr (LMK == LM_SHARED_RCP) {
    constexpr int TPE = Geo<ND, N>::TPE;
    constexpr int target = sizeof(T) == 8 ? DG_VOLUME_PIPE_TARGET_THREADS_F64 : DG_VOLUME_PIPE_TARGET_THREADS;
    constexpr int EPB = TPE >= target ? 1 : target / TPE;
    constexpr bool fused = EPI != EPI_STORE;
    constexpr size_t smem = PipeSmem<ND, N, T>::bytes(EPB, fused);
    if constexpr (smem <= 227 * 1024) {
      if (!var.pipe) return cudaErrorNotSupported;
      if constexpr (PipeSmem<ND, N, T>::kBulk) {  // bulk copies start on 16-byte boundaries
        bool ok = aligned16(u) && aligned16(face) && (var.cart || (aligned16(Ja) && aligned16(invJ)));
        if (fused) ok = ok && aligned16(epi.u) && aligned16(EPI == EPI_RK4 ? epi.acc : epi.y);
        if (!ok) return cudaErrorNotSupported;
      }
      auto kern = volume_pipe_kernel<ND, N, T, EPB, EPI>;
      // occupancy and SM count of the device (resident CTAs: their product), computed once per device together
      // with the opt-in
      static PerDeviceCache cache;
      long long occ_sms = 0;
      cudaError_t ce = per_device(cache, &occ_sms, [&](long long* v) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, occ = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, EPB * TPE, smem)) != cudaSuccess)
          return e;
        if (occ < 1) return cudaErrorNotSupported;
        *v = ((long long)occ << 32) | (long long)sms;
        return cudaSuccess;
      });
      if (ce != cudaSuccess) return ce;
      const int sms = (int)(occ_sms & 0xFFFFFFFF);
      const long long ctas = (occ_sms >> 32) * sms;
      const int ntiles = (md.E - var.ghost + EPB - 1) / EPB;  // from element var.ghost on
      // auto: enough tiles per CTA, and not FP32 at p = 2 (3 elements of 27 threads per CTA, each thread issuing
      // many small copies: measured 25 % slower than the per-tile kernel; every other degree and precision gains)
      constexpr bool kAutoOk = !(sizeof(T) == 4 && N == 3);
      if (var.pipe == 1 && (!kAutoOk || (long long)ntiles < (long long)DG_VOLUME_PIPE_MIN_TILES_PER_CTA * ctas))
        return cudaErrorNotSupported;
      const int grid = ntiles < ctas ? ntiles : (int)ctas;
      // round-robin, or tiles from the context's counter with the last round in half tiles (tile_plan.h), only
      // where a half tile's lines of one direction fill whole warps (the pair phase assigns threads
      // direction-major: 3D p = 3 and p = 1; elsewhere its warps would run partly empty)
      constexpr bool kHalfWarps = EPB % 2 == 0 && (EPB / 2) * Geo<ND, N>::NL % 32 == 0;
      constexpr bool kDyn = kHalfWarps && (sizeof(T) == 8 ? DG_VOLUME_DYNAMIC_TILES_F64 : DG_VOLUME_DYNAMIC_TILES);
      const TilePlan tp = tile_plan(md.E - var.ghost, EPB, grid, sms, kDyn && var.tiles != nullptr);
      const cudaError_t e =
          launch_kernel(kern, dim3(grid), dim3(EPB * TPE), smem, s, var.overlap != 0, u, Ja, invJ, face, du, md,
                        op_table<N, T>(), (T)gamma, flag, epi, var, tp.ntiles, tp.nfull, tp.counter ? var.tiles : nullptr);
      return e != cudaSuccess ? e : cudaGetLastError();
    }
  }
  return cudaErrorNotSupported;
}

template <int ND, int N, typename T, int EPI, int LMK>
cudaError_t launch_volume_k(MeshDims md, const double* u, const T* Ja, const double* invJ, const T* face, double* du,
                            double gamma, int* flag, cudaStream_t s, const Epilogue& epi, const Variant& var) {
  const cudaError_t pe = launch_volume_pipe<ND, N, T, EPI, LMK>(md, u, Ja, invJ, face, du, gamma, flag, s, epi, var);
  if (pe != cudaErrorNotSupported) return pe;
  constexpr int EPB = elems_per_block<ND, N, T>();
  constexpr int threads = EPB * Geo<ND, N>::TPE;
  const size_t smem = VolumeSmem<ND, N, T>::bytes(EPB, EPI != EPI_STORE, LMK == LM_PRELOG);
  auto kern = volume_kernel<ND, N, T, EPB, EPI, LMK>;
  static PerDeviceCache cache;  // the shared-memory opt-in, once per device
  long long done = 0;
  cudaError_t ae = per_device(cache, &done, [&](long long* v) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    *v = 1;
    return e;
  });
  if (ae != cudaSuccess) return ae;
  const int blocks = (md.E - var.ghost + EPB - 1) / EPB;  // from element var.ghost on
  kern<<<blocks, threads, smem, s>>>(u, Ja, invJ, face, du, md, op_table<N, T>(), (T)gamma, flag, epi, var);
  return cudaGetLastError();
}

// the log-mean variants: all four for dg_rhs; the default and precomputed logarithms for the fused stage update
template <int ND, int N, typename T, int EPI>
cudaError_t launch_volume_e(MeshDims md, const double* u, const T* Ja, const double* invJ, const T* face, double* du,
                            double gamma, int* flag, cudaStream_t s, const Epilogue& epi, const Variant& var) {
  if (var.lm == LM_PRELOG)
    return launch_volume_k<ND, N, T, EPI, LM_PRELOG>(md, u, Ja, invJ, face, du, gamma, flag, s, epi, var);
  if constexpr (EPI == EPI_STORE) {
    if (var.lm == LM_ALG)
      return launch_volume_k<ND, N, T, EPI, LM_ALG>(md, u, Ja, invJ, face, du, gamma, flag, s, epi, var);
    if (var.lm == LM_ALG_POLY)
      return launch_volume_k<ND, N, T, EPI, LM_ALG_POLY>(md, u, Ja, invJ, face, du, gamma, flag, s, epi, var);
  } else {
    if (var.lm != LM_SHARED_RCP) return cudaErrorInvalidValue;
  }
  return launch_volume_k<ND, N, T, EPI, LM_SHARED_RCP>(md, u, Ja, invJ, face, du, gamma, flag, s, epi, var);
}

template <int ND, int N, typename T>
cudaError_t launch_volume_t(MeshDims md, const double* u, const T* Ja, const double* invJ, const T* face, double* du,
                            double gamma, int* flag, cudaStream_t s, const Epilogue* epi, const Variant* var) {
  Variant v{};  // default: Ranocha's flux, metric arrays
  if (var) v = *var;
  if (!epi || epi->mode == EPI_STORE) {
    Epilogue none{};
    none.mode = EPI_STORE;
    return launch_volume_e<ND, N, T, EPI_STORE>(md, u, Ja, invJ, face, du, gamma, flag, s, none, v);
  }
  if (epi->mode == EPI_RK4)
    return launch_volume_e<ND, N, T, EPI_RK4>(md, u, Ja, invJ, face, du, gamma, flag, s, *epi, v);
  return launch_volume_e<ND, N, T, EPI_CK45>(md, u, Ja, invJ, face, du, gamma, flag, s, *epi, v);
}

}  // namespace volume_detail

template <int ND, int N, typename T>
cudaError_t launch_volume_n(MeshDims md, const double* u, const T* Ja, const double* invJ, const T* face, double* du,
                            double gamma, int* flag, cudaStream_t s, const Epilogue* epi, const Variant* var) {
  return volume_detail::launch_volume_t<ND, N, T>(md, u, Ja, invJ, face, du, gamma, flag, s, epi, var);
}

}  // namespace dgk
