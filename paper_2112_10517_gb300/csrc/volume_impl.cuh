// Volume-kernel launchers, instantiated per dimension and flux precision in volume_{2d,3d}_{f64,f32}.cu (separate
// translation units so that the build compiles them in parallel).
#pragma once

#include "kernels.cuh"

namespace dgk {
namespace volume_detail {


constexpr int kTargetThreads = 192;

template <int ND, int N>
constexpr int elems_per_block() {
  return Geo<ND, N>::TPE >= kTargetThreads ? 1 : kTargetThreads / Geo<ND, N>::TPE;
}

template <int ND, int N, typename T, int EPI>
cudaError_t launch_volume_e(MeshDims md, const double* u, const T* Ja, const double* invJ, const T* face, double* du,
                            double gamma, int* flag, cudaStream_t s, const Epilogue& epi, const Variant& var) {
  constexpr int EPB = elems_per_block<ND, N>();
  constexpr int threads = EPB * Geo<ND, N>::TPE;
  const size_t smem = VolumeSmem<ND, N, T>::bytes(EPB, EPI != EPI_STORE);
  auto kern = volume_kernel<ND, N, T, EPB, EPI>;
  static bool attr_set = false;  // idempotent; a benign race sets the same value twice
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  OpTable<N, T> op;
  const RefTables& t = ref_tables(N - 1);
  for (int i = 0; i < N * N; ++i) op.Dt8[i] = (T)(0.125 * t.Dt[i]);
  op.winv = (T)(1.0 / t.w[0]);
  const int blocks = (md.E + EPB - 1) / EPB;
  kern<<<blocks, threads, smem, s>>>(u, Ja, invJ, face, du, md, op, (T)gamma, flag, epi, var);
  return cudaGetLastError();
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

template <int ND, typename T>
cudaError_t dispatch_p_impl(int p, MeshDims md, const double* u, const void* Ja, const double* invJ, const void* face,
                       double* du, double gamma, int* flag, cudaStream_t s, const Epilogue* epi, const Variant* var) {
  const T* ja = static_cast<const T*>(Ja);
  const T* fc = static_cast<const T*>(face);
  switch (p) {
    case 1: return launch_volume_t<ND, 2, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    case 2: return launch_volume_t<ND, 3, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    case 3: return launch_volume_t<ND, 4, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    case 4: return launch_volume_t<ND, 5, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    case 5: return launch_volume_t<ND, 6, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    case 6: return launch_volume_t<ND, 7, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    case 7: return launch_volume_t<ND, 8, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace volume_detail

template <int ND, typename T>
cudaError_t volume_dispatch(int p, MeshDims md, const double* u, const void* Ja, const double* invJ, const void* face,
                            double* du, double gamma, int* flag, cudaStream_t s, const Epilogue* epi,
                            const Variant* var) {
  return volume_detail::dispatch_p_impl<ND, T>(p, md, u, Ja, invJ, face, du, gamma, flag, s, epi, var);
}

}  // namespace dgk
