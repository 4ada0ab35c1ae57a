// Instantiation and launch of the interface-flux kernel.
#include "kernels.cuh"

namespace dgk {
namespace {

template <int ND, int N, typename T>
cudaError_t launch_interface_t(int llf, MeshDims md, const double* u, const T* Ja, T* face, double gamma, int* flag,
                               cudaStream_t s, const Variant& var) {
  const long long total = (long long)ND * ((var.if_e1 > 0 ? var.if_e1 : md.E) - var.if_e0) * Geo<ND, N>::NL;
  if (total <= 0) return cudaSuccess;
  // 128 threads per CTA: at 96 registers (FP64) five CTAs fit per SM (20 warps, 94 % of the register file)
  // where two of 256 threads left a quarter of it unused, and a 16^3 launch (1,536 CTAs, 10.1 per SM) balances
  // to within one CTA per SM instead of 2.5 waves of the larger CTAs. Measured on the 16^3 RK4 step: FP64 -2 %,
  // FP32 -1 % against 256 threads; 64 threads measure the same as 128.
  const int threads = 128;
  const long long blocks = (total + threads - 1) / threads;
  auto kern = llf ? interface_kernel<ND, N, T, true> : interface_kernel<ND, N, T, false>;
  if constexpr (sizeof(T) == 4) kern = llf ? interface_kernel_f32<ND, N, true> : interface_kernel_f32<ND, N, false>;
  const cudaError_t e = launch_kernel(kern, dim3((unsigned)blocks), dim3(threads), 0, s, var.overlap != 0, u, Ja, face,
                                      md, (T)gamma, flag, var);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int ND, typename T>
cudaError_t dispatch_p(int p, int llf, MeshDims md, const double* u, const void* Ja, void* face, double gamma,
                       int* flag, cudaStream_t s, const Variant& var) {
  const T* ja = static_cast<const T*>(Ja);
  T* fc = static_cast<T*>(face);
  switch (p) {
    case 1: return launch_interface_t<ND, 2, T>(llf, md, u, ja, fc, gamma, flag, s, var);
    case 2: return launch_interface_t<ND, 3, T>(llf, md, u, ja, fc, gamma, flag, s, var);
    case 3: return launch_interface_t<ND, 4, T>(llf, md, u, ja, fc, gamma, flag, s, var);
    case 4: return launch_interface_t<ND, 5, T>(llf, md, u, ja, fc, gamma, flag, s, var);
    case 5: return launch_interface_t<ND, 6, T>(llf, md, u, ja, fc, gamma, flag, s, var);
    case 6: return launch_interface_t<ND, 7, T>(llf, md, u, ja, fc, gamma, flag, s, var);
    case 7: return launch_interface_t<ND, 8, T>(llf, md, u, ja, fc, gamma, flag, s, var);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_interface(int nd, int p, int precision, int llf, MeshDims md, const double* u, const void* Ja,
                             void* face, double gamma, int* flag, cudaStream_t s, const Variant* var) {
  if (md.E <= 0) return cudaSuccess;
  Variant v{};  // default: Ranocha's flux, metric arrays
  if (var) v = *var;
  if (nd == 2)
    return precision == DG_FP32 ? dispatch_p<2, float>(p, llf, md, u, Ja, face, gamma, flag, s, v)
                                : dispatch_p<2, double>(p, llf, md, u, Ja, face, gamma, flag, s, v);
  return precision == DG_FP32 ? dispatch_p<3, float>(p, llf, md, u, Ja, face, gamma, flag, s, v)
                              : dispatch_p<3, double>(p, llf, md, u, Ja, face, gamma, flag, s, v);
}

}  // namespace dgk
