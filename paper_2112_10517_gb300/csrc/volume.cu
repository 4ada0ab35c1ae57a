// Volume kernel (flux differencing + surface lift + Jacobian scaling [+ fused RK stage update]): dispatch by
// dimension, precision and polynomial degree; the kernels are instantiated in volume_inst.cu.
#include "kernels.cuh"

namespace dgk {

template <int ND, int N, typename T>
cudaError_t launch_volume_n(MeshDims md, const double* u, const T* Ja, const double* invJ, const T* face, double* du,
                            double gamma, int* flag, cudaStream_t s, const Epilogue* epi, const Variant* var);

#define DG_VOLUME_EXTERN(ND, N, T)                                                                              \
  extern template cudaError_t launch_volume_n<ND, N, T>(MeshDims, const double*, const T*, const double*,     \
                                                        const T*, double*, double, int*, cudaStream_t,          \
                                                        const Epilogue*, const Variant*);
#define DG_VOLUME_EXTERN_ALL(ND, T) \
  DG_VOLUME_EXTERN(ND, 2, T)        \
  DG_VOLUME_EXTERN(ND, 3, T)        \
  DG_VOLUME_EXTERN(ND, 4, T)        \
  DG_VOLUME_EXTERN(ND, 5, T)        \
  DG_VOLUME_EXTERN(ND, 6, T)        \
  DG_VOLUME_EXTERN(ND, 7, T)        \
  DG_VOLUME_EXTERN(ND, 8, T)
DG_VOLUME_EXTERN_ALL(2, double)
DG_VOLUME_EXTERN_ALL(2, float)
DG_VOLUME_EXTERN_ALL(3, double)
DG_VOLUME_EXTERN_ALL(3, float)

namespace {
template <int ND, typename T>
cudaError_t dispatch_p(int p, MeshDims md, const double* u, const void* Ja, const double* invJ, const void* face,
                       double* du, double gamma, int* flag, cudaStream_t s, const Epilogue* epi, const Variant* var) {
  const T* ja = static_cast<const T*>(Ja);
  const T* fc = static_cast<const T*>(face);
  switch (p) {
    case 1: return launch_volume_n<ND, 2, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    case 2: return launch_volume_n<ND, 3, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    case 3: return launch_volume_n<ND, 4, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    case 4: return launch_volume_n<ND, 5, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    case 5: return launch_volume_n<ND, 6, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    case 6: return launch_volume_n<ND, 7, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    case 7: return launch_volume_n<ND, 8, T>(md, u, ja, invJ, fc, du, gamma, flag, s, epi, var);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_volume(int nd, int p, int precision, MeshDims md, const double* u, const void* Ja,
                          const double* invJ, const void* face, double* du, double gamma, int* flag, cudaStream_t s,
                          const Epilogue* epi, const Variant* var) {
  if (md.E <= 0) return cudaSuccess;
  if (nd == 2)
    return precision == DG_FP32 ? dispatch_p<2, float>(p, md, u, Ja, invJ, face, du, gamma, flag, s, epi, var)
                                : dispatch_p<2, double>(p, md, u, Ja, invJ, face, du, gamma, flag, s, epi, var);
  return precision == DG_FP32 ? dispatch_p<3, float>(p, md, u, Ja, invJ, face, du, gamma, flag, s, epi, var)
                              : dispatch_p<3, double>(p, md, u, Ja, invJ, face, du, gamma, flag, s, epi, var);
}

}  // namespace dgk
