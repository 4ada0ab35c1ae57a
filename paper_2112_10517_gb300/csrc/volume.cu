// Volume kernel (flux differencing + surface lift + Jacobian scaling [+ fused RK stage update]): dispatch by
// dimension and precision; the kernels are instantiated in volume_{2d,3d}_{f64,f32}.cu.
#include "kernels.cuh"

namespace dgk {

template <int ND, typename T>
cudaError_t volume_dispatch(int p, MeshDims md, const double* u, const void* Ja, const double* invJ, const void* face,
                            double* du, double gamma, int* flag, cudaStream_t s, const Epilogue* epi,
                            const Variant* var);
extern template cudaError_t volume_dispatch<2, double>(int, MeshDims, const double*, const void*, const double*,
                                                       const void*, double*, double, int*, cudaStream_t,
                                                       const Epilogue*, const Variant*);
extern template cudaError_t volume_dispatch<2, float>(int, MeshDims, const double*, const void*, const double*,
                                                      const void*, double*, double, int*, cudaStream_t, const Epilogue*,
                                                      const Variant*);
extern template cudaError_t volume_dispatch<3, double>(int, MeshDims, const double*, const void*, const double*,
                                                       const void*, double*, double, int*, cudaStream_t,
                                                       const Epilogue*, const Variant*);
extern template cudaError_t volume_dispatch<3, float>(int, MeshDims, const double*, const void*, const double*,
                                                      const void*, double*, double, int*, cudaStream_t, const Epilogue*,
                                                      const Variant*);

cudaError_t launch_volume(int nd, int p, int precision, MeshDims md, const double* u, const void* Ja,
                          const double* invJ, const void* face, double* du, double gamma, int* flag, cudaStream_t s,
                          const Epilogue* epi, const Variant* var) {
  if (md.E <= 0) return cudaSuccess;
  if (nd == 2)
    return precision == DG_FP32 ? volume_dispatch<2, float>(p, md, u, Ja, invJ, face, du, gamma, flag, s, epi, var)
                                : volume_dispatch<2, double>(p, md, u, Ja, invJ, face, du, gamma, flag, s, epi, var);
  return precision == DG_FP32 ? volume_dispatch<3, float>(p, md, u, Ja, invJ, face, du, gamma, flag, s, epi, var)
                              : volume_dispatch<3, double>(p, md, u, Ja, invJ, face, du, gamma, flag, s, epi, var);
}

}  // namespace dgk
