// Volume kernels for 2D, FP64 flux arithmetic (see volume_impl.cuh).
#include "volume_impl.cuh"

namespace dgk {
template cudaError_t volume_dispatch<2, double>(int, MeshDims, const double*, const void*, const double*, const void*,
                                             double*, double, int*, cudaStream_t, const Epilogue*, const Variant*);
}  // namespace dgk
