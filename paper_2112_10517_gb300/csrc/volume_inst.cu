// Instantiations of the volume-kernel launcher for VOL_ND dimensions, flux type VOL_T and node counts
// VOL_NLO..VOL_NHI. The build compiles this file once per (dimension, precision, node range) so that the kernels
// compile in parallel; volume.cu dispatches to them.
#include "volume_impl.cuh"

#if !defined(VOL_ND) || !defined(VOL_T) || !defined(VOL_NLO) || !defined(VOL_NHI)
#error "volume_inst.cu needs -DVOL_ND=.. -DVOL_T=.. -DVOL_NLO=.. -DVOL_NHI=.."
#endif

#define DG_VOLUME_INST(N)                                                                                      \
  template cudaError_t launch_volume_n<VOL_ND, N, VOL_T>(MeshDims, const double*, const VOL_T*, const double*, \
                                                         const VOL_T*, double*, double, int*, cudaStream_t,     \
                                                         const Epilogue*, const Variant*);

namespace dgk {
#if VOL_NLO <= 2 && 2 <= VOL_NHI
DG_VOLUME_INST(2)
#endif
#if VOL_NLO <= 3 && 3 <= VOL_NHI
DG_VOLUME_INST(3)
#endif
#if VOL_NLO <= 4 && 4 <= VOL_NHI
DG_VOLUME_INST(4)
#endif
#if VOL_NLO <= 5 && 5 <= VOL_NHI
DG_VOLUME_INST(5)
#endif
#if VOL_NLO <= 6 && 6 <= VOL_NHI
DG_VOLUME_INST(6)
#endif
#if VOL_NLO <= 7 && 7 <= VOL_NHI
DG_VOLUME_INST(7)
#endif
#if VOL_NLO <= 8 && 8 <= VOL_NHI
DG_VOLUME_INST(8)
#endif
}  // namespace dgk
