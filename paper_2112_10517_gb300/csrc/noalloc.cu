// dg_rhs_noalloc: the RHS of dg_rhs for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host application whose memory manager owns all device memory (every
// allocation must go through its pool and its accounting), or code on a latency-critical path where an
// allocation or a free could synchronize the device. This entry point needs no context and allocates nothing:
// the caller passes the state, the metric terms and the output in its own device memory, and the interface
// fluxes, which dg_rhs keeps in a per-context workspace, live in one file-scope device array of fixed size.
#include <mutex>

#include "dg_internal.h"

namespace {

// Scratch shared by every call on a device: a 256-byte slot for the non-physical-state flag (used when the
// caller passes no flag), then the interface fluxes. Every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_rhs_scratch[DG_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_rhs_scratch on the current device (the host-side name is only a stand-in for it).
// Looked up once per device, on the first call made with that device current.
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_rhs_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

dg_status to_status(cudaError_t e) { return e == cudaSuccess ? DG_OK : DG_ERR_CUDA; }

}  // namespace

extern "C" dg_status dg_rhs_noalloc(int ndims, const int* nelem, int polydeg, int precision, int surface_flux,
                                    double gamma, const double* u, const void* Ja, const double* invJ, double* du,
                                    int* flag, dg_stream_t stream) {
  if ((ndims != 2 && ndims != 3) || !nelem || !u || !Ja || !invJ || !du) return DG_ERR_ARG;
  if (polydeg < 1 || polydeg >= DG_MAXN) return DG_ERR_UNSUPPORTED;
  if (precision != DG_FP64 && precision != DG_FP32) return DG_ERR_ARG;
  if (surface_flux != DG_SURF_EC && surface_flux != DG_SURF_EC_LLF) return DG_ERR_ARG;
  if (!(gamma > 1.0)) return DG_ERR_ARG;
  long long E = 1;
  for (int d = 0; d < ndims; ++d) {
    if (nelem[d] < 1 || nelem[d] > (1 << 20)) return DG_ERR_ARG;
    E *= nelem[d];
  }
  const int N = polydeg + 1, nv = ndims + 2;
  const long long face_nodes = ndims == 3 ? (long long)N * N : N;
  const long long Nd = face_nodes * N;
  if (E * Nd * nv > (1LL << 31) - 1) return DG_ERR_UNSUPPORTED;
  const size_t face_bytes =
      (size_t)ndims * E * nv * face_nodes * (precision == DG_FP32 ? sizeof(float) : sizeof(double));
  if (face_bytes > DG_NOALLOC_SCRATCH_BYTES - 256) return DG_ERR_UNSUPPORTED;  // mesh too large for the array
  const size_t state_bytes = (size_t)E * nv * Nd * sizeof(double);
  const char *ub = (const char*)u, *db = (const char*)du;
  if (ub < db + state_bytes && db < ub + state_bytes) return DG_ERR_ARG;  // u and du overlap
  // every array is read or written in whole elements: misaligned pointers are rejected before any launch
  if (((uintptr_t)u | (uintptr_t)du | (uintptr_t)invJ) & 7) return DG_ERR_ARG;
  if ((uintptr_t)Ja & (precision == DG_FP32 ? 3 : 7)) return DG_ERR_ARG;
  if ((uintptr_t)flag & 3) return DG_ERR_ARG;

  unsigned char* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return to_status(e);
  int* fl = flag ? flag : reinterpret_cast<int*>(scratch);
  cudaStream_t s = (cudaStream_t)stream;
  e = cudaMemsetAsync(fl, 0, sizeof(int), s);  // the flag must start at zero; the fluxes are overwritten in full
  if (e != cudaSuccess) return to_status(e);
  dgk::MeshDims md;
  md.n1 = nelem[0];
  md.n2 = nelem[1];
  md.n3 = ndims == 3 ? nelem[2] : 1;
  md.E = (int)E;
  void* face = scratch + 256;
  e = dgk::launch_interface(ndims, polydeg, precision, surface_flux == DG_SURF_EC_LLF, md, u, Ja, face, gamma, fl, s);
  if (e != cudaSuccess) return to_status(e);
  e = dgk::launch_volume(ndims, polydeg, precision, md, u, Ja, invJ, face, du, gamma, fl, s);
  return to_status(e);
}
