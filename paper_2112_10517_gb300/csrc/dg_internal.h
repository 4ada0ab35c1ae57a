// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dg.h"

#define DG_MAXN 8  // polydeg <= 7

namespace dgk {

// Per-launch geometry of a structured periodic mesh.
struct MeshDims {
  int n1, n2, n3;  // elements per direction (n3 = 1 in 2D)
  int E;
};

// Device tables for one polynomial degree (host copies; uploaded to constant memory once per device).
struct RefTables {
  double x[DG_MAXN], w[DG_MAXN];
  double D[DG_MAXN * DG_MAXN];   // nodal derivative matrix, D[i*N + k]
  double Dt[DG_MAXN * DG_MAXN];  // flux-differencing matrix 2D - M^{-1}B (Eq. opDsplit), zero diagonal
};

// Kernel ids for profiling
enum { KID_VOLUME = 0, KID_INTERFACE = 1, KID_UPDATE = 2, KID_COUNT = 3 };

// Reference tables of degree p (1..7), computed once on the host.
const RefTables& ref_tables(int p);

// RHS kernels. Each returns the launch error. Ja is FP64 for precision DG_FP64 and FP32 for DG_FP32; the face
// buffer holds the same type.
cudaError_t launch_interface(int nd, int p, int precision, int llf, MeshDims md, const double* u, const void* Ja,
                             void* face, double gamma, int* flag, cudaStream_t s);
cudaError_t launch_volume(int nd, int p, int precision, MeshDims md, const double* u, const void* Ja, const double* invJ,
                          const void* face, double* du, double gamma, int* flag, cudaStream_t s);
// RK stage update (FP64).
cudaError_t launch_rk_update(int scheme, int stage, size_t n, double dt, double* u, double* y, double* acc,
                             const double* du, cudaStream_t s);
// Entropy-rate partial sums into partial[nblocks][2]; then a single block reduces into out[2].
cudaError_t launch_entropy_rate(int nd, int p, MeshDims md, const double* u, const double* du, const double* JW,
                                double gamma, double* partial, int nblocks, double* out, cudaStream_t s);
int entropy_rate_blocks();

}  // namespace dgk

// The context behind the opaque dg_ctx handle.
struct dg_ctx {
  int device;
  int nd, p, N, Nd, nv;
  dgk::MeshDims md;
  long long E, ndofs, state_len;
  double gamma;
  int precision, surface_flux, volume_flux;
  // host copies (FP64)
  double* h_xyz;  // [E][nd][Nd]
  double* h_Ja;   // [E][nd][nd][Nd]
  double* h_J;    // [E][Nd]
  // device data
  double* d_Ja;    // [E][nd][nd][Nd] FP64
  float* d_Ja32;   // FP32 copy (precision == DG_FP32)
  double* d_invJ;  // [E][Nd]
  double* d_JW;    // J * tensor LGL weight, [E][Nd]
  void* d_face;    // face fluxes [nd][E][nv][N^(nd-1)], FP64 or FP32
  double* d_du;    // RHS workspace for dg_step
  double* d_red;   // entropy-rate partials + result
  int* d_flag;     // non-physical-state flag
  cudaStream_t last_stream;
  // profiling
  int prof_on;
  cudaEvent_t* prof_ev;  // pairs
  int prof_cap, prof_n[dgk::KID_COUNT];
  int* prof_kid;
  int prof_used;
  long long launches;
};
