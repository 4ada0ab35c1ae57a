// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/dg.h"

#define DG_MAXN 8  // polydeg <= 7

namespace dgk {

// A launch setting of one kernel that holds per device: the dynamic shared-memory opt-in is a function attribute
// of each device, and the resident CTAs (occupancy x SM count) may differ between devices. per_device runs
// init(&v) once for the current device (under the cache's lock, so concurrent host threads do not race) and
// returns the cached v (> 0) afterwards.
constexpr int kMaxDevices = 64;
struct PerDeviceCache {
  std::mutex m;
  long long value[kMaxDevices] = {};  // 0: not computed yet on that device
};
template <class F>
cudaError_t per_device(PerDeviceCache& c, long long* out, F&& init) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(c.m);
  if (c.value[dev] <= 0) {
    long long v = 0;
    e = init(&v);
    if (e != cudaSuccess) return e;
    c.value[dev] = v;
  }
  *out = c.value[dev];
  return cudaSuccess;
}

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

// Bits of the per-context device flag: a non-physical state (set with atomicOr(flag, 1)); a bounded wait of a
// kernel on its own asynchronous copies that ran out (the kernel then skipped its work).
enum { FLAG_NONPHYSICAL = 1, FLAG_WAIT_TIMEOUT = 4 };

// Kernel ids for profiling (KID_PROJECT: the entropy projection of the Gauss collocation scheme)
enum { KID_VOLUME = 0, KID_INTERFACE = 1, KID_PROJECT = 2, KID_COUNT = 3 };

// Reference tables of degree p (1..7), computed once on the host.
const RefTables& ref_tables(int p);

// What the volume kernel does with the RHS value k at each node: store it as du, or apply the stage update of
// a Runge-Kutta method in place of a separate update kernel.
enum { EPI_STORE = 0, EPI_RK4 = 1, EPI_CK45 = 2 };
struct Epilogue {
  int mode;        // EPI_*
  int stage;       // stage index
  double dt;       // time step
  double a, b;     // CK45: A_s, B_s
  double ca, cy;   // RK4: the stage's weights of k in acc (b_s dt) and in the next stage state (c_{s+1} dt),
                   // computed on the host (no FP64 division per node)
  double* u;       // RK4: solution at the start of the step (updated at the last stage); CK45: the state
  double* y;       // RK4: next stage state; CK45: the K register
  double* acc;     // RK4: accumulated sum of b_s dt k_s
  double* uw;      // where the stage writes the updated state: u, or (dg_step_host's last stage) the device address
                   // of the caller's pinned host buffer, which then receives the new state as it is computed
};

// Runtime variant of the RHS kernels (uniform over a launch): the two-point flux and the Cartesian
// specialisation of affine axis-aligned meshes, whose metric terms are the constants Ja^n = jn[n] e_n and J = 1/invJ.
// Log-mean variants of the volume terms (see log_means_alg / log_means_prelog in dgmath.cuh); 0..2 equal the
// DG_LOGMEAN_* codes of the ABI.
enum { LM_SHARED_RCP = 0, LM_ALG = 1, LM_ALG_POLY = 2, LM_PRELOG = 3 };
static_assert((int)LM_ALG == (int)DG_LOGMEAN_ALG && (int)LM_ALG_POLY == (int)DG_LOGMEAN_ALG_POLY, "log-mean codes");

struct Variant {
  int flux;      // DG_VOL_RANOCHA or DG_VOL_SHIMA (volume and surface)
  int cart;      // 1: constant diagonal metrics from jn/invJ, the metric arrays are not read
  int lm;        // log-mean variant of the volume terms (LM_* in dgmath.cuh; Ranocha's flux only)
  int pipe;      // volume kernel with bulk asynchronous tile copies (where supported): 0 never, 1 on meshes
                 // with enough tiles per resident CTA, 2 always
  int overlap;   // 1: the interface and pipelined volume kernels are launched as programmatic dependents of the
                 // kernel before them in the stream (they start while it drains; dg_opts.launch)
  double jn[3];  // Ja^n_n of a Cartesian mesh
  double invJ;   // 1/J of a Cartesian mesh
  // FP32 flux mode with a reference pressure (dg_opts.p_ref): the momentum equations' pressure terms are evaluated
  // on 2 (p - p_ref), with p - p_ref formed from the FP64 state. sh_eh + sh_el = p_ref / (gamma - 1), the energy of
  // the reference pressure split into two floats; sh_pp = 2 p_ref (a float). All zero: no shift (and in FP64).
  float sh_eh, sh_el, sh_pp;
  // Partitioned context (dg_init_part): the first `ghost` elements of the element range are the ghost layer (one
  // element layer along the last direction, standing for the neighbouring partitions). The volume kernel computes
  // elements [ghost, E) only; the interface kernel computes only the last direction's faces of ghost elements (the
  // partition's lower boundary). 0: an ordinary context.
  int ghost;
  // FP64, curvilinear: per interface node, the lower element's metric vector scaled for the lifted flux
  // (m2 = p(p+1)/8 Ja^n at the face node) and the LLF wave speed's geometric factor gamma |m2|^2 / 2, as
  // [E][ND][4][NL] (computed once at dg_init); nullptr: the interface kernel forms them from the metric terms.
  const double* fgeo;
  // The interface kernel's elements: the faces of elements [if_e0, if_e1) (if_e1 = 0: all; dg_step_host's first
  // interface fluxes, computed per chunk of the state as it arrives from the host). if_e1 may exceed E: the range
  // then wraps around to element 0 (a slab's boundary faces: its last own layer and its ghost layer).
  int if_e0, if_e1;
  // The pipelined volume kernel's tile counter and its count of finished CTAs (both zero between launches; the
  // last CTA of a launch resets them); nullptr: tiles round-robin over the grid.
  int* tiles;
};

// Chunks of element layers in which dg_step_host / dg_rhs_host bring the state to the device (measured on the
// 16^3 FP64 step through dg_step_host, e2e ns/DOF: 1 chunk 0.840, 2 0.827, 3 0.830, 4 0.833, 8 0.850: each
// further chunk adds an interface launch that waits for its copy and so cannot be scheduled ahead).
enum { kUploadChunks = 2 };

// RHS kernels. Each returns the launch error. Ja is FP64 for precision DG_FP64 and FP32 for DG_FP32; the face
// buffer holds the same type.
cudaError_t launch_interface(int nd, int p, int precision, int llf, MeshDims md, const double* u, const void* Ja,
                             void* face, double gamma, int* flag, cudaStream_t s, const Variant* var = nullptr);
// epi == nullptr stores du; otherwise du is unused and the stage update of *epi is applied.
cudaError_t launch_volume(int nd, int p, int precision, MeshDims md, const double* u, const void* Ja, const double* invJ,
                          const void* face, double* du, double gamma, int* flag, cudaStream_t s,
                          const Epilogue* epi = nullptr, const Variant* var = nullptr);
// Entropy-rate partial sums into partial[nblocks][2]; then a single block reduces into out[2].
cudaError_t launch_entropy_rate(int nd, int p, MeshDims md, const double* u, const double* du, const double* JW,
                                double gamma, double* partial, int nblocks, double* out, cudaStream_t s);
int entropy_rate_blocks();
// Conserved totals sum J W q per variable over nelem elements: partials into partial[nblocks][nvar] (nblocks <=
// entropy_rate_blocks()), the totals into out[nvar]. Deterministic order.
cudaError_t launch_totals(int nd, int p, long long nelem, const double* q, const double* JW, double* partial,
                          int nblocks, double* out, cudaStream_t s);
// Halo planes of a partitioned context (see misc.cu): pack copies the owned boundary planes of state u into
// send_lo/send_hi; unpack copies recv_lo/recv_hi into the ghost layer's two planes. layer: elements per layer;
// first_owned, last_owned: the first elements of the first and last owned layers.
// overlap: launched as a programmatic dependent of the kernel before it in s (dg_opts.launch).
cudaError_t launch_halo(int nd, int p, int layer, long long first_owned, long long last_owned, double* u,
                        const double* recv_lo, const double* recv_hi, double* send_lo, double* send_hi, bool pack,
                        bool overlap, cudaStream_t s);
// One CTA whose bounded mbarrier wait runs out and sets FLAG_WAIT_TIMEOUT in *flag (dg_selftest_wait_timeout).
cudaError_t launch_wait_probe(int* flag, cudaStream_t s);
void ck45_coefficients(int stage, double* a, double* b);

// Legendre-Gauss reference tables of degree p (Sec. 6): nodes, weights and derivative matrix in `ref` (ref.Dt is
// unused), and the Lagrange basis at xi = -1 and +1 (the rows of the face restriction R along a line).
struct GaussTables {
  RefTables ref;
  double lm[DG_MAXN], lp[DG_MAXN];
};
const GaussTables& gauss_tables(int p);

// One part of the Gauss collocation RHS (Sec. 6) on a Cartesian mesh: part 0 the entropy projection (u -> gface),
// part 1 the interface fluxes (gface -> fstar), part 2 the volume term, lift and surface term (-> du, or the
// stage update of *epi).
struct GaussLaunch {
  int nd, p, llf, part;
  MeshDims md;
  const double* u;
  double* gface;  // [nd][E][2][nv][N^(nd-1)] entropy-projected face states (side 0: xi_n = -1)
  double* fstar;  // [nd][E][nv][N^(nd-1)] outward flux of each element's upper face, scaled by 8
  double* du;
  double c[3];    // 2/h_n
  double gamma;
  int* flag;
  const Epilogue* epi;
  cudaStream_t s;
};
cudaError_t launch_gauss(const GaussLaunch& L);

}  // namespace dgk

// The context behind the opaque dg_ctx handle.
struct dg_ctx {
  int device;
  int nd, p, N, Nd, nv;
  dgk::MeshDims md;
  long long E, ndofs, state_len;
  double gamma;
  int precision, surface_flux, volume_flux;
  int nodes;          // DG_NODES_LGL or DG_NODES_GAUSS
  double gauss_c[3];  // Gauss collocation: 2/h_n
  dgk::Variant var;  // flux and Cartesian specialisation used by dg_rhs / dg_step
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
  double* d_fadj;  // dg_vjp: face adjoint contributions [nd][E][2][nv][N^(nd-1)] (allocated at the first dg_vjp)
  double* d_gface;  // Gauss collocation: projected face states [nd][E][2][nv][N^(nd-1)]
  double* d_hstage;  // dg_step_host / dg_rhs_host: device copies of the host state (3 state arrays, first call)
  cudaStream_t up_stream;                       // ... and their copy stream and events (first call)
  cudaEvent_t up_ev[1 + dgk::kUploadChunks];
  // partitioned context (dg_init_part): ghost layer of `layer` elements first, then `owned` layers; 0 otherwise
  int part_dir, part_begin, part_end;
  long long layer;       // elements per layer (the ghost layer and each halo plane's element count)
  long long owned_elems;  // elements computed (E minus the ghost layer)
  double* d_fgeo;  // interface geometry (Variant::fgeo; FP64 curvilinear contexts)
  double* d_red;   // entropy-rate partials + result
  int* d_flag;     // non-physical-state flag
  int* d_tiles;    // the pipelined volume kernel's tile counters (Variant::tiles)
  cudaStream_t last_stream;
  // profiling
  int prof_on;
  unsigned prof_mask;    // kernels timed while profiling is on (bit k: kernel id k)
  int prof_every;        // time every prof_every-th launch of each of them
  long long prof_seen[dgk::KID_COUNT];  // launches of each kernel since the enable
  cudaEvent_t* prof_ev;  // pairs
  int prof_cap, prof_n[dgk::KID_COUNT];
  int* prof_kid;
  int prof_used;
  long long launches;
};
