/*
 * dg.h -- C ABI of a GB300-native (sm_103a) library for the right-hand side of entropy-stable,
 * kinetic-energy-preserving flux-differencing LGL-DGSEM for the compressible Euler equations
 * (Ranocha, Schlottke-Lakemper, Chan, Rueda-Ramirez, Winters, Hindenlang, Gassner, arXiv:2112.10517).
 *
 * The semidiscretization (Sec. 2, Eq. fluxdiff-SBP-opDsplit, curvilinear via Eq. curvilinear-rearrange):
 *
 *   du_i = -(1/J_i) [ sum_n sum_k Dt_{i_n k_n} f(u_i, u_k, (Ja^n_i + Ja^n_k)/2)            (volume)
 *                   + sum_n ( [i_n = p] f*_{upper face} - [i_n = 0] f*_{lower face} ) / w_0 ] (surface)
 *
 * with Dt = 2D - M^{-1} B the flux-differencing operator (Eq. opDsplit), f Ranocha's EC/KEP two-point flux
 * (Eq. flux_ranocha) in directional form, f* the same flux plus optional local Lax-Friedrichs dissipation at
 * each interface, Ja the contravariant metric terms and J the Jacobian (Sec. 2.3).
 *
 * CONVENTIONS (all entry points)
 *   Layout.   A state u (and du, and RK scratch) is a C-order array of doubles u[E][nvar][Nd]:
 *             E elements in lexicographic order (e = e1 + n1*(e2 + n2*e3), e1 fastest), nvar = ndims+2
 *             conserved variables (rho, rho v_1..rho v_d, rho e), Nd = (p+1)^ndims LGL nodes per element
 *             with node index i = i1 + N*i2 + N*N*i3 (i1 along xi_1 fastest, N = p+1).
 *   Memory.   Pointers named *_host are host memory; all other state pointers are DEVICE memory on the
 *             device that was current at dg_init, 8-byte aligned. The caller owns u, du and scratch and
 *             keeps them valid until the work queued on `stream` has completed. The library owns its
 *             context (metrics, tables, workspaces) and frees it in dg_free.
 *   Streams.  Work is queued on `stream` (NULL: the legacy default stream). Entry points do not
 *             synchronize the host except where stated (dg_entropy_rate, dg_check_status, the getters).
 *             Calls that share one context must not run concurrently on different streams (they share
 *             the context's workspaces).
 *   Errors.   Every entry point returns a dg_status and never throws or aborts. Argument errors are
 *             detected before any work is queued. Non-physical states (rho <= 0, p <= 0 or NaN) met by a
 *             kernel set an asynchronous flag that dg_check_status reports as DG_ERR_NONPHYSICAL.
 *   Boundary. Every direction is periodic (the paper treats volume terms and interior interfaces only,
 *             Sec. 2); meshes are conforming, structured boxes of hexahedra (3D) or quadrilaterals (2D).
 *   Degree.   1 <= polydeg <= 7.
 */
#ifndef DG_H
#define DG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx;             /* opaque; created by dg_init, destroyed by dg_free */
typedef struct CUstream_st* dg_stream_t;  /* identical to cudaStream_t */

typedef enum dg_status {
  DG_OK = 0,
  DG_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, unsupported combination) */
  DG_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  DG_ERR_OOM = 3,          /* device allocation failed */
  DG_ERR_UNSUPPORTED = 4,  /* valid request the library does not implement (e.g. polydeg > 7) */
  DG_ERR_NONPHYSICAL = 5,  /* a kernel met rho <= 0, p <= 0 or NaN since the last dg_check_status */
  DG_ERR_TIMEOUT = 6       /* a bounded host wait gave up */
} dg_status;

enum { DG_MAP_AFFINE = 0, DG_MAP_SINE = 1, DG_MAP_NODES = 2 };
enum { DG_SURF_EC = 0, DG_SURF_EC_LLF = 1 };
enum { DG_FP64 = 0, DG_FP32 = 1 };
enum { DG_VOL_RANOCHA = 0, DG_VOL_SHIMA = 1 };
enum { DG_RK4_CLASSIC = 0, DG_LSRK45_CK = 1 };

/* Periodic box [lo, hi] with nelem[m] elements per direction (nelem[2], lo[2], hi[2] ignored in 2D).
   mapping: DG_MAP_AFFINE  x = xi;
            DG_MAP_SINE    x_m = xi_m + map_amp (L_m/2pi) prod_k sin(2pi (xi_k - c_k)/L_k), L = hi - lo,
                           c = (lo + hi)/2; on [-pi, pi]^3 this is x_m = xi_m + a sin(xi_1) sin(xi_2) sin(xi_3);
            DG_MAP_NODES   node_xyz (host, [E][ndims][Nd]) gives the physical node coordinates. */
typedef struct dg_mesh {
  int ndims;
  int nelem[3];
  double lo[3];
  double hi[3];
  int mapping;
  double map_amp;
  const double* node_xyz_host;
} dg_mesh;

/* Optional override of the metric terms (host memory, copied at dg_init):
   Ja_host [E][ndims][ndims][Nd], Ja[e][n][j][i] = (Ja^n)_j at node i (reference direction n, Cartesian
   component j); J_host [E][Nd]. When NULL, dg_init computes them from the node coordinates: 2D with the
   cross-product form and 3D with the conservative curl form (Sec. 2.3, free-stream preservation). */
typedef struct dg_metrics {
  const double* Ja_host;
  const double* J_host;
} dg_metrics;

/* gamma: ratio of specific heats (> 1). volume_flux: the two-point flux of the volume term and of the interfaces
   (as in the paper's runs, Sec. 4.1): DG_VOL_RANOCHA (Eq. flux_ranocha, entropy conservative) or DG_VOL_SHIMA
   (Eq. flux_shima_etal, kinetic energy and pressure equilibrium preserving, not entropy conservative; dg_vjp and
   dg_batch_* support DG_VOL_RANOCHA only).
   surface_flux: DG_SURF_EC (the two-point flux alone) or DG_SURF_EC_LLF (plus local Lax-Friedrichs dissipation).
   precision: DG_FP64, or DG_FP32 (two-point fluxes and line sums in FP32; metric terms computed in
   FP64 and rounded once; state, du, RK accumulation and the entropy diagnostic in FP64).
   precompute_logs, logmean: how the volume terms of Ranocha's flux evaluate the logarithmic mean of density and
   the inverse logarithmic mean of rho/p (Sec. 3.1, Algorithms 2 and 3; Sec. 7.2), for ablation studies. All
   variants compute the same means up to rounding; the default (both 0) is the fastest on this hardware.
     logmean = DG_LOGMEAN_SHARED_RCP  no division: one reciprocal serves both means' u and the inverse
                                      mean's series; the mean's series in the polynomial 1/log form; in FP64
                                      the series continued to u^7 for 1e-4 <= u < 1e-2 instead of logarithms;
               DG_LOGMEAN_ALG         Algorithms 2 and 3 as stated (divisions, log of the ratio per pair);
               DG_LOGMEAN_ALG_POLY    the same with the polynomial 1/log form of the mean's series branch.
     precompute_logs = 1              logarithms of density and rho/p once per node instead of once per pair
                                      (with DG_LOGMEAN_SHARED_RCP only; taken relative to each element's first
                                      node, which leaves the differences, i.e. the logs of the ratios, unchanged).
   Non-default values need DG_VOL_RANOCHA (else DG_ERR_UNSUPPORTED); the DG_LOGMEAN_ALG* variants run the
   general metric path on an affine mesh and are available in dg_rhs only (dg_step returns DG_ERR_UNSUPPORTED).
   The interface fluxes always use the default. dg_vjp accepts the default only; dg_batch_* the default or
   precompute_logs (the same for all contexts of a batch).
   nodes: DG_NODES_LGL, the flux-differencing LGL-DGSEM above, or DG_NODES_GAUSS, the Legendre-Gauss collocation
   scheme with entropy projection (Sec. 6, Eq. fluxdiff-GSBP-opDsplit with the hybridized volume terms of Eq.
   hybridized_gauss_formulation): the state lives at the tensor-product Gauss nodes (dg_get_node_coords), face
   states are u(R w(u)) of each element, interface fluxes are computed once per face node. DG_NODES_GAUSS needs
   DG_MAP_AFFINE without overrides, DG_VOL_RANOCHA, DG_FP64 and the default log mean (else DG_ERR_UNSUPPORTED);
   dg_vjp and dg_batch_* do not support it. Its face states need the entropy variables interpolated to the faces
   to stay admissible (rho/p > 0); otherwise the non-physical flag is raised.
   staging: how the volume kernel of dg_rhs / dg_step brings an element tile's data into shared memory.
     DG_STAGING_PIPELINED  the default log mean: persistent CTAs that copy each tile's data (stage input, metric
                           terms, 1/J, Runge-Kutta operands, interface fluxes) with asynchronous copies, each group
                           for the next tile as soon as the current tile has read it, so that the copies overlap
                           computation (bulk copies for an even number of nodes per line, which then needs
                           16-byte-aligned state arrays; per-thread copies otherwise); else as DG_STAGING_DIRECT.
     DG_STAGING_AUTO       as DG_STAGING_PIPELINED on meshes with at least 2 tiles per resident CTA (the first
                           tile's copies are not overlapped), except DG_FP32 at polydeg 2 (measured slower); else
                           as DG_STAGING_DIRECT.
     DG_STAGING_DIRECT     one CTA per tile, loads issued by its threads.
   All evaluate the same terms; the pipelined kernel starts each line's sums from the lifted interface fluxes and
   the direct one adds them after the sums, so the two agree to rounding (the parity bounds), and DG_STAGING_AUTO
   gives bit for bit the result of the kernel it selects. The order in which the pipelined kernel's CTAs take the
   tiles (round-robin, or on some DG_FP64 meshes from a counter in the context's workspace, with smaller tiles
   last) changes no result: each element's arithmetic is the same in any tile. A pipelined kernel whose wait for its own
   copies runs out (bounded; it cannot under normal operation) skips the rest of its tiles and raises the flag that
   dg_check_status reports as DG_ERR_TIMEOUT.
   launch: how dg_rhs / dg_step queue the interface kernel and the pipelined volume kernel.
     DG_LAUNCH_OVERLAP     (default) each as a programmatic dependent of the kernel before it in the stream: it is
                           scheduled ahead and its CTAs start as those of that kernel exit, set up, and copy the
                           metric terms of their first tile (written only by dg_init); every read of the state, the
                           interface fluxes and the Runge-Kutta operands, and every write, waits until the kernels
                           before it have completed and their writes are visible. Work queued on the stream by other
                           code is ordered as usual.
     DG_LAUNCH_SERIAL      ordinary launches: each kernel starts after the one before it has completed.
   Both compute the same values.
   p_ref: a reference pressure for the FP32 flux mode (>= 0, finite; 0: none; ignored in FP64). The momentum
   equations' pressure terms, {{p}} n of the two-point fluxes in the volume and at the interfaces, are then
   evaluated on p - p_ref, formed from the FP64 state's energy minus p_ref/(gamma-1) on the integer and FP32
   pipes, and the LLF dissipation's energy jump on the same relative energies. A constant pressure contributes
   nothing to the momentum RHS (its volume and lifted surface terms cancel by the discrete metric identities of
   Sec. 2.3, the property behind free-stream preservation), so the shift leaves the scheme's values unchanged up to
   rounding and removes the cancellation of large pressure terms that FP32 rounding would otherwise leave in the
   momentum RHS of a low-Mach flow (choose p_ref near the flow's mean pressure, e.g. 1/(gamma M^2) for a
   nondimensional flow at Mach M). p_ref is rounded to FP32. Needs the default log mean (DG_ERR_UNSUPPORTED
   otherwise); dg_batch_* reject contexts with p_ref != 0 in FP32 mode (DG_ERR_UNSUPPORTED). */
enum { DG_LOGMEAN_SHARED_RCP = 0, DG_LOGMEAN_ALG = 1, DG_LOGMEAN_ALG_POLY = 2 };
enum { DG_NODES_LGL = 0, DG_NODES_GAUSS = 1 };
enum { DG_STAGING_AUTO = 0, DG_STAGING_DIRECT = 1, DG_STAGING_PIPELINED = 2 };
enum { DG_LAUNCH_OVERLAP = 0, DG_LAUNCH_SERIAL = 1 };
typedef struct dg_opts {
  double gamma;
  int volume_flux;
  int surface_flux;
  int precision;
  int precompute_logs; /* 0 or 1 */
  int logmean;         /* DG_LOGMEAN_* */
  int nodes;           /* DG_NODES_* */
  int staging;         /* DG_STAGING_* */
  int launch;          /* DG_LAUNCH_* */
  double p_ref;        /* FP32 flux mode: reference pressure of the momentum pressure terms (0: none) */
} dg_opts;

/* Sizes of a context. */
typedef struct dg_info {
  int ndims, polydeg, nvar, nodes_per_elem;
  long long nelem_total;   /* E */
  long long ndofs;         /* E * Nd: the DOF count of the performance index (Sec. 4.1, Def. PID) */
  long long state_len;     /* E * nvar * Nd doubles in u, du */
  int precision, surface_flux;
} dg_info;

/* Build a context: LGL tables (Sec. 2), node coordinates, metric terms and Jacobian (Sec. 2.3) in FP64
   on the host, uploaded to the current device. Allocates device memory (about 100 bytes per DOF).
   With DG_MAP_AFFINE and no metric override the kernels use the Cartesian specialisation: the metric terms of an
   axis-aligned box element are constant and diagonal, so dg_rhs and dg_step read no metric arrays.
   Returns DG_ERR_ARG for a bad mesh/options, DG_ERR_UNSUPPORTED for polydeg outside 1..7, DG_ERR_OOM. */
dg_status dg_init(dg_ctx** out, const dg_mesh* mesh, int polydeg, const dg_metrics* metrics, const dg_opts* opts);

/* du = RHS(u) (Eq. fluxdiff-SBP-opDsplit). u, du: device [E][nvar][Nd], distinct, not overlapping.
   t is accepted for interface completeness and unused (autonomous, periodic problem). u is not modified.
   Queues 2 kernels (interface flux, then volume + surface lift + Jacobian) on `stream`, by default as programmatic
   dependent launches (dg_opts.launch). */
dg_status dg_rhs(dg_ctx* ctx, const double* u, double* du, double t, dg_stream_t stream);

/* One explicit time step u <- u + dt * (...) of the low-storage Runge-Kutta method `scheme` (Sec. 4.1):
   DG_RK4_CLASSIC  classical four-stage RK4 in low-storage form; scratch = 2 state arrays (2*state_len);
   DG_LSRK45_CK    five-stage fourth-order 2N method of Carpenter and Kennedy; scratch = 1 state array.
   u and scratch are device memory, not overlapping; scratch contents on entry are ignored. Each stage queues
   2 kernels: the interface fluxes, then the volume term whose epilogue applies the stage update in FP64 (launched
   as in dg_rhs). */
dg_status dg_step(dg_ctx* ctx, double* u, double* scratch, double t, double dt, int scheme, dg_stream_t stream);

/* The same with the state in host memory: queue on `stream` the host->device copy of u_host, dg_step (or dg_rhs)
   on device copies owned by the context, and the result into host memory (the new state into u_host, or du into
   du_host). When the result buffer is page-locked (cudaHostAlloc / cudaHostRegister, torch pin_memory), the last
   kernel writes the result straight into it through its device address, over the CPU-GPU link while it computes,
   and no device->host copy follows; otherwise a device->host copy does. Pinned host memory also makes the
   host->device copy asynchronous. LGL meshes with at least 4 element layers along the last direction get the
   state in 2 chunks of layers on a copy stream of the context (after the work queued on `stream` before the call),
   and the first interface fluxes per chunk on `stream` as soon as the chunk (and the next layer) is there, so the
   second chunk's copy overlaps the first chunk's fluxes; `stream` then waits for the copies. The caller
   synchronizes the stream before reading the result. The first call allocates three state arrays of device memory
   and the copy stream held by the context until dg_free. Errors as dg_step / dg_rhs. */
dg_status dg_step_host(dg_ctx* ctx, double* u_host, double t, double dt, int scheme, dg_stream_t stream);
dg_status dg_rhs_host(dg_ctx* ctx, const double* u_host, double* du_host, double t, dg_stream_t stream);

/* Entropy rate dS/dt = sum_e sum_i J_i W_i w(u_i) . du_i (Sec. 2: EC/ED semidiscretizations; W the tensor
   LGL weights, w the entropy variables of U = -rho s/(gamma-1)). FP64, deterministic order. Writes the value
   to *out_host and, when abs_out_host is not NULL, the magnitude sum_e sum_i sum_c |J_i W_i w_c(u_i) du_c,i| to
   *abs_out_host (the scale for judging dS/dt = 0). Synchronizes `stream`. */
dg_status dg_entropy_rate(dg_ctx* ctx, const double* u, const double* du, double* out_host, double* abs_out_host,
                          dg_stream_t stream);

/* Vector-Jacobian product (adjoint) of dg_rhs: ubar = (d RHS/du (u))^T gbar, FP64. u, gbar, ubar: device arrays of
   the state layout; ubar must not overlap u or gbar. The derivative of every step of the RHS is hand-written:
   the logarithmic means of Algorithms 2-3 (exact derivatives of the means in both branches), Ranocha's flux
   (Eq. flux_ranocha), the LLF dissipation (subgradient at its max/abs switches: the branch the forward flux
   takes, sign(0) = +1), the primitive variables, the flux-differencing sums (Eq. fluxdiff-SBP-opDsplit), the
   lift and the Jacobian scaling. Two kernels; the first call allocates the context's face-adjoint workspace
   (8 nvar (p+1)^(d-1) d bytes per element). FP64 contexts with polydeg <= 5; DG_ERR_UNSUPPORTED otherwise. */
dg_status dg_vjp(dg_ctx* ctx, const double* u, const double* gbar, double* ubar, dg_stream_t stream);

/* Reads and clears the asynchronous flag of non-physical states and of device-side waits that ran out. Waits
   (bounded, 60 s) for the work queued on the stream of the last call; returns DG_OK, DG_ERR_NONPHYSICAL or
   DG_ERR_TIMEOUT (the host wait gave up, or a pipelined kernel's bounded wait on its own copies ran out). */
dg_status dg_check_status(dg_ctx* ctx);

/* Failure-path self-test of the device-side bounded waits: queues on `stream` one CTA that waits, with the same
   bounded mbarrier wait the pipelined volume kernel uses, on an mbarrier that nothing completes. The wait gives up
   after about half a second and sets the context's timeout flag, so that the next dg_check_status returns
   DG_ERR_TIMEOUT (and clears it; the context stays usable). Nothing faults, traps or hangs. */
dg_status dg_selftest_wait_timeout(dg_ctx* ctx, dg_stream_t stream);

/* Getters (host copies; synchronize the device). */
dg_status dg_get_info(const dg_ctx* ctx, dg_info* info);
dg_status dg_get_node_coords(const dg_ctx* ctx, double* xyz_host /* [E][ndims][Nd] */);
dg_status dg_get_metrics(const dg_ctx* ctx, double* Ja_host /* [E][d][d][Nd] */, double* J_host /* [E][Nd] */);

/* Kernel timing with CUDA events recorded on the launching stream around every launch of kernel `which`
   (0 = volume term with surface lift and Jacobian, which in dg_step also applies the RK stage update;
   1 = interface flux; 2 = entropy projection of DG_NODES_GAUSS) while enabled. dg_profile_enable times every
   kernel (on != 0) or none; dg_profile_enable_kernels times the kernels of `mask` (bit k: kernel k; 0 = off), so
   that a timed region carries events around the kernel of interest only; dg_profile_enable_sampled times every
   `every`-th launch (>= 1) of each of them (with `every` coprime to the launches per step, every Runge-Kutta stage
   is sampled). dg_profile_read returns the summed milliseconds and the number of timed launches since the last
   enable, and synchronizes. dg_launch_count counts every kernel the context has launched since dg_init. */
dg_status dg_profile_enable(dg_ctx* ctx, int on);
dg_status dg_profile_enable_kernels(dg_ctx* ctx, unsigned mask);
dg_status dg_profile_enable_sampled(dg_ctx* ctx, unsigned mask, int every);
dg_status dg_profile_read(dg_ctx* ctx, int which, double* total_ms, long long* launches);
long long dg_launch_count(const dg_ctx* ctx);

void dg_free(dg_ctx* ctx);
const char* dg_status_string(dg_status s);

/* ---------------------------------------------------------------------------------------------------------
 * Partitioned meshes: one periodic mesh split into slabs, one context per slab (one GPU or one process each).
 *
 * The volume terms are element-local and the interface fluxes couple face neighbours only (Sec. 2.4; the
 * surface flux is evaluated once per interface node from the two adjacent elements' face states), so a slab needs,
 * besides its own elements, one plane of face states from each neighbouring slab per RHS: N^(d-1) nvar values per
 * element face on the cut. The cut runs along the LAST direction (xi_3 in 3D, xi_2 in 2D), between element layers.
 *
 * dg_init_part creates the context of the element layers [begin, end) of the GLOBAL mesh `mesh` along the last
 * direction (0 <= begin < end <= nelem[last]); the other directions stay periodic within the slab, the last is
 * periodic across slabs (the slab of layer 0 is the upper neighbour of the slab ending at nelem[last]). Mappings
 * DG_MAP_AFFINE and DG_MAP_SINE only (the node coordinates and metric terms of every element are those the global
 * context computes, bit for bit); no metric override; DG_NODES_LGL. Its state arrays (u, du, RK scratch) hold
 * E = layer * (1 + end - begin) elements, layer = nelem[0] (2D) or nelem[0] nelem[1] (3D): first a GHOST layer of
 * `layer` elements, then the slab's own layers in the global element order. Only two planes of the ghost layer are
 * read: its node plane i_last = p, which must hold the lower neighbour slab's last layer's plane i_last = p, and its
 * plane i_last = 0, which must hold the upper neighbour slab's first layer's plane i_last = 0. The kernels compute
 * the slab's own elements; the ghost layer of du and of the RK arrays is never written.
 *
 * Per RHS (and per Runge-Kutta stage, on that stage's input state):
 *   1. dg_part_pack(ctx, state, send_lo, send_hi): send_lo <- plane i_last = 0 of the first own layer, send_hi <-
 *      plane i_last = p of the last own layer (device buffers of dg_part_info.halo_len doubles each, layout
 *      [layer][nvar][N^(d-1)], layer elements in element order, face nodes in node order);
 *   2. the caller moves send_lo to the LOWER neighbour's recv_hi and send_hi to the UPPER neighbour's recv_lo (any
 *      transport: NCCL send/recv, peer copies, or, for a slab that is its own neighbour, local copies);
 *   3. dg_part_unpack(ctx, state, recv_lo, recv_hi) writes them into the ghost layer of `state`;
 *   4. dg_rhs(ctx, state, du) or dg_step_stage(ctx, u, scratch, ..., stage).
 * A stage can also overlap the transport of step 2 (Sec. 2.4: only the faces at the slab's ends read the ghost
 * layer): dg_stage_interface(..., DG_REGION_INTERIOR) between steps 1 and 3, then after step 3
 * dg_stage_interface(..., DG_REGION_BOUNDARY) and dg_stage_volume; the three together are dg_step_stage.
 * Each call queues on `stream` and synchronizes nothing. The result equals, bit for bit, the same elements of the
 * global context's result when both use the same volume-kernel staging. dg_step, dg_step_host, dg_rhs_host,
 * dg_vjp and dg_batch_* return DG_ERR_UNSUPPORTED for a partitioned context (they cannot exchange halos between
 * stages); dg_entropy_rate and dg_conserved_totals sum the slab's own elements (sum them over the slabs: one
 * all-reduce of nvar + 2 scalars). dg_get_node_coords / dg_get_metrics return all E elements, the ghost layer
 * included; dg_get_info reports nelem_total = E and state_len for the arrays, ndofs for the slab's own elements.
 * --------------------------------------------------------------------------------------------------------- */
typedef struct dg_part {
  int begin;  /* first element layer along the last direction owned by this slab */
  int end;    /* one past the last */
} dg_part;

typedef struct dg_part_info {
  long long layer;       /* elements per element layer (ghost layer and halo planes) */
  long long own_elems;   /* elements the slab computes: layer * (end - begin) */
  long long ghost_elems; /* elements before them in the state arrays: layer */
  long long halo_len;    /* doubles in each of send_lo, send_hi, recv_lo, recv_hi: layer * nvar * N^(d-1) */
  int begin, end;
} dg_part_info;

dg_status dg_init_part(dg_ctx** out, const dg_mesh* mesh, int polydeg, const dg_opts* opts, const dg_part* part);
dg_status dg_part_get_info(const dg_ctx* ctx, dg_part_info* info);
/* DG_ERR_ARG for an ordinary context or null pointers; buffers are device memory, distinct from the state. */
dg_status dg_part_pack(dg_ctx* ctx, const double* state, double* send_lo, double* send_hi, dg_stream_t stream);
dg_status dg_part_unpack(dg_ctx* ctx, double* state, const double* recv_lo, const double* recv_hi, dg_stream_t stream);

/* One stage of dg_step's scheme (stage 0 .. 3 for DG_RK4_CLASSIC, 0 .. 4 for DG_LSRK45_CK; arguments as dg_step):
   running stages 0, 1, ... in order on the same u and scratch is dg_step. Stage `stage` reads the state that
   dg_stage_input names: 0 = u, 1 = scratch (its first state array). Partitioned contexts exchange halos on that
   state before each stage. Ordinary contexts accept it too. */
dg_status dg_step_stage(dg_ctx* ctx, double* u, double* scratch, double t, double dt, int scheme, int stage,
                        dg_stream_t stream);
int dg_stage_input(int scheme, int stage); /* 0: u, 1: scratch, -1: invalid scheme or stage */

/* dg_step_stage in parts, for a partitioned context that overlaps its halo transport with computation (Sec. 2.4):
   dg_stage_interface computes the interface fluxes of the stage's input state (dg_stage_input) for the faces of a
   region of the slab: DG_REGION_INTERIOR, the faces of the own layers except the last, which read no ghost-layer
   data (queue it before the ghost layer is unpacked); DG_REGION_BOUNDARY, the rest (the last own layer's faces and
   the faces of the ghost layer, whose two planes must then hold the neighbours' data). dg_stage_volume then runs
   the stage's volume kernel and update. Interior, boundary, volume in this order on one stream equal
   dg_step_stage bit for bit. Arguments as dg_step_stage; DG_ERR_ARG for an ordinary context or another region. */
enum { DG_REGION_INTERIOR = 0, DG_REGION_BOUNDARY = 1 };
dg_status dg_stage_interface(dg_ctx* ctx, double* u, double* scratch, int scheme, int stage, int region,
                             dg_stream_t stream);
dg_status dg_stage_volume(dg_ctx* ctx, double* u, double* scratch, double t, double dt, int scheme, int stage,
                          dg_stream_t stream);

/* Conserved totals sum_e sum_i J_i W_i q_i per variable (Sec. 2: discrete conservation; q a device state array, W
   the tensor LGL weights), FP64 in a fixed order, into out_host[nvar]; the slab's own elements for a partitioned
   context. Synchronizes `stream`. */
dg_status dg_conserved_totals(dg_ctx* ctx, const double* q, double* out_host, dg_stream_t stream);

/* ---------------------------------------------------------------------------------------------------------
 * Batched RHS: many independent meshes of uneven size and degree in one persistent launch.
 * The per-element work is that of dg_rhs (Eq. fluxdiff-SBP-opDsplit); only the scheduling differs.
 *
 * dg_batch_create binds n contexts and their state buffers: u[i], du[i] are device arrays of context i's
 * layout (distinct, not overlapping; the caller keeps them valid for the plan's lifetime and may change their
 * contents between calls). All contexts must be 3D, on the current device, with one precision, surface flux and
 * gamma, and polydeg <= 5 (DG_ERR_UNSUPPORTED otherwise). Uses the contexts' metric terms, interface-flux
 * workspaces and non-physical flags (dg_check_status of each context reports its instance). Allocates small
 * device tables (work lists) and synchronizes.
 * dg_batch_rhs computes du[i] = RHS_i(u[i]) for every instance: it queues one memset and the interface fluxes of
 * all instances on `stream`, then per degree one persistent volume kernel (whose CTAs take that degree's element
 * tiles from a shared counter) on the plan's own streams, forked from `stream` by an event and joined back into it
 * before the call returns; work queued later on `stream` follows all of it. It allocates nothing and does not synchronize, so a sequence of calls
 * can be captured in a CUDA graph after a first call outside the capture. Plans sharing a context must not run
 * concurrently (they share its workspace).
 * dg_batch_autotune times every tile shape (threads per CTA 128/192/256, which sets the elements per tile of
 * each degree) and persistent grid size (1..occupancy CTAs per SM) on the bound buffers, keeps the fastest, and
 * when cache_path is not NULL reads the choice from, or appends it to, that text file (one line per
 * device + batch signature). Synchronizes. dg_batch_set_tuning sets a choice directly (ctas_per_sm 0 = occupancy).
 * --------------------------------------------------------------------------------------------------------- */
typedef struct dg_batch dg_batch;
dg_status dg_batch_create(dg_batch** out, dg_ctx* const* ctxs, int n, const double* const* u, double* const* du);
dg_status dg_batch_rhs(dg_batch* batch, dg_stream_t stream);
dg_status dg_batch_autotune(dg_batch* batch, const char* cache_path, dg_stream_t stream, int* threads_out,
                            int* ctas_per_sm_out);
dg_status dg_batch_set_tuning(dg_batch* batch, int threads, int ctas_per_sm);
void dg_batch_free(dg_batch* batch);

/* ---------------------------------------------------------------------------------------------------------
 * dg_rhs_noalloc -- the paper has no counterpart to this entry point; it serves callers of this library.
 *
 * Computes the same du = RHS(u) as dg_rhs, without a context and without allocating any memory. It is for
 * callers that cannot call cudaMalloc: an application whose memory manager owns all device memory (every
 * allocation has to go through its pool and its accounting), or code on a latency-critical path where an
 * allocation or a free could synchronize the device. Such a caller keeps u, du and the metric terms in its own
 * device memory; the interface fluxes, which dg_rhs keeps in a per-context workspace, go to one fixed device
 * array of DG_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads the library holds until the
 * process exits. The call uses no cudaMalloc, cudaFree or allocating library routine.
 *
 *   ndims, nelem[ndims], polydeg, precision, surface_flux, gamma: as in dg_mesh / dg_opts (periodic box,
 *        structured, lexicographic element order).
 *   u, du  device [E][nvar][Nd] doubles, distinct and not overlapping (layout as for dg_rhs).
 *   Ja     device metric terms [E][ndims][ndims][Nd], Ja[e][n][j][i] = (Ja^n)_j at node i: doubles for DG_FP64,
 *          floats for DG_FP32 (dg_get_metrics returns them in FP64).
 *   invJ   device [E][Nd] doubles, 1/J at every node.
 *   flag   optional device int: set to 0 at the start of the call, then non-zero if a kernel meets rho <= 0,
 *          p <= 0 or NaN. NULL uses a slot in the library's array.
 * Returns DG_ERR_UNSUPPORTED when the interface fluxes of the mesh do not fit the array (ndims * E * nvar *
 * (p+1)^(ndims-1) values of the flux precision, plus 256 bytes; at 64 MiB this admits 32^3 elements at p = 3 in
 * FP64) or polydeg is outside 1..7, DG_ERR_ARG for other invalid arguments, DG_ERR_CUDA if a launch fails.
 * The first call made on a device looks up the array's device address for that device (cudaGetSymbolAddress);
 * make that first call before any stream capture. Every call on a device shares the one array, and it keeps
 * the last call's contents: calls that may overlap on the GPU (different streams, or threads without ordering)
 * race on it and must be serialized by the caller. Work is queued on `stream`; the host is not synchronized.
 * --------------------------------------------------------------------------------------------------------- */
#define DG_NOALLOC_SCRATCH_BYTES (64u << 20)
dg_status dg_rhs_noalloc(int ndims, const int* nelem, int polydeg, int precision, int surface_flux, double gamma,
                         const double* u, const void* Ja, const double* invJ, double* du, int* flag,
                         dg_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* DG_H */
