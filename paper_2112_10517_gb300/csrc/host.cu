// Host side of the library: reference element, mesh geometry, metric terms, context management and the
// C-ABI entry points. Arithmetic here is FP64 (long double for the LGL tables) and runs once per dg_init.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <new>
#include <vector>

#include "dg_internal.h"

namespace {

// ---------------------------------------------------------------------------------------------------
// Reference element (Sec. 2, LGL example): LGL nodes are +-1 and the roots of P_p'. They are the roots of
// q = P_{p+1} - P_{p-1} = (2p+1)(x^2-1)P_p'/(p(p+1)), and q' = (2p+1) P_p, which gives a Newton step that
// needs only Legendre values. Weights 2/(p(p+1) P_p(x)^2). The derivative matrix uses the closed form for
// LGL nodes: D_ik = P_p(x_i) / (P_p(x_k) (x_i - x_k)) off the diagonal, D_00 = -p(p+1)/4, D_pp = p(p+1)/4.
// ---------------------------------------------------------------------------------------------------

void legendre_upto(long double x, int n, long double* P /* P[0..n] */) {
  P[0] = 1.0L;
  if (n >= 1) P[1] = x;
  for (int k = 2; k <= n; ++k) P[k] = ((2 * k - 1) * x * P[k - 1] - (k - 1) * P[k - 2]) / k;
}

void build_ref_tables(int p, dgk::RefTables* t) {
  const int N = p + 1;
  long double X[DG_MAXN], Pp[DG_MAXN];
  long double P[DG_MAXN + 2];
  for (int i = 0; i < N; ++i) {
    long double xi;
    if (i == 0) {
      xi = -1.0L;
    } else if (i == p) {
      xi = 1.0L;
    } else {
      xi = -cosl(3.141592653589793238462643383279502884L * (long double)i / (long double)p);
      for (int it = 0; it < 100; ++it) {
        legendre_upto(xi, p + 1, P);
        const long double step = (P[p + 1] - P[p - 1]) / ((2.0L * p + 1.0L) * P[p]);
        xi -= step;
        if (fabsl(step) <= 1e-19L) break;
      }
    }
    X[i] = xi;
    legendre_upto(xi, p, P);
    Pp[i] = P[p];
  }
  memset(t, 0, sizeof(*t));
  for (int i = 0; i < N; ++i) {
    t->x[i] = (double)X[i];
    t->w[i] = (double)(2.0L / ((long double)p * (p + 1) * Pp[i] * Pp[i]));
  }
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < N; ++k) {
      long double d;
      if (i != k)
        d = Pp[i] / (Pp[k] * (X[i] - X[k]));
      else if (i == 0)
        d = -(long double)p * (p + 1) / 4.0L;
      else if (i == p)
        d = (long double)p * (p + 1) / 4.0L;
      else
        d = 0.0L;
      t->D[i * N + k] = (double)d;
      // flux-differencing operator Dt = 2D - M^{-1} B (Eq. opDsplit): M^{-1}B = diag(-1/w_0, 0, .., 1/w_p);
      // its diagonal vanishes (Sec. 2.2: M Dt is skew-symmetric), so it is set to exactly zero.
      t->Dt[i * N + k] = (i == k) ? 0.0 : (double)(2.0L * d);
    }
}


int ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

// ---------------------------------------------------------------------------------------------------
// Geometry (Sec. 2.3)
// ---------------------------------------------------------------------------------------------------

// Node coordinates of `nlayers` element layers along the last direction, local layer l being the mesh's layer
// (layer0 + l) mod nelem[last] (periodic): the whole mesh for layer0 = 0, nlayers = nelem[last]; a partitioned
// context's ghost layer and own layers otherwise. Each element's nodes follow from its global element indices, so a
// slab's geometry is bit for bit that of the same elements of the whole mesh.
void node_coords(const dg_mesh* m, int p, const dgk::RefTables& t, double* xyz, int layer0, int nlayers) {
  const int nd = m->ndims, N = p + 1, Nd = ipow(N, nd);
  const int last = nd - 1, nlast = m->nelem[last];
  const int n1 = m->nelem[0], n2 = nd == 3 ? m->nelem[1] : nlayers, n3 = nd == 3 ? nlayers : 1;
  const double twopi = 6.283185307179586476925286766559;
  for (int e = 0; e < n1 * n2 * n3; ++e) {
    int ei[3] = {e % n1, (e / n1) % n2, e / (n1 * n2)};
    ei[last] = ((layer0 + ei[last]) % nlast + nlast) % nlast;
    for (int i = 0; i < Nd; ++i) {
      const int ii[3] = {i % N, (i / N) % N, i / (N * N)};
      double xi[3];
      for (int d = 0; d < nd; ++d) {
        const double h = (m->hi[d] - m->lo[d]) / m->nelem[d];
        xi[d] = m->lo[d] + h * (ei[d] + 0.5 * (t.x[ii[d]] + 1.0));
      }
      double s = 1.0;
      if (m->mapping == DG_MAP_SINE)
        for (int d = 0; d < nd; ++d) {
          const double L = m->hi[d] - m->lo[d];
          s *= sin(twopi * (xi[d] - 0.5 * (m->lo[d] + m->hi[d])) / L);
        }
      for (int d = 0; d < nd; ++d) {
        const double L = m->hi[d] - m->lo[d];
        const double pert = m->mapping == DG_MAP_SINE ? m->map_amp * (L / twopi) * s : 0.0;
        xyz[((size_t)e * nd + d) * Nd + i] = xi[d] + pert;
      }
    }
  }
}

// out = (D along reference direction `dir`) g, for one element's nodal field (Nd values)
void deriv(int nd, int N, const double* D, int dir, const double* g, double* out) {
  const int Nd = ipow(N, nd), st = ipow(N, dir);
  for (int i = 0; i < Nd; ++i) {
    const int a = (i / st) % N;
    const double* line = g + (i - a * st);
    double acc = 0.0;
    for (int k = 0; k < N; ++k) acc += D[a * N + k] * line[k * st];
    out[i] = acc;
  }
}

// Metric terms: 2D cross-product form (Sec. 2.3); 3D conservative curl form (Ja^n)_j =
// -[curl_xi I^N(X_l grad_xi X_m)]_n, (j, m, l) cyclic, which satisfies the discrete metric identities
// sum_n D_n (Ja^n)_j = 0 and so preserves free streams (Sec. 2.3). J = det(dx/dxi).
bool compute_metrics(int nd, int p, long long E, const double* xyz, const dgk::RefTables& t, double* Ja, double* J) {
  const int N = p + 1, Nd = ipow(N, nd);
  std::vector<double> g(9 * Nd), V(3 * Nd), a(Nd), b(Nd);
  for (long long e = 0; e < E; ++e) {
    const double* X = xyz + (size_t)e * nd * Nd;
    double* Jae = Ja + (size_t)e * nd * nd * Nd;
    double* Je = J + (size_t)e * Nd;
    // g[(k*nd + m)*Nd + i] = d x_m / d xi_k
    for (int k = 0; k < nd; ++k)
      for (int m = 0; m < nd; ++m) deriv(nd, N, t.D, k, X + (size_t)m * Nd, &g[(k * nd + m) * Nd]);
    if (nd == 2) {
      for (int i = 0; i < Nd; ++i) {
        const double x_1 = g[0 * Nd + i], y_1 = g[1 * Nd + i], x_2 = g[2 * Nd + i], y_2 = g[3 * Nd + i];
        Jae[0 * Nd + i] = y_2;   // (Ja^1)_1
        Jae[1 * Nd + i] = -x_2;  // (Ja^1)_2
        Jae[2 * Nd + i] = -y_1;  // (Ja^2)_1
        Jae[3 * Nd + i] = x_1;   // (Ja^2)_2
        Je[i] = x_1 * y_2 - x_2 * y_1;
      }
    } else {
      for (int i = 0; i < Nd; ++i) {
        double c[3][3];
        for (int k = 0; k < 3; ++k)
          for (int m = 0; m < 3; ++m) c[k][m] = g[(k * 3 + m) * Nd + i];
        Je[i] = c[0][0] * (c[1][1] * c[2][2] - c[2][1] * c[1][2]) + c[0][1] * (c[1][2] * c[2][0] - c[1][0] * c[2][2]) +
                c[0][2] * (c[1][0] * c[2][1] - c[1][1] * c[2][0]);
      }
      for (int j = 0; j < 3; ++j) {
        const int m = (j + 1) % 3, l = (j + 2) % 3;
        // X_l relative to the element's first node: the curl of c grad X_m is zero for constant c, so the metric
        // is unchanged, and the rounding of the products scales with the element size instead of with |x|.
        const double x0 = X[(size_t)l * Nd];
        for (int k = 0; k < 3; ++k)
          for (int i = 0; i < Nd; ++i) V[k * Nd + i] = (X[(size_t)l * Nd + i] - x0) * g[(k * 3 + m) * Nd + i];
        for (int n = 0; n < 3; ++n) {
          const int n1 = (n + 1) % 3, n2 = (n + 2) % 3;
          deriv(3, N, t.D, n1, &V[n2 * Nd], a.data());
          deriv(3, N, t.D, n2, &V[n1 * Nd], b.data());
          for (int i = 0; i < Nd; ++i) Jae[(n * 3 + j) * Nd + i] = b[i] - a[i];
        }
      }
    }
    for (int i = 0; i < Nd; ++i)
      if (!(Je[i] > 0.0)) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------------------------------
// Context helpers
// ---------------------------------------------------------------------------------------------------

dg_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return DG_OK;
  if (e == cudaErrorMemoryAllocation) return DG_ERR_OOM;
  return DG_ERR_CUDA;
}

template <typename T>
cudaError_t dev_alloc(T** p, size_t count) {
  return cudaMalloc((void**)p, count * sizeof(T) + 16);
}

void release(dg_ctx* c) {
  if (!c) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  cudaFree(c->d_Ja);
  cudaFree(c->d_Ja32);
  cudaFree(c->d_invJ);
  cudaFree(c->d_JW);
  cudaFree(c->d_face);
  cudaFree(c->d_fadj);
  cudaFree(c->d_gface);
  cudaFree(c->d_hstage);
  if (c->up_stream) {
    cudaStreamDestroy(c->up_stream);
    for (int k = 0; k <= dgk::kUploadChunks; ++k) cudaEventDestroy(c->up_ev[k]);
  }
  cudaFree(c->d_red);
  cudaFree(c->d_fgeo);
  cudaFree(c->d_flag);
  cudaFree(c->d_tiles);
  if (c->prof_ev) {
    for (int i = 0; i < 2 * c->prof_cap; ++i) cudaEventDestroy(c->prof_ev[i]);
    free(c->prof_ev);
  }
  free(c->prof_kid);
  free(c->h_xyz);
  free(c->h_Ja);
  free(c->h_J);
  if (prev >= 0) cudaSetDevice(prev);
  delete c;
}

// Bounded wait on `s`: poll an event for up to `seconds`.
dg_status bounded_sync(cudaStream_t s, double seconds) {
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaEventRecord(ev, s);
  if (e != cudaSuccess) {
    cudaEventDestroy(ev);
    return cuda_status(e);
  }
  dg_status st = DG_ERR_TIMEOUT;
  const long long max_polls = (long long)(seconds * 1e4);
  for (long long i = 0; i < max_polls; ++i) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) {
      st = DG_OK;
      break;
    }
    if (e != cudaErrorNotReady) {
      st = cuda_status(e);
      break;
    }
    struct timespec ts = {0, 100000};  // 100 us
    nanosleep(&ts, nullptr);
  }
  cudaEventDestroy(ev);
  return st;
}

}  // namespace

namespace dgk {
void prof_begin(dg_ctx* c, int kid, cudaStream_t s, int* slot);
void prof_end(dg_ctx* c, cudaStream_t s, int slot);
}  // namespace dgk

namespace {
// The Gauss collocation RHS (Sec. 6): entropy projection, interface fluxes, volume term (store du, or the stage
// update of *epi).
dg_status gauss_rhs(dg_ctx* c, const double* u, double* du, const dgk::Epilogue* epi, cudaStream_t s) {
  dgk::GaussLaunch L{};
  L.nd = c->nd;
  L.p = c->p;
  L.llf = c->surface_flux == DG_SURF_EC_LLF;
  L.md = c->md;
  L.u = u;
  L.gface = c->d_gface;
  L.fstar = static_cast<double*>(c->d_face);
  L.du = du;
  for (int d = 0; d < 3; ++d) L.c[d] = c->gauss_c[d];
  L.gamma = c->gamma;
  L.flag = c->d_flag;
  L.epi = epi;
  L.s = s;
  const int kid[3] = {dgk::KID_PROJECT, dgk::KID_INTERFACE, dgk::KID_VOLUME};
  for (int part = 0; part < 3; ++part) {
    L.part = part;
    int slot;
    dgk::prof_begin(c, kid[part], s, &slot);
    const cudaError_t e = dgk::launch_gauss(L);
    dgk::prof_end(c, s, slot);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return DG_OK;
}
}  // namespace

namespace dgk {
const RefTables& ref_tables(int p) {
  struct All {
    RefTables t[DG_MAXN];
    All() {
      for (int q = 1; q < DG_MAXN; ++q) build_ref_tables(q, &t[q]);
    }
  };
  static const All all;  // thread-safe one-time initialisation
  return all.t[p];
}
}  // namespace dgk

// ---------------------------------------------------------------------------------------------------
// Profiling hooks used by the launch wrappers
// ---------------------------------------------------------------------------------------------------
namespace dgk {
void prof_begin(dg_ctx* c, int kid, cudaStream_t s, int* slot) {
  *slot = -1;
  c->launches++;
  if (!c->prof_on || !((c->prof_mask >> kid) & 1u) || c->prof_used >= c->prof_cap) return;
  if (c->prof_seen[kid]++ % c->prof_every != 0) return;  // every prof_every-th launch of the kernel
  *slot = c->prof_used++;
  c->prof_kid[*slot] = kid;
  cudaEventRecord(c->prof_ev[2 * *slot], s);
}
void prof_end(dg_ctx* c, cudaStream_t s, int slot) {
  if (slot >= 0) cudaEventRecord(c->prof_ev[2 * slot + 1], s);
}
}  // namespace dgk

// ---------------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------------
extern "C" {

const char* dg_status_string(dg_status s) {
  switch (s) {
    case DG_OK: return "ok";
    case DG_ERR_ARG: return "invalid argument";
    case DG_ERR_CUDA: return "CUDA runtime error";
    case DG_ERR_OOM: return "device out of memory";
    case DG_ERR_UNSUPPORTED: return "unsupported";
    case DG_ERR_NONPHYSICAL: return "non-physical state (rho <= 0, p <= 0 or NaN)";
    case DG_ERR_TIMEOUT: return "timeout";
  }
  return "unknown status";
}

}  // extern "C"

namespace {
// dg_init and dg_init_part: part == nullptr builds the context of the whole mesh; otherwise that of the slab of
// element layers [part->begin, part->end) along the last direction, with a ghost layer in front.
dg_status init_ctx(dg_ctx** out, const dg_mesh* mesh, int polydeg, const dg_metrics* metrics, const dg_opts* opts,
                   const dg_part* part) {
  if (!out || !mesh || !opts) return DG_ERR_ARG;
  *out = nullptr;
  const int nd = mesh->ndims;
  if (nd != 2 && nd != 3) return DG_ERR_ARG;
  if (polydeg < 1 || polydeg >= DG_MAXN) return DG_ERR_UNSUPPORTED;
  for (int d = 0; d < nd; ++d) {
    if (mesh->nelem[d] < 1 || mesh->nelem[d] > (1 << 20)) return DG_ERR_ARG;
    if (!(mesh->hi[d] > mesh->lo[d])) return DG_ERR_ARG;
  }
  if (mesh->mapping < DG_MAP_AFFINE || mesh->mapping > DG_MAP_NODES) return DG_ERR_ARG;
  if (mesh->mapping == DG_MAP_NODES && !mesh->node_xyz_host) return DG_ERR_ARG;
  if (!(opts->gamma > 1.0)) return DG_ERR_ARG;
  if (opts->volume_flux != DG_VOL_RANOCHA && opts->volume_flux != DG_VOL_SHIMA) return DG_ERR_ARG;
  if (opts->surface_flux != DG_SURF_EC && opts->surface_flux != DG_SURF_EC_LLF) return DG_ERR_ARG;
  if (opts->precision != DG_FP64 && opts->precision != DG_FP32) return DG_ERR_ARG;
  if (opts->launch != DG_LAUNCH_OVERLAP && opts->launch != DG_LAUNCH_SERIAL) return DG_ERR_ARG;
  if (opts->staging < DG_STAGING_AUTO || opts->staging > DG_STAGING_PIPELINED) return DG_ERR_ARG;
  if (opts->nodes != DG_NODES_LGL && opts->nodes != DG_NODES_GAUSS) return DG_ERR_ARG;
  const bool gauss = opts->nodes == DG_NODES_GAUSS;
  if (gauss && (mesh->mapping != DG_MAP_AFFINE || (metrics && metrics->Ja_host) || opts->precision != DG_FP64 ||
                opts->volume_flux != DG_VOL_RANOCHA || opts->precompute_logs || opts->logmean))
    return DG_ERR_UNSUPPORTED;
  if (opts->precompute_logs != 0 && opts->precompute_logs != 1) return DG_ERR_ARG;
  if (opts->logmean < DG_LOGMEAN_SHARED_RCP || opts->logmean > DG_LOGMEAN_ALG_POLY) return DG_ERR_ARG;
  if ((opts->precompute_logs || opts->logmean) && opts->volume_flux != DG_VOL_RANOCHA) return DG_ERR_UNSUPPORTED;
  if (opts->precompute_logs && opts->logmean != DG_LOGMEAN_SHARED_RCP) return DG_ERR_UNSUPPORTED;
  if (!(opts->p_ref >= 0.0) || !isfinite(opts->p_ref)) return DG_ERR_ARG;
  if (opts->p_ref != 0.0 && opts->precision == DG_FP32 && (opts->precompute_logs || opts->logmean))
    return DG_ERR_UNSUPPORTED;
  if (metrics && ((metrics->Ja_host == nullptr) != (metrics->J_host == nullptr))) return DG_ERR_ARG;
  // local element counts: a slab has its own layers plus the ghost layer along the last direction
  int nloc[3] = {mesh->nelem[0], mesh->nelem[1], nd == 3 ? mesh->nelem[2] : 1};
  if (part) {
    const int nlast = mesh->nelem[nd - 1];
    if (part->begin < 0 || part->end <= part->begin || part->end > nlast) return DG_ERR_ARG;
    if (mesh->mapping == DG_MAP_NODES || (metrics && metrics->Ja_host) || gauss) return DG_ERR_UNSUPPORTED;
    nloc[nd - 1] = part->end - part->begin + 1;
  }
  const long long n3 = nd == 3 ? nloc[2] : 1;
  const long long E = (long long)nloc[0] * nloc[1] * n3;
  const int N = polydeg + 1, Nd = ipow(N, nd), nv = nd + 2;
  if (E * Nd * nv > (1LL << 31) - 1) return DG_ERR_UNSUPPORTED;  // 32-bit node offsets in the kernels

  dg_ctx* c = new (std::nothrow) dg_ctx();
  if (!c) return DG_ERR_OOM;
  memset(c, 0, sizeof(*c));
  cudaError_t ce = cudaGetDevice(&c->device);
  if (ce != cudaSuccess) {
    delete c;
    return cuda_status(ce);
  }
  c->nd = nd;
  c->p = polydeg;
  c->N = N;
  c->Nd = Nd;
  c->nv = nv;
  c->md.n1 = nloc[0];
  c->md.n2 = nloc[1];
  c->md.n3 = (int)n3;
  c->layer = part ? (nd == 3 ? (long long)nloc[0] * nloc[1] : nloc[0]) : 0;
  c->owned_elems = E - c->layer;
  c->part_dir = part ? nd - 1 : -1;
  c->part_begin = part ? part->begin : 0;
  c->part_end = part ? part->end : 0;
  c->var.ghost = (int)c->layer;
  c->ndofs = c->owned_elems * Nd;  // the DOF the context computes (a slab: its own elements)
  c->md.E = (int)E;
  c->E = E;
  // (c->ndofs is set above: the DOF of the elements the context computes)
  c->state_len = E * Nd * nv;
  c->gamma = opts->gamma;
  c->precision = opts->precision;
  c->surface_flux = opts->surface_flux;
  c->volume_flux = opts->volume_flux;
  c->nodes = opts->nodes;
  // Cartesian specialisation: an affine box mesh has Ja^n = (prod_{k != n} h_k/2) e_n and J = prod_k h_k/2
  c->var.flux = opts->volume_flux;
  c->var.cart = (mesh->mapping == DG_MAP_AFFINE && !(metrics && metrics->Ja_host) &&
                 opts->logmean == DG_LOGMEAN_SHARED_RCP) ? 1 : 0;
  c->var.lm = opts->precompute_logs ? dgk::LM_PRELOG : opts->logmean;  // DG_LOGMEAN_* equal LM_* 0..2
  c->var.pipe = opts->staging == DG_STAGING_AUTO ? 1 : (opts->staging == DG_STAGING_PIPELINED ? 2 : 0);
  c->var.overlap = opts->launch == DG_LAUNCH_OVERLAP ? 1 : 0;
  if (opts->precision == DG_FP32 && opts->p_ref > 0.0) {
    // the kernels form p - p_ref = (gamma-1)_f (E - E_ref - ke/2) with their FP32 gamma - 1: E_ref = p_ref/(gamma-1)_f
    // (FP64) makes (gamma-1)_f E_ref = p_ref exactly in exact arithmetic; p_ref and 2 p_ref are floats
    const float pr = (float)opts->p_ref;
    const float gm1f = (float)opts->gamma - 1.0f;
    const double er = (double)pr / (double)gm1f;
    c->var.sh_eh = (float)er;
    c->var.sh_el = (float)(er - (double)c->var.sh_eh);
    c->var.sh_pp = 2.0f * pr;
  }
  {
    double hh[3] = {1.0, 1.0, 1.0}, jac = 1.0;
    for (int d = 0; d < nd; ++d) {
      hh[d] = 0.5 * (mesh->hi[d] - mesh->lo[d]) / mesh->nelem[d];
      jac *= hh[d];
    }
    for (int d = 0; d < 3; ++d) c->var.jn[d] = d < nd ? jac / hh[d] : 0.0;
    c->var.invJ = 1.0 / jac;
    for (int d = 0; d < 3; ++d) c->gauss_c[d] = d < nd ? 1.0 / hh[d] : 0.0;  // 2/h_n
  }

  // LGL or Legendre-Gauss tables: node coordinates, metric terms and the quadrature weights of J*W follow them
  const dgk::RefTables& t = gauss ? dgk::gauss_tables(polydeg).ref : dgk::ref_tables(polydeg);
  const size_t nx = (size_t)E * nd * Nd, nja = (size_t)E * nd * nd * Nd, nj = (size_t)E * Nd;
  c->h_xyz = (double*)malloc(nx * sizeof(double));
  c->h_Ja = (double*)malloc(nja * sizeof(double));
  c->h_J = (double*)malloc(nj * sizeof(double));
  if (!c->h_xyz || !c->h_Ja || !c->h_J) {
    release(c);
    return DG_ERR_OOM;
  }
  if (mesh->mapping == DG_MAP_NODES)
    memcpy(c->h_xyz, mesh->node_xyz_host, nx * sizeof(double));
  else
    node_coords(mesh, polydeg, t, c->h_xyz, part ? part->begin - 1 : 0, nloc[nd - 1]);
  if (metrics && metrics->Ja_host) {
    memcpy(c->h_Ja, metrics->Ja_host, nja * sizeof(double));
    memcpy(c->h_J, metrics->J_host, nj * sizeof(double));
    for (size_t i = 0; i < nj; ++i)
      if (!(c->h_J[i] > 0.0)) {
        release(c);
        return DG_ERR_ARG;
      }
  } else if (!compute_metrics(nd, polydeg, E, c->h_xyz, t, c->h_Ja, c->h_J)) {
    release(c);
    return DG_ERR_ARG;  // inverted or degenerate element
  }

  // device copies: Ja (FP64, plus an FP32 rounding for the FP32 flux path), 1/J, J*W
  std::vector<double> invJ(nj), JW(nj);
  for (long long e = 0; e < E; ++e)
    for (int i = 0; i < Nd; ++i) {
      double W = 1.0;
      int r = i;
      for (int d = 0; d < nd; ++d) {
        W *= t.w[r % N];
        r /= N;
      }
      invJ[(size_t)e * Nd + i] = 1.0 / c->h_J[(size_t)e * Nd + i];
      JW[(size_t)e * Nd + i] = c->h_J[(size_t)e * Nd + i] * W;
    }
  const size_t nface = (size_t)nd * E * nv * ipow(N, nd - 1);
  const size_t face_bytes = nface * (c->precision == DG_FP32 ? sizeof(float) : sizeof(double));
  ce = dev_alloc(&c->d_Ja, nja);
  if (ce == cudaSuccess) ce = dev_alloc(&c->d_invJ, nj);
  if (ce == cudaSuccess) ce = dev_alloc(&c->d_JW, nj);
  if (ce == cudaSuccess) ce = cudaMalloc(&c->d_face, face_bytes + 16);
  // reduction scratch: entropy-rate pairs or conserved totals (nvar per block), then the result
  if (ce == cudaSuccess) ce = dev_alloc(&c->d_red, (size_t)(nv + 2) * dgk::entropy_rate_blocks() + nv + 2);
  if (ce == cudaSuccess) ce = dev_alloc(&c->d_flag, 1);
  if (ce == cudaSuccess) ce = dev_alloc(&c->d_tiles, 2);
  if (ce == cudaSuccess && c->precision == DG_FP32) ce = dev_alloc(&c->d_Ja32, nja);
  if (ce == cudaSuccess && gauss) ce = dev_alloc(&c->d_gface, 2 * nface);
  if (ce == cudaSuccess) ce = cudaMemcpy(c->d_Ja, c->h_Ja, nja * sizeof(double), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(c->d_invJ, invJ.data(), nj * sizeof(double), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(c->d_JW, JW.data(), nj * sizeof(double), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemset(c->d_flag, 0, sizeof(int));
  if (ce == cudaSuccess) ce = cudaMemset(c->d_tiles, 0, 2 * sizeof(int));
  c->var.tiles = c->d_tiles;
  // interface geometry of FP64 curvilinear contexts: per interface node (element e, direction n, face node l) the
  // lower element's metric vector at its face node scaled by p(p+1)/8 (the lifted flux's factor: 2 x N(N-1)/16) and
  // gamma |m2|^2 / 2, the LLF wave speed's geometric factor (Variant::fgeo, [E][nd][4][NL])
  if (ce == cudaSuccess && c->precision == DG_FP64 && !c->var.cart && !gauss) {
    const int NL = Nd / N;
    std::vector<double> fg((size_t)E * nd * 4 * NL, 0.0);
    const double sc = N * (N - 1) / 8.0;
    for (long long e = 0; e < E; ++e)
      for (int n = 0; n < nd; ++n) {
        const int st = ipow(N, n);
        for (int l = 0; l < NL; ++l) {
          const int node = l % st + (N - 1) * st + (l / st) * st * N;
          double mm = 0.0;
          double* g = &fg[(((size_t)e * nd + n) * 4) * NL + l];
          for (int j = 0; j < nd; ++j) {
            const double m2 = c->h_Ja[(((size_t)e * nd + n) * nd + j) * Nd + node] * sc;
            g[(size_t)j * NL] = m2;
            mm += m2 * m2;
          }
          g[(size_t)3 * NL] = 0.5 * opts->gamma * mm;
        }
      }
    ce = dev_alloc(&c->d_fgeo, fg.size());
    if (ce == cudaSuccess) ce = cudaMemcpy(c->d_fgeo, fg.data(), fg.size() * sizeof(double), cudaMemcpyHostToDevice);
    c->var.fgeo = c->d_fgeo;
  }
  if (ce == cudaSuccess && c->precision == DG_FP32) {
    std::vector<float> ja32(nja);
    for (size_t i = 0; i < nja; ++i) ja32[i] = (float)c->h_Ja[i];
    ce = cudaMemcpy(c->d_Ja32, ja32.data(), nja * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (ce != cudaSuccess) {
    release(c);
    return cuda_status(ce);
  }
  c->prof_cap = 1 << 14;
  c->prof_ev = (cudaEvent_t*)calloc(2 * c->prof_cap, sizeof(cudaEvent_t));
  c->prof_kid = (int*)calloc(c->prof_cap, sizeof(int));
  if (!c->prof_ev || !c->prof_kid) {
    release(c);
    return DG_ERR_OOM;
  }
  for (int i = 0; i < 2 * c->prof_cap; ++i) {
    ce = cudaEventCreate(&c->prof_ev[i]);
    if (ce != cudaSuccess) {
      c->prof_cap = i / 2;
      break;
    }
  }
  *out = c;
  return DG_OK;
}
}  // namespace

extern "C" {

dg_status dg_init(dg_ctx** out, const dg_mesh* mesh, int polydeg, const dg_metrics* metrics, const dg_opts* opts) {
  return init_ctx(out, mesh, polydeg, metrics, opts, nullptr);
}

dg_status dg_init_part(dg_ctx** out, const dg_mesh* mesh, int polydeg, const dg_opts* opts, const dg_part* part) {
  if (!part) return DG_ERR_ARG;
  return init_ctx(out, mesh, polydeg, nullptr, opts, part);
}

dg_status dg_part_get_info(const dg_ctx* c, dg_part_info* info) {
  if (!c || !info || c->layer == 0) return DG_ERR_ARG;
  info->layer = c->layer;
  info->own_elems = c->owned_elems;
  info->ghost_elems = c->layer;
  info->halo_len = c->layer * c->nv * (c->Nd / c->N);
  info->begin = c->part_begin;
  info->end = c->part_end;
  return DG_OK;
}

dg_status dg_part_pack(dg_ctx* c, const double* state, double* send_lo, double* send_hi, dg_stream_t stream) {
  if (!c || c->layer == 0 || !state || !send_lo || !send_hi || send_lo == send_hi) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  c->launches += 1;
  return cuda_status(dgk::launch_halo(c->nd, c->p, (int)c->layer, c->layer, c->E - c->layer, const_cast<double*>(state),
                                      nullptr, nullptr, send_lo, send_hi, true, c->var.overlap != 0, s));
}

dg_status dg_part_unpack(dg_ctx* c, double* state, const double* recv_lo, const double* recv_hi, dg_stream_t stream) {
  if (!c || c->layer == 0 || !state || !recv_lo || !recv_hi) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  c->launches += 1;
  return cuda_status(dgk::launch_halo(c->nd, c->p, (int)c->layer, c->layer, c->E - c->layer, state, recv_lo, recv_hi,
                                      nullptr, nullptr, false, c->var.overlap != 0, s));
}

int dg_stage_input(int scheme, int stage) {
  if (scheme == DG_RK4_CLASSIC) return stage >= 0 && stage < 4 ? (stage > 0 ? 1 : 0) : -1;
  if (scheme == DG_LSRK45_CK) return stage >= 0 && stage < 5 ? 0 : -1;
  return -1;
}

dg_status dg_conserved_totals(dg_ctx* c, const double* q, double* out_host, dg_stream_t stream) {
  if (!c || !q || !out_host) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const int nb = dgk::entropy_rate_blocks();
  c->launches += 2;
  const size_t g = (size_t)c->layer;  // a slab's own elements follow its ghost layer
  cudaError_t e = dgk::launch_totals(c->nd, c->p, c->E - c->layer, q + g * c->nv * c->Nd, c->d_JW + g * c->Nd,
                                     c->d_red, nb, c->d_red + (size_t)c->nv * nb, s);
  if (e != cudaSuccess) return cuda_status(e);
  std::vector<double> res(c->nv);
  e = cudaMemcpyAsync(res.data(), c->d_red + (size_t)c->nv * nb, c->nv * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_status(e);
  const dg_status st = bounded_sync(s, 60.0);
  if (st != DG_OK) return st;
  for (int k = 0; k < c->nv; ++k) out_host[k] = res[k];
  return DG_OK;
}

void dg_free(dg_ctx* ctx) { release(ctx); }

}  // extern "C"

namespace {
// The interface kernel (unless interface_done: already queued, per chunk, by upload_interface) and the volume
// kernel storing du, on stream s.
dg_status rhs_kernels(dg_ctx* c, const double* u, double* du, cudaStream_t s, bool interface_done) {
  int slot;
  const void* ja = c->precision == DG_FP32 ? (const void*)c->d_Ja32 : (const void*)c->d_Ja;
  cudaError_t e = cudaSuccess;
  if (!interface_done) {
    dgk::prof_begin(c, dgk::KID_INTERFACE, s, &slot);
    e = dgk::launch_interface(c->nd, c->p, c->precision, c->surface_flux == DG_SURF_EC_LLF, c->md, u, ja, c->d_face,
                              c->gamma, c->d_flag, s, &c->var);
    dgk::prof_end(c, s, slot);
    if (e != cudaSuccess) return cuda_status(e);
  }
  dgk::prof_begin(c, dgk::KID_VOLUME, s, &slot);
  e = dgk::launch_volume(c->nd, c->p, c->precision, c->md, u, ja, c->d_invJ, c->d_face, du, c->gamma, c->d_flag, s,
                         nullptr, &c->var);
  dgk::prof_end(c, s, slot);
  return cuda_status(e);
}
}  // namespace

extern "C" {

dg_status dg_rhs(dg_ctx* c, const double* u, double* du, double t, dg_stream_t stream) {
  (void)t;
  if (!c || !u || !du) return DG_ERR_ARG;
  const size_t bytes = (size_t)c->state_len * sizeof(double);
  const char *ub = (const char*)u, *db = (const char*)du;
  if (ub < db + bytes && db < ub + bytes) return DG_ERR_ARG;  // u and du overlap
  if (((uintptr_t)u | (uintptr_t)du) & 7) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  if (c->nodes == DG_NODES_GAUSS) return gauss_rhs(c, u, du, nullptr, s);
  return rhs_kernels(c, u, du, s, false);
}

}  // extern "C"

namespace {
// Argument checks shared by dg_step and dg_step_stage.
dg_status check_step_args(const dg_ctx* c, const double* u, const double* scratch, double dt, int scheme) {
  if (!c || !u || !scratch) return DG_ERR_ARG;
  if (scheme != DG_RK4_CLASSIC && scheme != DG_LSRK45_CK) return DG_ERR_ARG;
  if (!(dt == dt)) return DG_ERR_ARG;
  if (c->var.lm == dgk::LM_ALG || c->var.lm == dgk::LM_ALG_POLY) return DG_ERR_UNSUPPORTED;  // dg_rhs only
  if (((uintptr_t)u | (uintptr_t)scratch) & 7) return DG_ERR_ARG;
  const size_t n = (size_t)c->state_len;
  const size_t bytes = n * sizeof(double) * (scheme == DG_RK4_CLASSIC ? 2 : 1);
  const char *ub = (const char*)u, *sb = (const char*)scratch;
  if (ub < sb + bytes && sb < ub + n * sizeof(double)) return DG_ERR_ARG;  // u overlaps the scratch
  return DG_OK;
}

// Stage `st` of the scheme: the interface fluxes of the stage state, then the volume term whose epilogue applies
// the stage update (no du round trip, no update kernel). uw (optional): where the stage writes the updated state
// instead of u (dg_step_host's last stage: the caller's pinned host buffer).
dg_status run_stage(dg_ctx* c, double* u, double* scratch, double dt, int scheme, int st, cudaStream_t s,
                    double* uw = nullptr, bool interface_done = false) {
  const size_t n = (size_t)c->state_len;
  const void* ja = c->precision == DG_FP32 ? (const void*)c->d_Ja32 : (const void*)c->d_Ja;
  dgk::Epilogue epi{};
  epi.mode = scheme == DG_RK4_CLASSIC ? dgk::EPI_RK4 : dgk::EPI_CK45;
  epi.dt = dt;
  epi.u = u;
  epi.uw = uw ? uw : u;
  epi.y = scratch;
  epi.acc = scheme == DG_RK4_CLASSIC ? scratch + n : nullptr;
  // stage state: RK4 evaluates u, then y; CK45 evaluates u (updated in place)
  const double* in = dg_stage_input(scheme, st) == 1 ? scratch : u;
  epi.stage = st;
  if (scheme == DG_LSRK45_CK) dgk::ck45_coefficients(st, &epi.a, &epi.b);
  epi.ca = (st == 0 || st == 3) ? dt / 6.0 : dt / 3.0;
  epi.cy = st == 2 ? dt : 0.5 * dt;
  if (c->nodes == DG_NODES_GAUSS) return gauss_rhs(c, in, nullptr, &epi, s);
  int slot;
  cudaError_t e = cudaSuccess;
  if (!interface_done) {  // (dg_step_host's first stage: queued per chunk of the state by upload_interface)
    dgk::prof_begin(c, dgk::KID_INTERFACE, s, &slot);
    e = dgk::launch_interface(c->nd, c->p, c->precision, c->surface_flux == DG_SURF_EC_LLF, c->md, in, ja,
                              c->d_face, c->gamma, c->d_flag, s, &c->var);
    dgk::prof_end(c, s, slot);
    if (e != cudaSuccess) return cuda_status(e);
  }
  dgk::prof_begin(c, dgk::KID_VOLUME, s, &slot);
  e = dgk::launch_volume(c->nd, c->p, c->precision, c->md, in, ja, c->d_invJ, c->d_face, nullptr, c->gamma,
                         c->d_flag, s, &epi, &c->var);
  dgk::prof_end(c, s, slot);
  return cuda_status(e);
}
}  // namespace

extern "C" {

dg_status dg_step(dg_ctx* c, double* u, double* scratch, double t, double dt, int scheme, dg_stream_t stream) {
  (void)t;
  dg_status st = check_step_args(c, u, scratch, dt, scheme);
  if (st != DG_OK) return st;
  if (c->layer) return DG_ERR_UNSUPPORTED;  // a slab exchanges halos between stages: dg_step_stage
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const int stages = scheme == DG_RK4_CLASSIC ? 4 : 5;
  for (int k = 0; k < stages; ++k) {
    st = run_stage(c, u, scratch, dt, scheme, k, s);
    if (st != DG_OK) return st;
  }
  return DG_OK;
}

dg_status dg_step_stage(dg_ctx* c, double* u, double* scratch, double t, double dt, int scheme, int stage,
                        dg_stream_t stream) {
  (void)t;
  const dg_status st = check_step_args(c, u, scratch, dt, scheme);
  if (st != DG_OK) return st;
  if (dg_stage_input(scheme, stage) < 0) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return run_stage(c, u, scratch, dt, scheme, stage, s);
}

dg_status dg_stage_interface(dg_ctx* c, double* u, double* scratch, int scheme, int stage, int region,
                             dg_stream_t stream) {
  dg_status st = check_step_args(c, u, scratch, 0.0, scheme);
  if (st != DG_OK) return st;
  if (!c->layer || dg_stage_input(scheme, stage) < 0) return DG_ERR_ARG;
  if (region != DG_REGION_INTERIOR && region != DG_REGION_BOUNDARY) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const double* in = dg_stage_input(scheme, stage) == 1 ? scratch : u;
  const void* ja = c->precision == DG_FP32 ? (const void*)c->d_Ja32 : (const void*)c->d_Ja;
  const long long E = c->md.E, layer = c->layer;
  // elements [layer, E - layer): the own layers but the last, whose faces read only own layers; the rest, one
  // range wrapping around: the last own layer [E - layer, E) and the ghost layer [0, layer) (its faces along the
  // cut only, the kernel's ghost rule)
  const long long e0 = region == DG_REGION_INTERIOR ? layer : E - layer;
  const long long e1 = region == DG_REGION_INTERIOR ? E - layer : E + layer;
  if (e1 <= e0) return DG_OK;  // a slab of one own layer has no interior faces
  dgk::Variant v = c->var;
  v.if_e0 = (int)e0;
  v.if_e1 = (int)e1;
  int slot;
  dgk::prof_begin(c, dgk::KID_INTERFACE, s, &slot);
  const cudaError_t e = dgk::launch_interface(c->nd, c->p, c->precision, c->surface_flux == DG_SURF_EC_LLF, c->md,
                                              in, ja, c->d_face, c->gamma, c->d_flag, s, &v);
  dgk::prof_end(c, s, slot);
  return cuda_status(e);
}

dg_status dg_stage_volume(dg_ctx* c, double* u, double* scratch, double t, double dt, int scheme, int stage,
                          dg_stream_t stream) {
  (void)t;
  const dg_status st = check_step_args(c, u, scratch, dt, scheme);
  if (st != DG_OK) return st;
  if (!c->layer || dg_stage_input(scheme, stage) < 0) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return run_stage(c, u, scratch, dt, scheme, stage, s, nullptr, true);
}

// Device staging of dg_step_host / dg_rhs_host: three state arrays, allocated at the first call.
static dg_status ensure_host_staging(dg_ctx* c) {
  if (!c->d_hstage) {
    const dg_status st = cuda_status(dev_alloc(&c->d_hstage, (size_t)c->state_len * 3));
    if (st != DG_OK) return st;
  }
  if (c->up_stream) return DG_OK;
  cudaEvent_t ev[1 + dgk::kUploadChunks];
  int made = 0;
  cudaError_t e = cudaSuccess;
  for (; made <= dgk::kUploadChunks; ++made)
    if ((e = cudaEventCreateWithFlags(&ev[made], cudaEventDisableTiming)) != cudaSuccess) break;
  cudaStream_t us = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&us, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    return cuda_status(e);
  }
  for (int k = 0; k <= dgk::kUploadChunks; ++k) c->up_ev[k] = ev[k];
  c->up_stream = us;
  return DG_OK;
}

// Brings the host state u_host into u (device) for dg_step_host / dg_rhs_host. On LGL meshes with at least two
// element layers per chunk along the last direction, the copy runs in kUploadChunks (2) chunks of layers on the
// context's copy stream, and the interface kernel of u is queued on s per chunk: the faces of the elements whose
// upper neighbours have all arrived (each face flux reads an element and its upper neighbour; the last layer's
// upper neighbour across the periodic boundary is the first chunk's), so that the copy of each chunk overlaps the
// interface fluxes of the one before. *interface_done tells the caller that the interface fluxes of u are queued.
// Otherwise one copy on s.
static dg_status upload_interface(dg_ctx* c, double* u, const double* u_host, cudaStream_t s, bool* interface_done) {
  *interface_done = false;
  const long long nlayer = c->nd == 3 ? c->md.n3 : c->md.n2;
  const long long per_layer = (long long)c->md.E / nlayer;  // elements per layer along the last direction
  const size_t per_elem = (size_t)c->nv * c->Nd;          // doubles per element
  constexpr int K = dgk::kUploadChunks;
  if (c->nodes == DG_NODES_GAUSS || nlayer < 2 * K)
    return cuda_status(cudaMemcpyAsync(u, u_host, (size_t)c->state_len * sizeof(double), cudaMemcpyHostToDevice, s));
  // the copies may start once the work queued on s before this call (which may read u) is done
  cudaError_t e = cudaEventRecord(c->up_ev[0], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->up_stream, c->up_ev[0], 0);
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    const long long z0 = k * nlayer / K, z1 = (k + 1) * nlayer / K;
    const size_t off = (size_t)(z0 * per_layer) * per_elem;
    e = cudaMemcpyAsync(u + off, u_host + off, (size_t)((z1 - z0) * per_layer) * per_elem * sizeof(double),
                        cudaMemcpyHostToDevice, c->up_stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->up_ev[1 + k], c->up_stream);
  }
  if (e != cudaSuccess) return cuda_status(e);
  const void* ja = c->precision == DG_FP32 ? (const void*)c->d_Ja32 : (const void*)c->d_Ja;
  for (int k = 0; k < K; ++k) {
    // chunk k holds layers [z_k, z_k+1): the elements of layers [z_k - 1, z_k+1 - 1) have all their upper
    // neighbours in chunks 0..k (the first part starts at layer 0, the last one ends at the last layer)
    const long long zk = k * nlayer / K, zn = (k + 1) * nlayer / K;
    dgk::Variant v = c->var;
    v.if_e0 = (int)(k == 0 ? 0 : (zk - 1) * per_layer);
    v.if_e1 = (int)(k == K - 1 ? c->md.E : (zn - 1) * per_layer);
    e = cudaStreamWaitEvent(s, c->up_ev[1 + k], 0);
    if (e != cudaSuccess) return cuda_status(e);
    int slot;
    dgk::prof_begin(c, dgk::KID_INTERFACE, s, &slot);
    e = dgk::launch_interface(c->nd, c->p, c->precision, c->surface_flux == DG_SURF_EC_LLF, c->md, u, ja, c->d_face,
                              c->gamma, c->d_flag, s, &v);
    dgk::prof_end(c, s, slot);
    if (e != cudaSuccess) return cuda_status(e);
  }
  *interface_done = true;
  return DG_OK;
}

// The device address of pinned host memory (nullptr for pageable memory): a kernel can then write results into the
// caller's host buffer as it computes them (over the CPU-GPU link, overlapped with the computation).
static double* mapped_host(void* p) {
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) {
    cudaGetLastError();  // not page-locked: clear the (non-sticky) error and copy instead
    return nullptr;
  }
  return static_cast<double*>(d);
}

dg_status dg_step_host(dg_ctx* c, double* u_host, double t, double dt, int scheme, dg_stream_t stream) {
  (void)t;
  if (!c || !u_host) return DG_ERR_ARG;
  if (c->layer) return DG_ERR_UNSUPPORTED;
  dg_status st = ensure_host_staging(c);
  if (st != DG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)c->state_len * sizeof(double);
  double* u = c->d_hstage;
  st = check_step_args(c, u, u + c->state_len, dt, scheme);
  if (st != DG_OK) return st;
  // pinned u_host: the last stage's volume kernel writes the new state straight into it (no device-to-host copy)
  double* out = mapped_host(u_host);
  c->last_stream = s;
  bool if_done = false;
  st = upload_interface(c, u, u_host, s, &if_done);  // the first stage's input is u
  if (st != DG_OK) return st;
  const int stages = scheme == DG_RK4_CLASSIC ? 4 : 5;
  for (int k = 0; k < stages; ++k) {
    st = run_stage(c, u, u + c->state_len, dt, scheme, k, s, k == stages - 1 ? out : nullptr, k == 0 && if_done);
    if (st != DG_OK) return st;
  }
  if (out) return DG_OK;
  return cuda_status(cudaMemcpyAsync(u_host, u, bytes, cudaMemcpyDeviceToHost, s));
}

dg_status dg_rhs_host(dg_ctx* c, const double* u_host, double* du_host, double t, dg_stream_t stream) {
  if (!c || !u_host || !du_host) return DG_ERR_ARG;
  if (c->layer) return DG_ERR_UNSUPPORTED;
  dg_status st = ensure_host_staging(c);
  if (st != DG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)c->state_len * sizeof(double);
  double* u = c->d_hstage;
  // pinned du_host: the volume kernel stores du straight into it (no device-to-host copy)
  double* out = mapped_host(du_host);
  double* du = out ? out : u + c->state_len;
  c->last_stream = s;
  bool if_done = false;
  st = upload_interface(c, u, u_host, s, &if_done);
  if (st != DG_OK) return st;
  st = if_done ? rhs_kernels(c, u, du, s, true) : dg_rhs(c, u, du, t, stream);
  if (st != DG_OK) return st;
  if (out) return DG_OK;
  return cuda_status(cudaMemcpyAsync(du_host, du, bytes, cudaMemcpyDeviceToHost, s));
}

dg_status dg_entropy_rate(dg_ctx* c, const double* u, const double* du, double* out_host, double* abs_out_host,
                          dg_stream_t stream) {
  if (!c || !u || !du || !out_host) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const int nb = dgk::entropy_rate_blocks();
  c->launches += 2;
  dgk::MeshDims own = c->md;  // a slab's own elements follow its ghost layer
  own.E = (int)(c->E - c->layer);
  const size_t g = (size_t)c->layer;
  cudaError_t e = dgk::launch_entropy_rate(c->nd, c->p, own, u + g * c->nv * c->Nd, du + g * c->nv * c->Nd,
                                           c->d_JW + g * c->Nd, c->gamma, c->d_red, nb, c->d_red + 2 * nb, s);
  if (e != cudaSuccess) return cuda_status(e);
  double res[2];
  e = cudaMemcpyAsync(res, c->d_red + 2 * nb, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_status(e);
  dg_status st = bounded_sync(s, 60.0);
  if (st != DG_OK) return st;
  *out_host = res[0];
  if (abs_out_host) *abs_out_host = res[1];
  return DG_OK;
}

dg_status dg_check_status(dg_ctx* c) {
  if (!c) return DG_ERR_ARG;
  dg_status st = bounded_sync(c->last_stream, 60.0);
  if (st != DG_OK) return st;
  int flag = 0;
  cudaError_t e = cudaMemcpy(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  if (flag) {
    e = cudaMemset(c->d_flag, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_status(e);
    // bit 0: a non-physical state; bit 2 (FLAG_WAIT_TIMEOUT): a kernel's bounded wait on its own copies ran out
    return (flag & dgk::FLAG_WAIT_TIMEOUT) ? DG_ERR_TIMEOUT : DG_ERR_NONPHYSICAL;
  }
  return DG_OK;
}

dg_status dg_selftest_wait_timeout(dg_ctx* c, dg_stream_t stream) {
  if (!c) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  c->launches += 1;
  return cuda_status(dgk::launch_wait_probe(c->d_flag, s));
}

dg_status dg_get_info(const dg_ctx* c, dg_info* info) {
  if (!c || !info) return DG_ERR_ARG;
  info->ndims = c->nd;
  info->polydeg = c->p;
  info->nvar = c->nv;
  info->nodes_per_elem = c->Nd;
  info->nelem_total = c->E;
  info->ndofs = c->ndofs;
  info->state_len = c->state_len;
  info->precision = c->precision;
  info->surface_flux = c->surface_flux;
  return DG_OK;
}

dg_status dg_get_node_coords(const dg_ctx* c, double* xyz) {
  if (!c || !xyz) return DG_ERR_ARG;
  memcpy(xyz, c->h_xyz, (size_t)c->E * c->nd * c->Nd * sizeof(double));
  return DG_OK;
}

dg_status dg_get_metrics(const dg_ctx* c, double* Ja, double* J) {
  if (!c || (!Ja && !J)) return DG_ERR_ARG;
  if (Ja) memcpy(Ja, c->h_Ja, (size_t)c->E * c->nd * c->nd * c->Nd * sizeof(double));
  if (J) memcpy(J, c->h_J, (size_t)c->E * c->Nd * sizeof(double));
  return DG_OK;
}

dg_status dg_profile_enable_sampled(dg_ctx* c, unsigned mask, int every) {
  if (!c || every < 1) return DG_ERR_ARG;
  c->prof_mask = mask;
  c->prof_every = every;
  c->prof_on = mask ? 1 : 0;
  c->prof_used = 0;
  for (int k = 0; k < dgk::KID_COUNT; ++k) c->prof_seen[k] = 0;
  return DG_OK;
}

dg_status dg_profile_enable_kernels(dg_ctx* c, unsigned mask) { return dg_profile_enable_sampled(c, mask, 1); }

dg_status dg_profile_enable(dg_ctx* c, int on) { return dg_profile_enable_sampled(c, on ? ~0u : 0u, 1); }

dg_status dg_profile_read(dg_ctx* c, int which, double* total_ms, long long* launches) {
  if (!c || which < 0 || which >= dgk::KID_COUNT || !total_ms) return DG_ERR_ARG;
  double tot = 0.0;
  long long n = 0;
  for (int i = 0; i < c->prof_used; ++i) {
    if (c->prof_kid[i] != which) continue;
    cudaError_t e = cudaEventSynchronize(c->prof_ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_status(e);
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_status(e);
    tot += ms;
    ++n;
  }
  *total_ms = tot;
  if (launches) *launches = n;
  return DG_OK;
}

long long dg_launch_count(const dg_ctx* c) { return c ? c->launches : -1; }

}  // extern "C"
