/*
 * oracle.c -- plain, slow, obviously correct FP64 reference for the right-hand side of entropy-stable,
 * kinetic-energy-preserving flux-differencing LGL-DGSEM for the compressible Euler equations
 * (Ranocha, Schlottke-Lakemper, Chan, Rueda-Ramirez, Winters, Hindenlang, Gassner, arXiv:2112.10517).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * build, load or call this file. The library (the CUDA path) shares no code, header, table or helper
 * with it, and the library never calls it.
 *
 * What it computes, and in which form (deliberately not the form the GPU path uses):
 *   - the strong form with the derivative matrix D and an explicit pointwise-flux surface term
 *     (Sec. 2, Eq. strong-form-SBP with the flux-differencing volume term of Eq. fluxdiff-SBP),
 *   - ALL ordered node pairs, including k = i, on each tensor line (Sec. 2.3, tensor-product sparsity),
 *   - CARTESIAN two-point fluxes contracted with the averaged contravariant vectors
 *     (Sec. 2.3, Eq. curvilinear-rewrite), not directional ones,
 *   - the plain logarithmic mean (Sec. 3.1, Eq. logmean) evaluated with log1p, not Algorithms 1-3,
 *   - 1/{{rho/p}}_log taken literally (Eq. flux_ranocha), not the division-free rewrite.
 * All arithmetic is IEEE double (orc_ld_t only for the LGL tables). Loops are in the paper's order.
 *
 * Data layout (shared with the test harness, not with the library):
 *   node index   i = i1 + N*i2 + N*N*i3 (i1 along xi_1 fastest), N = p+1, Nd = N^ndims nodes
 *   element      e = e1 + n1*(e2 + n2*e3) (lexicographic, e1 fastest); every direction periodic
 *   state        u[(e*nvar + v)*Nd + i], nvar = ndims+2, variables (rho, rho v_1..rho v_d, rho e)
 *   metrics      Ja[((e*ndims + n)*ndims + j)*Nd + i] = (Ja^n)_j: reference direction n, Cartesian j
 *   Jacobian     J[e*Nd + i]
 *   coordinates  xyz[(e*ndims + m)*Nd + i]
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Long double for the LGL tables; a typedef so that oracle_dual.cpp can compile this file with `double` taken
   as a dual number (forward-mode derivatives for the JVP). */
#ifndef ORC_LD_DEFINED
typedef long double orc_ld_t;
#endif

#define ORC_MAXN 16
#define ORC_PI_L 3.141592653589793238462643383279502884L

/* ------------------------------------------------------------------------------------------------ */
/* Legendre-Gauss-Lobatto nodes and weights (Sec. 2, LGL example: diagonal-norm SBP operators that   */
/* include the boundary nodes). Nodes: +-1 and the roots of P_p'; weights 2/(p(p+1) P_p(x)^2).       */
/* ------------------------------------------------------------------------------------------------ */

/* P_p(x) and P_{p-1}(x) by the three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static void orc_legendre(orc_ld_t x, int p, orc_ld_t* Pp, orc_ld_t* Pm1) {
  orc_ld_t P0 = 1.0L, P1 = x;
  if (p == 0) { *Pp = 1.0L; *Pm1 = 0.0L; return; }
  for (int k = 1; k < p; ++k) {
    orc_ld_t P2 = ((2.0L * k + 1.0L) * x * P1 - (orc_ld_t)k * P0) / (k + 1.0L);
    P0 = P1;
    P1 = P2;
  }
  *Pp = P1;
  *Pm1 = P0;
}

int orc_lgl(int p, double* x, double* w) {
  if (p < 1 || p >= ORC_MAXN) return -1;
  orc_ld_t X[ORC_MAXN];
  X[0] = -1.0L;
  X[p] = 1.0L;
  for (int i = 1; i < p; ++i) {
    /* Newton on P_p'(x) = 0. P_p' from (1-x^2) P_p' = p (P_{p-1} - x P_p); P_p'' from Legendre's ODE
       (1-x^2) P'' - 2x P' + p(p+1) P = 0. Start from the Chebyshev-Lobatto point. */
    orc_ld_t xi = -cosl(ORC_PI_L * (orc_ld_t)i / (orc_ld_t)p);
    for (int it = 0; it < 200; ++it) {
      orc_ld_t P, Pm;
      orc_legendre(xi, p, &P, &Pm);
      orc_ld_t one_m = 1.0L - xi * xi;
      orc_ld_t dP = (orc_ld_t)p * (Pm - xi * P) / one_m;
      orc_ld_t d2P = (2.0L * xi * dP - (orc_ld_t)p * (p + 1.0L) * P) / one_m;
      orc_ld_t dx = dP / d2P;
      xi -= dx;
      if (fabsl(dx) < 1e-19L) break;
    }
    X[i] = xi;
  }
  for (int i = 0; i <= p; ++i) {
    orc_ld_t P, Pm;
    orc_legendre(X[i], p, &P, &Pm);
    x[i] = (double)X[i];
    w[i] = (double)(2.0L / ((orc_ld_t)p * (p + 1.0L) * P * P));
  }
  return 0;
}

/* Nodal derivative matrix D (Sec. 2, Def. derivative matrix): D_ik = l_k'(x_i) of the Lagrange basis,
   by barycentric differentiation: lambda_k = 1/prod_{m!=k}(x_k - x_m),
   D_ik = (lambda_k/lambda_i)/(x_i - x_k) for i != k, and D_ii = -sum_{k!=i} D_ik (rows of D kill constants).
   D is row-major, D[i*N + k]. */
int orc_dmat(int p, const double* x, double* D) {
  if (p < 1 || p >= ORC_MAXN) return -1;
  const int N = p + 1;
  orc_ld_t lam[ORC_MAXN];
  for (int k = 0; k < N; ++k) {
    orc_ld_t prod = 1.0L;
    for (int m = 0; m < N; ++m)
      if (m != k) prod *= ((orc_ld_t)x[k] - (orc_ld_t)x[m]);
    lam[k] = 1.0L / prod;
  }
  for (int i = 0; i < N; ++i) {
    orc_ld_t diag = 0.0L;
    for (int k = 0; k < N; ++k) {
      if (k == i) continue;
      orc_ld_t dik = (lam[k] / lam[i]) / ((orc_ld_t)x[i] - (orc_ld_t)x[k]);
      D[i * N + k] = (double)dik;
      diag -= dik;
    }
    D[i * N + i] = (double)diag;
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------------ */
/* Compressible Euler equations with a perfect gas (Sec. 3, Eq. Euler).                              */
/* ------------------------------------------------------------------------------------------------ */

/* conserved -> primitive (rho, v, p), p = (gamma-1)(rho e - rho|v|^2/2) */
static void orc_prim(const double* u, int nd, double gamma, double* rho, double* v, double* p) {
  *rho = u[0];
  double kin = 0.0;
  for (int j = 0; j < nd; ++j) {
    v[j] = u[1 + j] / u[0];
    kin += u[1 + j] * v[j];
  }
  *p = (gamma - 1.0) * (u[nd + 1] - 0.5 * kin);
}

/* physical flux f^j(u) (Eq. Euler): (rho v_j, rho v_j v_i + p delta_ij, (rho e + p) v_j) */
void orc_euler_flux(const double* u, int nd, double gamma, int j, double* f) {
  double rho, v[3], p;
  orc_prim(u, nd, gamma, &rho, v, &p);
  f[0] = u[1 + j];
  for (int i = 0; i < nd; ++i) f[1 + i] = u[1 + j] * v[i] + (i == j ? p : 0.0);
  f[nd + 1] = (u[nd + 1] + p) * v[j];
}

/* logarithmic mean {{a}}_log = [[a]]/[[log a]] (Sec. 3.1, Eq. logmean) = a x/log(1 + x), x = (b - a)/a,
   written with log1p so that it stays accurate for b close to a. For abs(x) < 0.05 it is evaluated by the
   Taylor series of x/log(1 + x) through x^10 (the Gregory coefficients; truncation below 3e-17 relative): the
   closed form keeps its value there but its derivative loses about eps/abs(x) to cancellation (the dual-number
   JVP differentiates this function). NOT Algorithms 1-3. */
static const double ORC_GREGORY[11] = {1.0, 1.0 / 2.0, -1.0 / 12.0, 1.0 / 24.0, -19.0 / 720.0, 3.0 / 160.0,
                                       -863.0 / 60480.0, 275.0 / 24192.0, -33953.0 / 3628800.0, 8183.0 / 1036800.0,
                                       -3250433.0 / 479001600.0};

double orc_logmean(double a, double b) {
  double d = b - a;
  double x = d / a;
  if (fabs(x) < 0.05) {
    double s = ORC_GREGORY[10];
    for (int k = 9; k >= 0; --k) s = ORC_GREGORY[k] + x * s;
    return a * s;
  }
  return d / log1p(x);
}

/* Ranocha's EC/KEP/PEP flux in Cartesian direction j (Sec. 3.2, Eq. flux_ranocha with n = e_j):
     f_rho   = {{rho}}_log {{v_j}}
     f_rhov  = f_rho {{v}} + {{p}} e_j
     f_rhoe  = f_rho ((v;v))/2 + f_rho / ({{rho/p}}_log (gamma-1)) + ((p; v_j))
   with {{a}} = (a_+ + a_-)/2 and ((a;b)) = (a_+ b_- + a_- b_+)/2 (Eq. prodmean). */
void orc_flux_ranocha_cart(const double* um, const double* up, int nd, double gamma, int j, double* f) {
  double rm, vm[3], pm, rp, vp[3], pp;
  orc_prim(um, nd, gamma, &rm, vm, &pm);
  orc_prim(up, nd, gamma, &rp, vp, &pp);
  double rho_log = orc_logmean(rm, rp);
  double beta_log = orc_logmean(rm / pm, rp / pp); /* {{rho/p}}_log */
  double vj_avg = 0.5 * (vm[j] + vp[j]);
  double p_avg = 0.5 * (pm + pp);
  double vv_prod = 0.0; /* ((v;v)) = sum_i (v+_i v-_i + v-_i v+_i)/2 */
  for (int i = 0; i < nd; ++i) vv_prod += 0.5 * (vp[i] * vm[i] + vm[i] * vp[i]);
  double pvj_prod = 0.5 * (pp * vm[j] + pm * vp[j]); /* ((p; v_j)) */
  f[0] = rho_log * vj_avg;
  for (int i = 0; i < nd; ++i) f[1 + i] = f[0] * 0.5 * (vm[i] + vp[i]) + (i == j ? p_avg : 0.0);
  f[nd + 1] = f[0] * vv_prod / 2.0 + f[0] / (beta_log * (gamma - 1.0)) + pvj_prod;
}

/* Flux of Shima et al. (kinetic energy and pressure equilibrium preserving, not EC) in Cartesian direction j
   (Sec. 3.2, Eq. flux_shima_etal with n = e_j):
     f_rho  = {{rho}} {{v_j}}
     f_rhov = f_rho {{v}} + {{p}} e_j
     f_rhoe = f_rho ((v;v))/2 + {{p}} {{v_j}} / (gamma-1) + ((p; v_j)) */
void orc_flux_shima_cart(const double* um, const double* up, int nd, double gamma, int j, double* f) {
  double rm, vm[3], pm, rp, vp[3], pp;
  orc_prim(um, nd, gamma, &rm, vm, &pm);
  orc_prim(up, nd, gamma, &rp, vp, &pp);
  double rho_avg = 0.5 * (rm + rp);
  double vj_avg = 0.5 * (vm[j] + vp[j]);
  double p_avg = 0.5 * (pm + pp);
  double vv_prod = 0.0;
  for (int i = 0; i < nd; ++i) vv_prod += 0.5 * (vp[i] * vm[i] + vm[i] * vp[i]);
  double pvj_prod = 0.5 * (pp * vm[j] + pm * vp[j]);
  f[0] = rho_avg * vj_avg;
  for (int i = 0; i < nd; ++i) f[1 + i] = f[0] * 0.5 * (vm[i] + vp[i]) + (i == j ? p_avg : 0.0);
  f[nd + 1] = f[0] * vv_prod / 2.0 + p_avg * vj_avg / (gamma - 1.0) + pvj_prod;
}

/* Cartesian two-point flux: flux 0 = Ranocha (Eq. flux_ranocha), 1 = Shima et al. (Eq. flux_shima_etal) */
static void orc_flux_cart(int flux, const double* um, const double* up, int nd, double gamma, int j, double* f) {
  if (flux == 1)
    orc_flux_shima_cart(um, up, nd, gamma, j, f);
  else
    orc_flux_ranocha_cart(um, up, nd, gamma, j, f);
}

/* Directional two-point flux in a (not necessarily unit) direction m: the fluxes are linear in the
   direction, so f(u-, u+, m) = sum_j m_j F_j(u-, u+) (Sec. 2.3, the directional flux obtained from
   Eq. curvilinear-rearrange); the length of m scales the result as in the last step of Alg. 4. */
void orc_flux_dir(int flux, const double* um, const double* up, int nd, double gamma, const double* m, double* f) {
  const int nv = nd + 2;
  double Fj[5];
  for (int c = 0; c < nv; ++c) f[c] = 0.0;
  for (int j = 0; j < nd; ++j) {
    orc_flux_cart(flux, um, up, nd, gamma, j, Fj);
    for (int c = 0; c < nv; ++c) f[c] += m[j] * Fj[c];
  }
}

/* Surface flux f*(u_in, u_out, m): the directional two-point flux (the volume flux, as in the paper's runs,
   Sec. 4.1), minus (when llf != 0) local
   Lax-Friedrichs dissipation lambda/2 (u_out - u_in) with
   lambda = max(|v_in.m| + c_in |m|, |v_out.m| + c_out |m|), c = sqrt(gamma p / rho)
   (Sec. 4.2, surface dissipation; the formula is the standard Rusanov flux, not printed in the paper). */
void orc_surface_flux(int flux, const double* uin, const double* uout, int nd, double gamma, const double* m,
                      int llf, double* f) {
  const int nv = nd + 2;
  orc_flux_dir(flux, uin, uout, nd, gamma, m, f);
  if (!llf) return;
  double ri, vi[3], pi, ro, vo[3], po;
  orc_prim(uin, nd, gamma, &ri, vi, &pi);
  orc_prim(uout, nd, gamma, &ro, vo, &po);
  double mnorm = 0.0, vni = 0.0, vno = 0.0;
  for (int j = 0; j < nd; ++j) {
    mnorm += m[j] * m[j];
    vni += vi[j] * m[j];
    vno += vo[j] * m[j];
  }
  mnorm = sqrt(mnorm);
  double li = fabs(vni) + sqrt(gamma * pi / ri) * mnorm;
  double lo = fabs(vno) + sqrt(gamma * po / ro) * mnorm;
  double lam = li > lo ? li : lo;
  for (int c = 0; c < nv; ++c) f[c] -= 0.5 * lam * (uout[c] - uin[c]);
}

/* Batched wrappers used by the tests (n states, each nvar contiguous). */
void orc_flux_dir_batch(int flux, int n, const double* um, const double* up, int nd, double gamma, const double* m,
                        double* f) {
  const int nv = nd + 2;
  for (int s = 0; s < n; ++s) orc_flux_dir(flux, um + s * nv, up + s * nv, nd, gamma, m + s * nd, f + s * nv);
}
void orc_surface_flux_batch(int flux, int n, const double* uin, const double* uout, int nd, double gamma,
                            const double* m, int llf, double* f) {
  const int nv = nd + 2;
  for (int s = 0; s < n; ++s)
    orc_surface_flux(flux, uin + s * nv, uout + s * nv, nd, gamma, m + s * nd, llf, f + s * nv);
}
void orc_euler_flux_batch(int n, const double* u, int nd, double gamma, int j, double* f) {
  const int nv = nd + 2;
  for (int s = 0; s < n; ++s) orc_euler_flux(u + s * nv, nd, gamma, j, f + s * nv);
}
void orc_logmean_batch(int n, const double* a, const double* b, double* out) {
  for (int s = 0; s < n; ++s) out[s] = orc_logmean(a[s], b[s]);
}

/* ------------------------------------------------------------------------------------------------ */
/* Entropy (Sec. 2, entropy pair and Def. of EC fluxes). For Euler the pair under which Ranocha's flux */
/* is EC: U = -rho s/(gamma-1), s = log p - gamma log rho; entropy flux F^j = U v_j;                  */
/* entropy variables w = dU/du = ((gamma - s)/(gamma-1) - rho|v|^2/(2p), rho v/p, -rho/p).            */
/* ------------------------------------------------------------------------------------------------ */

double orc_entropy(const double* u, int nd, double gamma) {
  double rho, v[3], p;
  orc_prim(u, nd, gamma, &rho, v, &p);
  double s = log(p) - gamma * log(rho);
  return -rho * s / (gamma - 1.0);
}

void orc_entropy_vars(const double* u, int nd, double gamma, double* w) {
  double rho, v[3], p;
  orc_prim(u, nd, gamma, &rho, v, &p);
  double s = log(p) - gamma * log(rho);
  double v2 = 0.0;
  for (int j = 0; j < nd; ++j) v2 += v[j] * v[j];
  w[0] = (gamma - s) / (gamma - 1.0) - 0.5 * rho * v2 / p;
  for (int j = 0; j < nd; ++j) w[1 + j] = rho * v[j] / p;
  w[nd + 1] = -rho / p;
}

void orc_entropy_batch(int n, const double* u, int nd, double gamma, double* U, double* w) {
  const int nv = nd + 2;
  for (int s = 0; s < n; ++s) {
    if (U) U[s] = orc_entropy(u + s * nv, nd, gamma);
    if (w) orc_entropy_vars(u + s * nv, nd, gamma, w + s * nv);
  }
}

/* ------------------------------------------------------------------------------------------------ */
/* Structured periodic mesh: node coordinates and curvilinear metric terms (Sec. 2.3).               */
/* ------------------------------------------------------------------------------------------------ */

static int orc_ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

/* Node coordinates of a periodic box [lo, hi] split into nelem[m] elements per direction, mapped by
   mapping 0 (affine: x = xi) or mapping 1 (sine-perturbed: x_m = xi_m + amp (L_m/2pi) prod_k sin(2pi(xi_k - c_k)/L_k),
   c the box centre; on [-pi,pi]^d this is x_m = xi_m + amp prod_k sin(xi_k)). */
int orc_coords(int nd, const int* nelem, const double* lo, const double* hi, int p, int mapping, double amp,
               double* xyz) {
  if (nd < 2 || nd > 3 || p < 1 || p >= ORC_MAXN) return -1;
  const int N = p + 1, Nd = orc_ipow(N, nd);
  double xg[ORC_MAXN], wg[ORC_MAXN];
  orc_lgl(p, xg, wg);
  const int n1 = nelem[0], n2 = nelem[1], n3 = nd == 3 ? nelem[2] : 1;
  const double twopi = 6.283185307179586476925286766559;
  for (int e3 = 0; e3 < n3; ++e3)
    for (int e2 = 0; e2 < n2; ++e2)
      for (int e1 = 0; e1 < n1; ++e1) {
        const int e = e1 + n1 * (e2 + n2 * e3);
        const int eidx[3] = {e1, e2, e3};
        for (int i = 0; i < Nd; ++i) {
          const int ii[3] = {i % N, (i / N) % N, i / (N * N)};
          double xi[3], x[3];
          for (int m = 0; m < nd; ++m) {
            double h = (hi[m] - lo[m]) / nelem[m];
            xi[m] = lo[m] + h * (eidx[m] + 0.5 * (xg[ii[m]] + 1.0));
          }
          double prod = 1.0;
          for (int k = 0; k < nd; ++k) {
            double L = hi[k] - lo[k], c = 0.5 * (hi[k] + lo[k]);
            prod *= sin(twopi * (xi[k] - c) / L);
          }
          for (int m = 0; m < nd; ++m) {
            double L = hi[m] - lo[m];
            x[m] = xi[m] + (mapping == 1 ? amp * (L / twopi) * prod : 0.0);
            xyz[(e * nd + m) * Nd + i] = x[m];
          }
        }
      }
  return 0;
}

/* Apply the 1D matrix D along reference direction dir to a nodal field g (Nd values) -> out. */
static void orc_apply_dir(int nd, int N, const double* D, int dir, const double* g, double* out) {
  const int Nd = orc_ipow(N, nd);
  const int stride = orc_ipow(N, dir);
  for (int i = 0; i < Nd; ++i) {
    const int id = (i / stride) % N;
    const int base = i - id * stride;
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += D[id * N + k] * g[base + k * stride];
    out[i] = s;
  }
}

/* Metric terms from nodal coordinates.
   2D (Sec. 2.3, cross-product form): (Ja^1)_1 = D_2 x^2, (Ja^1)_2 = -D_2 x^1, (Ja^2)_1 = -D_1 x^2,
      (Ja^2)_2 = D_1 x^1, J = (Ja^2)_2 (Ja^1)_1 - (Ja^1)_2 (Ja^2)_1.
   3D, curl_form != 0 (Sec. 2.3: metric identities for free-stream preservation, Kopriva 2006):
      (Ja^n)_j = -e_n . curl_xi( I^N( X_l grad_xi X_m ) ) with (j, m, l) cyclic; the nodal products are
      formed first, then D is applied along the curl's directions, so sum_n D_n (Ja^n)_j = 0 discretely.
   3D, curl_form == 0: cross-product form (Ja^n) = a_{n+1} x a_{n+2} with a_k = D_k x at each node;
      it does not satisfy the discrete metric identities on curved elements (negative control only).
   J (3D): det of the covariant matrix [D_k x_m] at each node. */
int orc_metrics(int nd, int p, int nelem_total, const double* xyz, int curl_form, double* Ja, double* J) {
  if (nd < 2 || nd > 3 || p < 1 || p >= ORC_MAXN) return -1;
  const int N = p + 1, Nd = orc_ipow(N, nd);
  double xg[ORC_MAXN], wg[ORC_MAXN], D[ORC_MAXN * ORC_MAXN];
  orc_lgl(p, xg, wg);
  orc_dmat(p, xg, D);
  double* dx = (double*)malloc(sizeof(double) * 9 * Nd); /* dx[(k*3 + m)*Nd + i] = D_k x_m */
  double* V = (double*)malloc(sizeof(double) * 3 * Nd);
  double* tmp = (double*)malloc(sizeof(double) * Nd);
  double* tmp2 = (double*)malloc(sizeof(double) * Nd);
  for (int e = 0; e < nelem_total; ++e) {
    const double* X = xyz + (size_t)e * nd * Nd;
    double* Jae = Ja + (size_t)e * nd * nd * Nd;
    for (int k = 0; k < nd; ++k)
      for (int m = 0; m < nd; ++m) orc_apply_dir(nd, N, D, k, X + m * Nd, dx + (k * 3 + m) * Nd);
    if (nd == 2) {
      for (int i = 0; i < Nd; ++i) {
        const double x1_xi1 = dx[(0 * 3 + 0) * Nd + i], x2_xi1 = dx[(0 * 3 + 1) * Nd + i];
        const double x1_xi2 = dx[(1 * 3 + 0) * Nd + i], x2_xi2 = dx[(1 * 3 + 1) * Nd + i];
        Jae[(0 * 2 + 0) * Nd + i] = x2_xi2;  /* (Ja^1)_1 */
        Jae[(0 * 2 + 1) * Nd + i] = -x1_xi2; /* (Ja^1)_2 */
        Jae[(1 * 2 + 0) * Nd + i] = -x2_xi1; /* (Ja^2)_1 */
        Jae[(1 * 2 + 1) * Nd + i] = x1_xi1;  /* (Ja^2)_2 */
        J[(size_t)e * Nd + i] = Jae[(1 * 2 + 1) * Nd + i] * Jae[(0 * 2 + 0) * Nd + i] -
                                Jae[(0 * 2 + 1) * Nd + i] * Jae[(1 * 2 + 0) * Nd + i];
      }
      continue;
    }
    /* 3D */
    for (int i = 0; i < Nd; ++i) {
      double a[3][3]; /* a[k][m] = d x_m / d xi_k */
      for (int k = 0; k < 3; ++k)
        for (int m = 0; m < 3; ++m) a[k][m] = dx[(k * 3 + m) * Nd + i];
      J[(size_t)e * Nd + i] = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                              a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                              a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    }
    for (int j = 0; j < 3; ++j) {
      const int m = (j + 1) % 3, l = (j + 2) % 3;
      if (!curl_form) {
        for (int n = 0; n < 3; ++n) {
          const int n1 = (n + 1) % 3, n2 = (n + 2) % 3;
          for (int i = 0; i < Nd; ++i) {
            /* (a_{n1} x a_{n2})_j = a_{n1,m} a_{n2,l} - a_{n1,l} a_{n2,m} */
            Jae[(n * 3 + j) * Nd + i] = dx[(n1 * 3 + m) * Nd + i] * dx[(n2 * 3 + l) * Nd + i] -
                                        dx[(n1 * 3 + l) * Nd + i] * dx[(n2 * 3 + m) * Nd + i];
          }
        }
        continue;
      }
      /* V_k = X_l * D_k X_m at the nodes (k = 0,1,2), with X_l taken relative to the element's first node.
         The curl of c grad X_m vanishes for a constant c (tensor-product D's commute), so the metric is the
         same; relative coordinates keep the rounding of the products proportional to the element size h
         instead of to |x| (absolute coordinates make it grow like |x|/h and jump across periodic boundaries). */
      for (int k = 0; k < 3; ++k)
        for (int i = 0; i < Nd; ++i) V[k * Nd + i] = (X[l * Nd + i] - X[l * Nd]) * dx[(k * 3 + m) * Nd + i];
      /* (Ja^n)_j = -(curl V)_n: (curl V)_0 = D_1 V_2 - D_2 V_1, (curl V)_1 = D_2 V_0 - D_0 V_2,
         (curl V)_2 = D_0 V_1 - D_1 V_0 */
      for (int n = 0; n < 3; ++n) {
        const int n1 = (n + 1) % 3, n2 = (n + 2) % 3;
        orc_apply_dir(3, N, D, n1, V + n2 * Nd, tmp);
        orc_apply_dir(3, N, D, n2, V + n1 * Nd, tmp2);
        for (int i = 0; i < Nd; ++i) Jae[(n * 3 + j) * Nd + i] = -(tmp[i] - tmp2[i]);
      }
    }
  }
  free(dx);
  free(V);
  free(tmp);
  free(tmp2);
  return 0;
}

/* ------------------------------------------------------------------------------------------------ */
/* The semidiscretization (Sec. 2, Eq. strong-form-SBP with the volume term of Eq. fluxdiff-SBP,     */
/* volume and surface two-point flux `flux`: 0 Ranocha, 1 Shima et al.)                               */
/* on curvilinear elements via Eq. curvilinear-rewrite):                                             */
/*                                                                                                   */
/*  du_i = -(1/J_i) [ sum_n sum_{k on i's line along xi_n} D_{i_n k_n} sum_j (Ja^n_j(i) + Ja^n_j(k))  */
/*                                                              F_j(u_i, u_k)                        */
/*                  + sum_n [i_n = p] (1/w_p) ( f*(u_i, u_nbr, Ja^n(i)) - sum_j Ja^n_j(i) f^j(u_i) )  */
/*                  + sum_n [i_n = 0] (1/w_0) ( f*(u_i, u_nbr, -Ja^n(nbr)) + sum_j Ja^n_j(i) f^j(u_i) ) ] */
/*                                                                                                   */
/* The volume term is 2 sum_j sum_k (D_j)_{ik} F_j with (D_j)_{ik} = (1/J_i) sum_n alpha^{j,n}_{ik}   */
/* (D_n)_{ik}, alpha the averaged contravariant vector (Sec. 2.3); the surface term is               */
/* M^{-1} R^T B (f* - sum_j N_j R f^j) with the outward scaled normal +-Ja^n on face xi_n = +-1.     */
/* The paper does not print the curvilinear surface flux; here f* takes ONE normal per interface node,  */
/* Ja^n of the element below the interface along xi_n (curl-form metrics agree on both sides up to      */
/* rounding), which keeps the discrete scheme exactly conservative across every interface.             */
/* u_nbr is the coincident node of the neighbour across the face (periodic). Elements                */
/* [elem_begin, elem_end) are computed and stored in du as elements 0 .. elem_end-elem_begin-1.      */
/* scale_mode != 0 returns instead (1/J_i) times the sum of the absolute values of every term above   */
/* (each volume product and both surface products): the magnitude that rounding errors of any         */
/* evaluation of the sum scale with.                                                                  */
/* ------------------------------------------------------------------------------------------------ */

int orc_rhs(int nd, int p, const int* nelem, const double* Ja, const double* J, const double* u, double gamma,
            int flux, int llf, int elem_begin, int elem_end, int scale_mode, double* du) {
  if (nd < 2 || nd > 3 || p < 1 || p >= ORC_MAXN) return -1;
  const int N = p + 1, Nd = orc_ipow(N, nd), nv = nd + 2;
  const int n1 = nelem[0], n2 = nelem[1], n3 = nd == 3 ? nelem[2] : 1;
  double xg[ORC_MAXN], wg[ORC_MAXN], D[ORC_MAXN * ORC_MAXN];
  orc_lgl(p, xg, wg);
  orc_dmat(p, xg, D);
  for (int e = elem_begin; e < elem_end; ++e) {
    const int eidx[3] = {e % n1, (e / n1) % n2, e / (n1 * n2)};
    const int ne[3] = {n1, n2, n3};
    for (int i = 0; i < Nd; ++i) {
      const int ii[3] = {i % N, (i / N) % N, i / (N * N)};
      double ui[5], acc[5] = {0, 0, 0, 0, 0};
      for (int c = 0; c < nv; ++c) ui[c] = u[((size_t)e * nv + c) * Nd + i];
      for (int n = 0; n < nd; ++n) {
        const int stride = orc_ipow(N, n);
        /* volume: all k on the line through i along xi_n, including k = i */
        for (int kn = 0; kn < N; ++kn) {
          const int k = i + (kn - ii[n]) * stride;
          double uk[5], F[5];
          for (int c = 0; c < nv; ++c) uk[c] = u[((size_t)e * nv + c) * Nd + k];
          for (int j = 0; j < nd; ++j) {
            const double a = Ja[(((size_t)e * nd + n) * nd + j) * Nd + i] +
                             Ja[(((size_t)e * nd + n) * nd + j) * Nd + k];
            orc_flux_cart(flux, ui, uk, nd, gamma, j, F);
            for (int c = 0; c < nv; ++c) {
              const double term = D[ii[n] * N + kn] * a * F[c];
              acc[c] += scale_mode ? fabs(term) : term;
            }
          }
        }
        /* surface: faces xi_n = +1 (i_n = p) and xi_n = -1 (i_n = 0) */
        for (int side = 0; side < 2; ++side) {
          const int on_face = side == 0 ? (ii[n] == p) : (ii[n] == 0);
          if (!on_face) continue;
          const double sgn = side == 0 ? 1.0 : -1.0;
          int nb[3] = {eidx[0], eidx[1], eidx[2]};
          nb[n] = (nb[n] + (side == 0 ? 1 : ne[n] - 1)) % ne[n];
          const int enb = nb[0] + n1 * (nb[1] + n2 * nb[2]);
          const int inb = i + ((side == 0 ? 0 : p) - ii[n]) * stride;
          double unb[5], m[3], mf[3], fstar[5], fj[5], fn[5] = {0, 0, 0, 0, 0};
          for (int c = 0; c < nv; ++c) unb[c] = u[((size_t)enb * nv + c) * Nd + inb];
          /* m: outward scaled normal of this element at node i (its own metric); mf: the normal of the
             interface, one per interface node, taken from the element below it along xi_n (the same value
             on both sides, so each interface flux enters the two elements with opposite signs). */
          for (int j = 0; j < nd; ++j) {
            m[j] = sgn * Ja[(((size_t)e * nd + n) * nd + j) * Nd + i];
            mf[j] = side == 0 ? m[j] : -Ja[(((size_t)enb * nd + n) * nd + j) * Nd + inb];
          }
          orc_surface_flux(flux, ui, unb, nd, gamma, mf, llf, fstar);
          for (int j = 0; j < nd; ++j) {
            orc_euler_flux(ui, nd, gamma, j, fj);
            for (int c = 0; c < nv; ++c) fn[c] += m[j] * fj[c];
          }
          const double winv = 1.0 / wg[side == 0 ? p : 0];
          for (int c = 0; c < nv; ++c)
            acc[c] += scale_mode ? winv * (fabs(fstar[c]) + fabs(fn[c])) : winv * (fstar[c] - fn[c]);
        }
      }
      for (int c = 0; c < nv; ++c)
        du[((size_t)(e - elem_begin) * nv + c) * Nd + i] = (scale_mode ? acc[c] : -acc[c]) / J[(size_t)e * Nd + i];
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------------ */
/* Quadrature diagnostics: int q = sum_e sum_i J_i W_i q_i with W_i the tensor LGL weights.          */
/* Entropy rate dS/dt = sum_e sum_i J_i W_i w(u_i) . du_i (Sec. 2, EC/ED semidiscretization).        */
/* ------------------------------------------------------------------------------------------------ */

static double orc_tensor_weight(int nd, int N, const double* wg, int i) {
  double W = 1.0;
  for (int n = 0; n < nd; ++n) {
    W *= wg[i % N];
    i /= N;
  }
  return W;
}

/* out[c] = sum J W q_c for each of the nv fields of q (layout like u); abs_out[c] = sum |J W q_c| */
int orc_integrate(int nd, int p, int nelem_total, const double* J, const double* q, double* out, double* abs_out) {
  const int N = p + 1, Nd = orc_ipow(N, nd), nv = nd + 2;
  double xg[ORC_MAXN], wg[ORC_MAXN];
  orc_lgl(p, xg, wg);
  for (int c = 0; c < nv; ++c) out[c] = abs_out[c] = 0.0;
  for (int e = 0; e < nelem_total; ++e)
    for (int i = 0; i < Nd; ++i) {
      const double JW = J[(size_t)e * Nd + i] * orc_tensor_weight(nd, N, wg, i);
      for (int c = 0; c < nv; ++c) {
        out[c] += JW * q[((size_t)e * nv + c) * Nd + i];
        abs_out[c] += fabs(JW * q[((size_t)e * nv + c) * Nd + i]);
      }
    }
  return 0;
}

/* returns dS/dt; *abs_out = sum |J W w.du| (the scale used for relative checks) */
double orc_entropy_rate(int nd, int p, int nelem_total, const double* J, const double* u, const double* du,
                        double gamma, double* abs_out) {
  const int N = p + 1, Nd = orc_ipow(N, nd), nv = nd + 2;
  double xg[ORC_MAXN], wg[ORC_MAXN];
  orc_lgl(p, xg, wg);
  double s = 0.0, sa = 0.0;
  for (int e = 0; e < nelem_total; ++e)
    for (int i = 0; i < Nd; ++i) {
      double ui[5], w[5];
      for (int c = 0; c < nv; ++c) ui[c] = u[((size_t)e * nv + c) * Nd + i];
      orc_entropy_vars(ui, nd, gamma, w);
      const double JW = J[(size_t)e * Nd + i] * orc_tensor_weight(nd, N, wg, i);
      for (int c = 0; c < nv; ++c) {
        const double t = JW * w[c] * du[((size_t)e * nv + c) * Nd + i];
        s += t;
        sa += fabs(t);
      }
    }
  if (abs_out) *abs_out = sa;
  return s;
}

/* ------------------------------------------------------------------------------------------------ */
/* Time integration (Sec. 4.1): one step of                                                         */
/*   scheme 0: the classical four-stage, fourth-order Runge-Kutta method, textbook full-storage form;  */
/*   scheme 1: the five-stage, fourth-order 2N-storage method of Carpenter and Kennedy (1994), in its  */
/*             Williamson form K <- A_s K + dt f(U); U <- U + B_s K.                                 */
/* ------------------------------------------------------------------------------------------------ */

static const double ORC_CK_A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                                   -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double ORC_CK_B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                                   1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                                   2277821191437.0 / 14882151754819.0};

void orc_ck45_coeffs(double* A, double* B) {
  for (int s = 0; s < 5; ++s) {
    A[s] = ORC_CK_A[s];
    B[s] = ORC_CK_B[s];
  }
}

int orc_rk_step(int scheme, int nd, int p, const int* nelem, const double* Ja, const double* J, double gamma, int flux,
                int llf, double dt, double* u) {
  const int N = p + 1, Nd = orc_ipow(N, nd), nv = nd + 2;
  const int E = nelem[0] * nelem[1] * (nd == 3 ? nelem[2] : 1);
  const size_t n = (size_t)E * nv * Nd;
  if (scheme == 0) {
    double* k[4];
    double* y = (double*)malloc(sizeof(double) * n);
    for (int s = 0; s < 4; ++s) k[s] = (double*)malloc(sizeof(double) * n);
    orc_rhs(nd, p, nelem, Ja, J, u, gamma, flux, llf, 0, E, 0, k[0]);
    for (size_t q = 0; q < n; ++q) y[q] = u[q] + 0.5 * dt * k[0][q];
    orc_rhs(nd, p, nelem, Ja, J, y, gamma, flux, llf, 0, E, 0, k[1]);
    for (size_t q = 0; q < n; ++q) y[q] = u[q] + 0.5 * dt * k[1][q];
    orc_rhs(nd, p, nelem, Ja, J, y, gamma, flux, llf, 0, E, 0, k[2]);
    for (size_t q = 0; q < n; ++q) y[q] = u[q] + dt * k[2][q];
    orc_rhs(nd, p, nelem, Ja, J, y, gamma, flux, llf, 0, E, 0, k[3]);
    for (size_t q = 0; q < n; ++q) u[q] += dt / 6.0 * (k[0][q] + 2.0 * k[1][q] + 2.0 * k[2][q] + k[3][q]);
    free(y);
    for (int s = 0; s < 4; ++s) free(k[s]);
    return 0;
  }
  if (scheme == 1) {
    double* K = (double*)calloc(n, sizeof(double));
    double* f = (double*)malloc(sizeof(double) * n);
    for (int s = 0; s < 5; ++s) {
      orc_rhs(nd, p, nelem, Ja, J, u, gamma, flux, llf, 0, E, 0, f);
      for (size_t q = 0; q < n; ++q) {
        K[q] = ORC_CK_A[s] * K[q] + dt * f[q];
        u[q] += ORC_CK_B[s] * K[q];
      }
    }
    free(K);
    free(f);
    return 0;
  }
  return -1;
}
