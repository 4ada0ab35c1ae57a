/*
 * gauss.c -- plain, slow FP64 reference for the Legendre-Gauss collocation scheme with entropy projection
 * (Sec. 6, Eq. fluxdiff-GSBP-opDsplit with the volume terms of Eq. hybridized_gauss_formulation) on periodic
 * affine boxes (the Cartesian meshes of the paper's GaussSBP runs).
 *
 * TEST INFRASTRUCTURE, like oracle.c (compiled into the same liboracle.so): only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark use it; the library shares no code with it.
 *
 * Form (deliberately not the GPU path's line-by-line form): on every element the DENSE operators of the paper are
 * built over the combined set of volume nodes and face nodes -- M, D_j, the face restriction R (volume -> all face
 * nodes), B N_j (face weights times the outward normal component) -- and the hybridized operators
 *     Q_{h,j} = 1/2 [[M D_j - (M D_j)^T, R^T B N_j], [-B N_j R, 0]];
 * the volume term is M^{-1} [I; R]^T f_hybrid with f_hybrid_a = sum_j sum_b 2 (Q_{h,j})_{ab} f_j(u~_a, u~_b) over
 * all combined points b (Cartesian two-point fluxes f_j, zero operator entries skipped), and the surface term is
 * M^{-1} R^T B f_num. u~ is the entropy projection: u at volume nodes, u(R w(u)) at face nodes.
 *
 * Affine elements: x = x_e + (h/2) xi, so d/dx_j = (2/h_j) d/dxi_j. The mass matrix and the face measures carry
 * the same constant Jacobian, which cancels; the derivative and the normals carry c_j = 2/h_j.
 *
 * Data layout as in oracle.c (u[(e*nvar + v)*Nd + i], node i = i1 + N i2 + N^2 i3, lexicographic elements).
 * Face nodes of an element, f = ((n*2 + s)*NL + t): direction n, side s (0: xi_n = -1, 1: xi_n = +1), t the
 * index over the other directions in increasing order (t = i_a + N i_b, a < b the two other directions).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* from oracle.c (same library) */
int orc_dmat(int p, const double* x, double* D);
void orc_flux_ranocha_cart(const double* um, const double* up, int nd, double gamma, int j, double* f);
void orc_entropy_vars(const double* u, int nd, double gamma, double* w);

#define ORG_MAXN 16
#define ORG_PI_L 3.141592653589793238462643383279502884L

static int org_ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

/* Legendre-Gauss nodes and weights with N = p + 1 points: the roots of P_N, weights 2/((1 - x^2) P_N'(x)^2)
   (Sec. 6: collocation on Legendre-Gauss nodes). Newton on P_N from the guess cos(pi (i + 3/4)/(N + 1/2)),
   P_N' from (1 - x^2) P_N' = N (P_{N-1} - x P_N). Long double, rounded once; nodes ascending. */
int org_gauss(int p, double* x, double* w) {
  if (p < 1 || p >= ORG_MAXN) return -1;
  const int N = p + 1;
  for (int i = 0; i < N; ++i) {
    long double xi = -cosl(ORG_PI_L * ((long double)i + 0.75L) / ((long double)N + 0.5L));
    long double P = 0.0L, Pm = 0.0L, dP = 1.0L;
    for (int it = 0; it < 100; ++it) {
      long double P0 = 1.0L, P1 = xi;
      for (int k = 1; k < N; ++k) {
        long double P2 = ((2.0L * k + 1.0L) * xi * P1 - (long double)k * P0) / (k + 1.0L);
        P0 = P1;
        P1 = P2;
      }
      P = P1;
      Pm = P0;
      dP = (long double)N * (Pm - xi * P) / (1.0L - xi * xi);
      long double dx = P / dP;
      xi -= dx;
      if (fabsl(dx) < 1e-19L) break;
    }
    /* derivative at the converged root */
    {
      long double P0 = 1.0L, P1 = xi;
      for (int k = 1; k < N; ++k) {
        long double P2 = ((2.0L * k + 1.0L) * xi * P1 - (long double)k * P0) / (k + 1.0L);
        P0 = P1;
        P1 = P2;
      }
      dP = (long double)N * (P0 - xi * P1) / (1.0L - xi * xi);
    }
    x[i] = (double)xi;
    w[i] = (double)(2.0L / ((1.0L - xi * xi) * dP * dP));
  }
  return 0;
}

/* Lagrange basis of the nodes x (N = p + 1) at the point s: l_k(s) = prod_{m != k} (s - x_m)/(x_k - x_m). */
void org_lagrange_at(int p, const double* x, double s, double* l) {
  const int N = p + 1;
  for (int k = 0; k < N; ++k) {
    long double v = 1.0L;
    for (int m = 0; m < N; ++m)
      if (m != k) v *= ((long double)s - x[m]) / ((long double)x[k] - x[m]);
    l[k] = (double)v;
  }
}

/* Conserved variables from entropy variables, the inverse of w(u) of oracle.c (Sec. 2: entropy pair
   U = -rho s/(gamma-1), s = log p - gamma log rho): with b = rho/p = -w_last, v = w_v/b,
   s = gamma - (gamma - 1)(w_0 + b|v|^2/2), and s = (1 - gamma) log rho - log b,
   rho = exp((s + log b)/(1 - gamma)), p = rho/b, rho e = p/(gamma - 1) + rho|v|^2/2. */
void org_cons_from_entropy(const double* w, int nd, double gamma, double* u) {
  const double b = -w[nd + 1];
  double v[3], v2 = 0.0;
  for (int j = 0; j < nd; ++j) {
    v[j] = w[1 + j] / b;
    v2 += v[j] * v[j];
  }
  const double s = gamma - (gamma - 1.0) * (w[0] + 0.5 * b * v2);
  const double rho = exp((s + log(b)) / (1.0 - gamma));
  const double p = rho / b;
  u[0] = rho;
  for (int j = 0; j < nd; ++j) u[1 + j] = rho * v[j];
  u[nd + 1] = p / (gamma - 1.0) + 0.5 * rho * v2;
}

void org_cons_from_entropy_batch(int n, const double* w, int nd, double gamma, double* u) {
  for (int k = 0; k < n; ++k) org_cons_from_entropy(w + k * (nd + 2), nd, gamma, u + k * (nd + 2));
}

/* Node coordinates of the Gauss collocation mesh: x_m = lo_m + h_m (e_m + (xi_{i_m} + 1)/2). */
int org_gauss_coords(int nd, const int* nelem, const double* lo, const double* hi, int p, double* xyz) {
  if (nd < 2 || nd > 3 || p < 1 || p >= ORG_MAXN) return -1;
  const int N = p + 1, Nd = org_ipow(N, nd);
  double xg[ORG_MAXN], wg[ORG_MAXN];
  org_gauss(p, xg, wg);
  const int n1 = nelem[0], n2 = nelem[1], n3 = nd == 3 ? nelem[2] : 1;
  for (int e3 = 0; e3 < n3; ++e3)
    for (int e2 = 0; e2 < n2; ++e2)
      for (int e1 = 0; e1 < n1; ++e1) {
        const int e = e1 + n1 * (e2 + n2 * e3);
        const int eidx[3] = {e1, e2, e3};
        for (int i = 0; i < Nd; ++i) {
          const int ii[3] = {i % N, (i / N) % N, i / (N * N)};
          for (int m = 0; m < nd; ++m) {
            const double h = (hi[m] - lo[m]) / nelem[m];
            xyz[(e * nd + m) * Nd + i] = lo[m] + h * (eidx[m] + 0.5 * (xg[ii[m]] + 1.0));
          }
        }
      }
  return 0;
}

/* reference index of volume node i along direction m */
static int org_idx(int i, int m, int N) {
  for (int k = 0; k < m; ++k) i /= N;
  return i % N;
}

/* transverse index t of volume node i for direction n (the other directions in increasing order) */
static int org_transverse(int nd, int N, int i, int n) {
  int t = 0, scale = 1;
  for (int m = 0; m < nd; ++m) {
    if (m == n) continue;
    t += scale * org_idx(i, m, N);
    scale *= N;
  }
  return t;
}

/* neighbour of element e across direction n on side s (0: lower, 1: upper), periodic */
static int org_neighbor(int nd, const int* nelem, int e, int n, int s) {
  int c[3] = {0, 0, 0}, r = e;
  for (int m = 0; m < nd; ++m) {
    c[m] = r % nelem[m];
    r /= nelem[m];
  }
  c[n] = (c[n] + (s ? 1 : -1) + nelem[n]) % nelem[n];
  int out = 0;
  for (int m = nd - 1; m >= 0; --m) out = out * nelem[m] + c[m];
  return out;
}

/* The entropy projection of Sec. 6 on every element: face states u~_f = u(sum_i R_fi w(u_i)) for the Nf face
   nodes of each element (layout [E][Nf][nvar], face node order as above). */
int org_gauss_project(int nd, int p, int E, const double* u, double gamma, double* uface) {
  if (nd < 2 || nd > 3 || p < 1 || p >= ORG_MAXN) return -1;
  const int N = p + 1, Nd = org_ipow(N, nd), NL = org_ipow(N, nd - 1), nv = nd + 2, Nf = 2 * nd * NL;
  double xg[ORG_MAXN], wg[ORG_MAXN], lm[ORG_MAXN], lp[ORG_MAXN];
  org_gauss(p, xg, wg);
  org_lagrange_at(p, xg, -1.0, lm);
  org_lagrange_at(p, xg, 1.0, lp);
  double* wv = (double*)malloc(sizeof(double) * Nd * nv);
  if (!wv) return -2;
  for (int e = 0; e < E; ++e) {
    for (int i = 0; i < Nd; ++i) {
      double ui[5];
      for (int v = 0; v < nv; ++v) ui[v] = u[((size_t)e * nv + v) * Nd + i];
      orc_entropy_vars(ui, nd, gamma, wv + i * nv);
    }
    for (int f = 0; f < Nf; ++f) {
      const int n = f / (2 * NL), s = (f / NL) % 2, t = f % NL;
      double wf[5] = {0, 0, 0, 0, 0};
      for (int i = 0; i < Nd; ++i) {
        if (org_transverse(nd, N, i, n) != t) continue;
        const double r = s ? lp[org_idx(i, n, N)] : lm[org_idx(i, n, N)]; /* R_fi */
        for (int v = 0; v < nv; ++v) wf[v] += r * wv[i * nv + v];
      }
      org_cons_from_entropy(wf, nd, gamma, uface + ((size_t)e * Nf + f) * nv);
    }
  }
  free(wv);
  return 0;
}

/* The Gauss collocation RHS (Sec. 6). flux: Ranocha's EC flux in the volume and at the surface (the paper's
   entropy-conservative runs); llf adds -lambda/2 (u~_out - u~_in) with lambda = c_n max(|v_in,n| + c_in,
   |v_out,n| + c_out), c = sqrt(gamma p/rho), on the projected face states. du has the layout of u. */
int org_gauss_rhs(int nd, int p, const int* nelem, const double* lo, const double* hi, const double* u,
                  double gamma, int llf, double* du) {
  if (nd < 2 || nd > 3 || p < 1 || p >= ORG_MAXN) return -1;
  const int N = p + 1, Nd = org_ipow(N, nd), NL = org_ipow(N, nd - 1), nv = nd + 2;
  const int Nf = 2 * nd * NL, Np = Nd + Nf;
  int E = 1;
  for (int m = 0; m < nd; ++m) E *= nelem[m];
  double xg[ORG_MAXN], wg[ORG_MAXN], D1[ORG_MAXN * ORG_MAXN], lm[ORG_MAXN], lp[ORG_MAXN], c[3];
  org_gauss(p, xg, wg);
  orc_dmat(p, xg, D1);
  org_lagrange_at(p, xg, -1.0, lm);
  org_lagrange_at(p, xg, 1.0, lp);
  for (int m = 0; m < nd; ++m) c[m] = 2.0 / ((hi[m] - lo[m]) / nelem[m]);

  /* dense element operators: W (volume weights), R (Nf x Nd), Bw (face weights), face direction/side */
  double* W = (double*)malloc(sizeof(double) * Nd);
  double* R = (double*)calloc((size_t)Nf * Nd, sizeof(double));
  double* Bw = (double*)malloc(sizeof(double) * Nf);
  int* fdir = (int*)malloc(sizeof(int) * Nf);
  int* fside = (int*)malloc(sizeof(int) * Nf);
  double* MDj = (double*)malloc(sizeof(double) * Nd * Nd);
  double* Qh = (double*)malloc(sizeof(double) * (size_t)nd * Np * Np); /* Q_{h,j}, the same on every element */
  double* ut = (double*)malloc(sizeof(double) * (size_t)E * Np * nv); /* entropy-projected states, all elements */
  double* fh = (double*)malloc(sizeof(double) * Np * nv);
  if (!W || !R || !Bw || !fdir || !fside || !MDj || !Qh || !ut || !fh) return -2;
  for (int i = 0; i < Nd; ++i) {
    W[i] = 1.0;
    for (int m = 0; m < nd; ++m) W[i] *= wg[org_idx(i, m, N)];
  }
  for (int n = 0; n < nd; ++n)
    for (int s = 0; s < 2; ++s)
      for (int t = 0; t < NL; ++t) {
        const int f = (n * 2 + s) * NL + t;
        fdir[f] = n;
        fside[f] = s;
        Bw[f] = 1.0;
        for (int i = 0; i < Nd; ++i) {
          if (org_transverse(nd, N, i, n) != t) continue;
          R[(size_t)f * Nd + i] = s ? lp[org_idx(i, n, N)] : lm[org_idx(i, n, N)];
        }
        /* face weight: product of the transverse 1D weights of t */
        int tt = t;
        for (int m = 0; m < nd; ++m) {
          if (m == n) continue;
          Bw[f] *= wg[tt % N];
          tt /= N;
        }
      }

  /* the hybridized operators of each direction (element-independent on an affine mesh) */
  for (int j = 0; j < nd; ++j) {
    double* Q = Qh + (size_t)j * Np * Np;
    /* M D_j on the volume nodes: (M D_j)_ab = W_a D1[a_j][b_j] when a and b differ only along j */
    for (int a = 0; a < Nd; ++a)
      for (int b = 0; b < Nd; ++b) {
        int same = 1;
        for (int m = 0; m < nd; ++m)
          if (m != j && org_idx(a, m, N) != org_idx(b, m, N)) same = 0;
        MDj[a * Nd + b] = same ? W[a] * D1[org_idx(a, j, N) * N + org_idx(b, j, N)] : 0.0;
      }
    for (int a = 0; a < Np * Np; ++a) Q[a] = 0.0;
    for (int a = 0; a < Nd; ++a)
      for (int b = 0; b < Nd; ++b) Q[a * Np + b] = 0.5 * (MDj[a * Nd + b] - MDj[b * Nd + a]);
    for (int f = 0; f < Nf; ++f) {
      const double bn = fdir[f] == j ? Bw[f] * (fside[f] ? 1.0 : -1.0) : 0.0; /* (B N_j)_ff */
      for (int a = 0; a < Nd; ++a) {
        Q[a * Np + Nd + f] = 0.5 * R[(size_t)f * Nd + a] * bn;    /* R^T B N_j */
        Q[(Nd + f) * Np + a] = -0.5 * bn * R[(size_t)f * Nd + a]; /* -B N_j R */
      }
    }
  }

  /* entropy projection of every element: u~ = [u; u(R w(u))] */
  double* wv = (double*)malloc(sizeof(double) * Nd * nv);
  for (int e = 0; e < E; ++e) {
    double* ue = ut + (size_t)e * Np * nv;
    for (int i = 0; i < Nd; ++i) {
      double ui[5], wi[5];
      for (int v = 0; v < nv; ++v) ui[v] = u[((size_t)e * nv + v) * Nd + i];
      orc_entropy_vars(ui, nd, gamma, wi);
      for (int v = 0; v < nv; ++v) {
        ue[i * nv + v] = ui[v];
        wv[i * nv + v] = wi[v];
      }
    }
    for (int f = 0; f < Nf; ++f) {
      double wf[5] = {0, 0, 0, 0, 0};
      for (int i = 0; i < Nd; ++i)
        for (int v = 0; v < nv; ++v) wf[v] += R[(size_t)f * Nd + i] * wv[i * nv + v];
      org_cons_from_entropy(wf, nd, gamma, ue + (Nd + f) * nv);
    }
  }

  for (int e = 0; e < E; ++e) {
    const double* ue = ut + (size_t)e * Np * nv;
    for (int a = 0; a < Np * nv; ++a) fh[a] = 0.0;
    /* f_hybrid over the combined points, direction by direction */
    for (int j = 0; j < nd; ++j) {
      const double* Q = Qh + (size_t)j * Np * Np;
      for (int a = 0; a < Np; ++a)
        for (int b = 0; b < Np; ++b) {
          const double q = Q[a * Np + b];
          if (q == 0.0) continue;
          double f[5];
          orc_flux_ranocha_cart(ue + a * nv, ue + b * nv, nd, gamma, j, f);
          for (int v = 0; v < nv; ++v) fh[a * nv + v] += c[j] * 2.0 * q * f[v];
        }
    }
    /* numerical fluxes at the face nodes (outward normal sign and the scale c_n included) */
    for (int f = 0; f < Nf; ++f) {
      const int n = fdir[f], s = fside[f], t = f % NL;
      const int en = org_neighbor(nd, nelem, e, n, s);
      const int fo = (n * 2 + (1 - s)) * NL + t; /* the coincident face node of the neighbour */
      const double* uin = ue + (Nd + f) * nv;
      const double* uout = ut + ((size_t)en * Np + Nd + fo) * nv;
      double F[5];
      orc_flux_ranocha_cart(uin, uout, nd, gamma, n, F);
      const double sg = s ? 1.0 : -1.0;
      double fn[5];
      for (int v = 0; v < nv; ++v) fn[v] = sg * F[v];
      if (llf) {
        double lam = 0.0;
        const double* st[2] = {uin, uout};
        for (int k = 0; k < 2; ++k) {
          const double rho = st[k][0];
          double v2 = 0.0;
          for (int m = 0; m < nd; ++m) v2 += st[k][1 + m] * st[k][1 + m];
          const double pr = (gamma - 1.0) * (st[k][nd + 1] - 0.5 * v2 / rho);
          const double l = fabs(st[k][1 + n] / rho) + sqrt(gamma * pr / rho);
          if (l > lam) lam = l;
        }
        for (int v = 0; v < nv; ++v) fn[v] -= 0.5 * lam * (uout[v] - uin[v]);
      }
      /* surface term R^T B f_num, and the face rows of f_hybrid lifted by R^T */
      for (int a = 0; a < Nd; ++a) {
        const double r = R[(size_t)f * Nd + a];
        if (r == 0.0) continue;
        for (int v = 0; v < nv; ++v) fh[a * nv + v] += r * (fh[(Nd + f) * nv + v] + Bw[f] * c[n] * fn[v]);
      }
    }
    for (int a = 0; a < Nd; ++a)
      for (int v = 0; v < nv; ++v) du[((size_t)e * nv + v) * Nd + a] = -fh[a * nv + v] / W[a];
  }
  free(W);
  free(R);
  free(Bw);
  free(fdir);
  free(fside);
  free(MDj);
  free(Qh);
  free(ut);
  free(fh);
  free(wv);
  return 0;
}
