// Legendre-Gauss collocation with entropy projection (Sec. 6, Eq. fluxdiff-GSBP-opDsplit with the volume terms of
// Eq. hybridized_gauss_formulation) on Cartesian (affine) periodic meshes, FP64, Ranocha's flux.
//
// On an affine element the hybridized operators factor into lines: along direction n each line of N Gauss nodes
// couples with its two face points (xi_n = -1, +1), and the transverse quadrature weights cancel. With the 1D Gauss
// weights w, derivative matrix D, S_ik = w_i D_ik - w_k D_ki (the volume block of 2 Q_h), l_k(+-1) the rows of R,
// sigma = -1, +1 the outward normal signs and F(a, b) = f(a, b, c_n e_n) (c_n = 2/h_n):
//   acc_i = sum_k S_ik F(u_i, u_k) + sum_s sigma_s l_i(s) F(u_i, u~_s)      (volume rows of 2 Q_h)
//   H_s   = sum_k l_k(s) F(u~_s, u_k)                                      (face rows, up to -sigma_s)
//   du_i += -(1/w_i) [ acc_i - sum_s sigma_s l_i(s) H_s + sum_s l_i(s) f*_s ] (M^{-1} [I; R]^T and M^{-1} R^T B)
// with u~_s = u(R w(u)) the entropy-projected face states and f*_s the outward interface flux.
//
// Three kernels per RHS: (1) the entropy projection of every element's lines to its face points, (2) one
// interface flux per face node, (3) the volume kernel (line pairs i < k once, node-face-point pairs once, lift,
// surface term, sum over directions, optional Runge-Kutta stage update).
#include <math.h>
#include <string.h>

#include "kernels.cuh"

namespace dgk {

// ---------------------------------------------------------------------------------------------------
// Reference tables (host): Gauss nodes are the roots of P_N; Newton with P_N' from the derivative recurrence
// P'_{k+1} = P'_{k-1} + (2k+1) P_k. Weights 2/((1-x^2) P_N'(x)^2). D by barycentric weights; l_k(+-1) by the
// barycentric interpolation formula.
// ---------------------------------------------------------------------------------------------------
namespace {
void legendre_and_derivative(long double x, int n, long double* P, long double* dP) {
  long double p0 = 1.0L, p1 = x, d0 = 0.0L, d1 = 1.0L;
  if (n == 0) {
    *P = 1.0L;
    *dP = 0.0L;
    return;
  }
  for (int k = 1; k < n; ++k) {
    const long double p2 = ((2.0L * k + 1.0L) * x * p1 - (long double)k * p0) / (k + 1.0L);
    const long double d2 = d0 + (2.0L * k + 1.0L) * p1;
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
  }
  *P = p1;
  *dP = d1;
}

void build_gauss_tables(int p, GaussTables* g) {
  memset(g, 0, sizeof(*g));
  const int N = p + 1;
  long double X[DG_MAXN], lam[DG_MAXN];
  for (int i = 0; i < N; ++i) {
    // the i-th root in ascending order, from the asymptotic guess
    long double x = -cosl(3.141592653589793238462643383279502884L * (4.0L * i + 3.0L) / (4.0L * N + 2.0L));
    long double P, dP;
    for (int it = 0; it < 100; ++it) {
      legendre_and_derivative(x, N, &P, &dP);
      const long double step = P / dP;
      x -= step;
      if (fabsl(step) <= 1e-19L) break;
    }
    legendre_and_derivative(x, N, &P, &dP);
    X[i] = x;
    g->ref.x[i] = (double)x;
    g->ref.w[i] = (double)(2.0L / ((1.0L - x * x) * dP * dP));
  }
  for (int k = 0; k < N; ++k) {
    long double prod = 1.0L;
    for (int m = 0; m < N; ++m)
      if (m != k) prod *= X[k] - X[m];
    lam[k] = 1.0L / prod;
  }
  for (int i = 0; i < N; ++i) {
    long double diag = 0.0L;
    for (int k = 0; k < N; ++k) {
      if (k == i) continue;
      const long double d = (lam[k] / lam[i]) / (X[i] - X[k]);
      g->ref.D[i * N + k] = (double)d;
      diag -= d;
    }
    g->ref.D[i * N + i] = (double)diag;
  }
  for (int side = 0; side < 2; ++side) {
    const long double s = side ? 1.0L : -1.0L;
    long double den = 0.0L, terms[DG_MAXN];
    for (int k = 0; k < N; ++k) {
      terms[k] = lam[k] / (s - X[k]);
      den += terms[k];
    }
    for (int k = 0; k < N; ++k) (side ? g->lp : g->lm)[k] = (double)(terms[k] / den);
  }
}
}  // namespace

const GaussTables& gauss_tables(int p) {
  struct All {
    GaussTables t[DG_MAXN];
    All() {
      for (int q = 1; q < DG_MAXN; ++q) build_gauss_tables(q, &t[q]);
    }
  };
  static const All all;
  return all.t[p];
}

// Kernel-parameter operators along a line
template <int N>
struct GaussOps {
  double S8[N * N];  // (w_i D_ik - w_k D_ki) / 8 (fluxes come scaled by 8)
  double lm8[N], lp8[N];  // l_k(-1)/8, l_k(+1)/8
  double lm[N], lp[N];    // l_k(-1), l_k(+1)
  double winv[N];         // 1/w_i
};

// ---------------------------------------------------------------------------------------------------
// Entropy variables and their inverse (Sec. 2 entropy pair U = -rho s/(gamma-1), s = log p - gamma log rho):
//   w = ((gamma - s)/(gamma-1) - rho|v|^2/(2p), rho v/p, -rho/p)
//   u(w): b = -w_E = rho/p, v = w_v/b, s = gamma - (gamma-1)(w_0 + b|v|^2/2), rho = exp((s + log b)/(1-gamma)).
// Each returns false for a state outside the admissible set (rho, p or b not positive).
// ---------------------------------------------------------------------------------------------------
// igm1 = 1/(gamma - 1), passed in so that neither map divides.
template <int ND>
__device__ __forceinline__ bool entropy_vars(const double* u, double gamma, double igm1, double* w) {
  const double rho = u[0];
  const double ir = Num<double>::rcp(rho);
  double v[ND], mv = 0.0;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    v[j] = u[1 + j] * ir;
    mv += u[1 + j] * v[j];
  }
  const double p = (gamma - 1.0) * (u[ND + 1] - 0.5 * mv);
  const double b = rho * Num<double>::rcp(p);  // rho / p
  const double s = log_f64(p) - gamma * log_f64(rho);
  w[0] = (gamma - s) * igm1 - 0.5 * b * (mv * ir);
#pragma unroll
  for (int j = 0; j < ND; ++j) w[1 + j] = b * v[j];
  w[ND + 1] = -b;
  return rho > 0.0 && p > 0.0;
}

template <int ND>
__device__ __forceinline__ bool cons_from_entropy(const double* w, double gamma, double igm1, double* u) {
  const double b = -w[ND + 1];
  const double ib = Num<double>::rcp(b);
  double v[ND], v2 = 0.0;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    v[j] = w[1 + j] * ib;
    v2 += v[j] * v[j];
  }
  const double s = gamma - (gamma - 1.0) * (w[0] + 0.5 * b * v2);
  const double rho = exp(-(s + log_f64(b)) * igm1);
  const double p = rho * ib;
  u[0] = rho;
#pragma unroll
  for (int j = 0; j < ND; ++j) u[1 + j] = rho * v[j];
  u[ND + 1] = p * igm1 + 0.5 * rho * v2;
  return b > 0.0 && rho > 0.0 && rho < 1e300;
}

// component 1 + n of a register array for a run-time direction n (an unrolled select keeps the array in registers)
template <int ND>
__device__ __forceinline__ double vel(const double* q, int n) {
  double v = q[1];
#pragma unroll
  for (int j = 1; j < ND; ++j)
    if (j == n) v = q[1 + j];
  return v;
}

// Elements per CTA: about 192 threads in the line phases.
template <int ND, int N>
constexpr int gauss_epb() {
  return Geo<ND, N>::TPE >= 192 ? 1 : 192 / Geo<ND, N>::TPE;
}

// ---------------------------------------------------------------------------------------------------
// (1) Entropy projection: w(u) per node in shared memory, then one thread per (element, direction, line)
// interpolates w to the line's two face points and maps back. gface layout [n][E][2][NV][NL] (side 0: xi_n = -1).
// ---------------------------------------------------------------------------------------------------
template <int ND, int N, int EPB>
__global__ void __launch_bounds__(EPB* Geo<ND, N>::TPE)
    gauss_project_kernel(const double* __restrict__ u, double* __restrict__ gface, MeshDims md, GaussOps<N> op,
                         double gamma, int* flag) {
  using G = Geo<ND, N>;
  constexpr int kThreads = EPB * G::TPE;
  __shared__ double s_w[EPB * G::NV * G::NDOF];
  const int e0 = blockIdx.x * EPB, tid = threadIdx.x;
  const int nel = min(EPB, md.E - e0);
  const double igm1 = 1.0 / (gamma - 1.0);
  bool ok = true;
  for (int idx = tid; idx < nel * G::NDOF; idx += kThreads) {
    const int el = idx / G::NDOF, i = idx - el * G::NDOF;
    const double* ue = u + (size_t)(e0 + el) * G::NV * G::NDOF + i;
    double uc[G::NV], w[G::NV];
#pragma unroll
    for (int c = 0; c < G::NV; ++c) uc[c] = ue[c * G::NDOF];
    ok &= entropy_vars<ND>(uc, gamma, igm1, w);
#pragma unroll
    for (int c = 0; c < G::NV; ++c) s_w[(el * G::NV + c) * G::NDOF + i] = w[c];
  }
  __syncthreads();
  if (tid < nel * G::TPE) {
    const int el = tid / G::TPE, r = tid - el * G::TPE;
    const int n = r / G::NL, l = r - n * G::NL;
    const int st = G::stride(n), base = G::line_base(n, l);
    const double* sw = s_w + el * G::NV * G::NDOF + base;
    double wm[G::NV], wp[G::NV];
#pragma unroll
    for (int c = 0; c < G::NV; ++c) {
      double am = 0.0, ap = 0.0;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const double wi = sw[c * G::NDOF + i * st];
        am += op.lm[i] * wi;
        ap += op.lp[i] * wi;
      }
      wm[c] = am;
      wp[c] = ap;
    }
    double um[G::NV], up[G::NV];
    ok &= cons_from_entropy<ND>(wm, gamma, igm1, um);
    ok &= cons_from_entropy<ND>(wp, gamma, igm1, up);
    double* gf = gface + ((size_t)n * md.E + (e0 + el)) * 2 * G::NV * G::NL + l;
#pragma unroll
    for (int c = 0; c < G::NV; ++c) {
      gf[c * G::NL] = um[c];
      gf[(G::NV + c) * G::NL] = up[c];
    }
  }
  if (!ok) atomicOr(flag, 1);
}

// ---------------------------------------------------------------------------------------------------
// (2) Interface flux per face node (element-major like the LGL interface kernel): between the upper face state of
// e and the lower face state of its upper neighbour; fstar8[n][E][NV][NL] = 8 c_n [f(u~_in, u~_out, e_n)
// - lambda/2 (u~_out - u~_in)], the outward flux of e's upper face (e+'s lower face takes its negative).
// ---------------------------------------------------------------------------------------------------
template <int ND, int N, bool LLF>
__global__ void __launch_bounds__(256)
    gauss_interface_kernel(const double* __restrict__ gface, double* __restrict__ fstar8, MeshDims md, double c0,
                           double c1, double c2, double gamma, int* flag) {
  using G = Geo<ND, N>;
  const long long total = (long long)ND * md.E * G::NL;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int idx = (int)g;
  const int fn = idx % G::NL, t = idx / G::NL, n = t % ND, e = t / ND;
  const int eR = upper_neighbor(md, e, n);
  const double cn = n == 0 ? c0 : (n == 1 ? c1 : c2);
  const double* gin = gface + (((size_t)n * md.E + e) * 2 + 1) * G::NV * G::NL + fn;  // e, side 1
  const double* gout = gface + (((size_t)n * md.E + eR) * 2 + 0) * G::NV * G::NL + fn;  // e+, side 0
  double uin[G::NV], uout[G::NV];
#pragma unroll
  for (int c = 0; c < G::NV; ++c) {
    uin[c] = gin[c * G::NL];
    uout[c] = gout[c * G::NL];
  }
  const double gm1 = gamma - 1.0;
  double qa[NodeQ<ND>::NQ], qb[NodeQ<ND>::NQ], F[G::NV], ira, irb;
  const bool ok = node_quantities<ND, double>(uin, gm1, 2.0 / gm1, qa, &ira) &
                  node_quantities<ND, double>(uout, gm1, 2.0 / gm1, qb, &irb);
  if (!ok) atomicOr(flag, 1);
  const double va = vel<ND>(qa, n), vb = vel<ND>(qb, n);
  pair_flux8_cart<ND, double, 0>(qa, qb, va, vb, 2.0 * cn, n, F);
  if (LLF) {
    const double hg = 0.5 * gamma;
    const double la = fabs(va) + sqrt(hg * qa[NodeQ<ND>::PP] * ira);
    const double lb = fabs(vb) + sqrt(hg * qb[NodeQ<ND>::PP] * irb);
    const double lam4 = 4.0 * cn * (la > lb ? la : lb);
#pragma unroll
    for (int c = 0; c < G::NV; ++c) F[c] -= lam4 * (uout[c] - uin[c]);
  }
  double* fo = fstar8 + ((size_t)n * md.E + e) * G::NV * G::NL + fn;
#pragma unroll
  for (int c = 0; c < G::NV; ++c) fo[c * G::NL] = F[c];
}

// ---------------------------------------------------------------------------------------------------
// (3) Volume kernel: node quantities of the element's nodes and of its projected face states in shared memory;
// one thread per (element, direction, line) evaluates the line's pairs i < k once and every node-face-point pair
// once, forms the hybridized volume term, the lifted face rows and the surface term, divides by w_i and leaves
// the direction's contribution in shared memory; then one thread per node sums the directions, negates, and
// stores du or applies the Runge-Kutta stage update.
// ---------------------------------------------------------------------------------------------------
template <int ND, int N, int EPB, int EPI>
__global__ void __launch_bounds__(EPB* Geo<ND, N>::TPE)
    gauss_volume_kernel(const double* __restrict__ u, const double* __restrict__ gface,
                        const double* __restrict__ fstar8, double* __restrict__ du, MeshDims md, GaussOps<N> op,
                        double c0, double c1, double c2, double gamma, int* flag, Epilogue epi) {
  using G = Geo<ND, N>;
  using Q = NodeQ<ND>;
  constexpr int NQ = Q::NQ;
  constexpr int kThreads = EPB * G::TPE;
  constexpr int kFace = ND * 2 * G::NL;  // face points per element
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_q = reinterpret_cast<double*>(smem_raw);  // [EPB][NQ][NDOF]
  double* s_qf = s_q + EPB * NQ * G::NDOF;             // [EPB][NQ][kFace], face point (n*2 + s)*NL + l
  double* s_acc = s_qf + EPB * NQ * kFace;             // [EPB][ND][NV][NDOF]
  const int e0 = blockIdx.x * EPB, tid = threadIdx.x;
  const int nel = min(EPB, md.E - e0);
  const double gm1 = gamma - 1.0, tg = 2.0 / gm1;
  bool ok = true;
  for (int idx = tid; idx < nel * G::NDOF; idx += kThreads) {
    const int el = idx / G::NDOF, i = idx - el * G::NDOF;
    const double* ue = u + (size_t)(e0 + el) * G::NV * G::NDOF + i;
    double uc[G::NV], q[NQ];
#pragma unroll
    for (int c = 0; c < G::NV; ++c) uc[c] = ue[c * G::NDOF];
    ok &= node_quantities<ND, double>(uc, gm1, tg, q);
#pragma unroll
    for (int c = 0; c < NQ; ++c) s_q[(el * NQ + c) * G::NDOF + i] = q[c];
  }
  for (int idx = tid; idx < nel * kFace; idx += kThreads) {
    const int el = idx / kFace, f = idx - el * kFace;
    const int l = f % G::NL, ns = f / G::NL, n = ns >> 1, s = ns & 1;
    const double* gf = gface + (((size_t)n * md.E + (e0 + el)) * 2 + s) * G::NV * G::NL + l;
    double uc[G::NV], q[NQ];
#pragma unroll
    for (int c = 0; c < G::NV; ++c) uc[c] = gf[c * G::NL];
    ok &= node_quantities<ND, double>(uc, gm1, tg, q);
#pragma unroll
    for (int c = 0; c < NQ; ++c) s_qf[(el * NQ + c) * kFace + f] = q[c];
  }
  if (!ok) atomicOr(flag, 1);
  __syncthreads();

  if (tid < nel * G::TPE) {
    const int el = tid / G::TPE, r = tid - el * G::TPE;
    const int n = r / G::NL, l = r - n * G::NL;
    const int st = G::stride(n), base = G::line_base(n, l);
    const double* sp = s_q + el * NQ * G::NDOF + base;
    const double n2n = 2.0 * (n == 0 ? c0 : (n == 1 ? c1 : c2));
    double acc[N][G::NV];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int c = 0; c < G::NV; ++c) acc[i][c] = 0.0;
    // volume pairs i < k (S skew: S_ki = -S_ik)
#pragma unroll
    for (int i = 0; i < N - 1; ++i) {
      double a[NQ];
#pragma unroll
      for (int c = 0; c < NQ; ++c) a[c] = sp[c * G::NDOF + i * st];
#pragma unroll
      for (int k = i + 1; k < N; ++k) {
        double b[NQ], F[G::NV];
#pragma unroll
        for (int c = 0; c < NQ; ++c) b[c] = sp[c * G::NDOF + k * st];
        pair_flux8_cart<ND, double, 0>(a, b, sp[(1 + n) * G::NDOF + i * st], sp[(1 + n) * G::NDOF + k * st], n2n,
                                        n, F);
        const double sik = op.S8[i * N + k];
#pragma unroll
        for (int c = 0; c < G::NV; ++c) {
          acc[i][c] += sik * F[c];
          acc[k][c] -= sik * F[c];
        }
      }
    }
    // node-face-point pairs: F(u_i, u~_s) enters acc_i with sigma_s l_i(s) and H_s with l_i(s)
    double H[2][G::NV];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const double* sf = s_qf + el * NQ * kFace + (n * 2 + s) * G::NL + l;
      double qs[NQ];
#pragma unroll
      for (int c = 0; c < NQ; ++c) qs[c] = sf[c * kFace];
#pragma unroll
      for (int c = 0; c < G::NV; ++c) H[s][c] = 0.0;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        double a[NQ], F[G::NV];
#pragma unroll
        for (int c = 0; c < NQ; ++c) a[c] = sp[c * G::NDOF + i * st];
        pair_flux8_cart<ND, double, 0>(a, qs, sp[(1 + n) * G::NDOF + i * st], sf[(1 + n) * kFace], n2n, n, F);
        const double li8 = s ? op.lp8[i] : op.lm8[i];
#pragma unroll
        for (int c = 0; c < G::NV; ++c) {
          acc[i][c] += (s ? li8 : -li8) * F[c];
          H[s][c] += li8 * F[c];
        }
      }
    }
    // interface fluxes of the line's two face points (outward): +f* of e's upper face, -f* of e-'s upper face
    const int eg = e0 + el;
    const double* fu = fstar8 + ((size_t)n * md.E + eg) * G::NV * G::NL + l;
    const double* fl = fstar8 + ((size_t)n * md.E + neighbor(md, eg, n, -1)) * G::NV * G::NL + l;
    double fsm[G::NV], fsp[G::NV];
#pragma unroll
    for (int c = 0; c < G::NV; ++c) {
      fsp[c] = 0.125 * fu[c * G::NL];
      fsm[c] = -0.125 * fl[c * G::NL];
    }
    double* sa = s_acc + (el * ND + n) * G::NV * G::NDOF + base;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const double lmi = op.lm[i], lpi = op.lp[i];
#pragma unroll
      for (int c = 0; c < G::NV; ++c) {
        // - sum_s sigma_s l_i(s) H_s + sum_s l_i(s) f*_s
        const double t = acc[i][c] + lmi * (H[0][c] + fsm[c]) + lpi * (fsp[c] - H[1][c]);
        sa[c * G::NDOF + i * st] = op.winv[i] * t;
      }
    }
  }
  __syncthreads();

  for (int idx = tid; idx < nel * G::NDOF; idx += kThreads) {
    const int el = idx / G::NDOF, i = idx - el * G::NDOF;
    const size_t off = (size_t)(e0 + el) * G::NV * G::NDOF + i;
#pragma unroll
    for (int c = 0; c < G::NV; ++c) {
      double s = 0.0;
#pragma unroll
      for (int n = 0; n < ND; ++n) s += s_acc[((el * ND + n) * G::NV + c) * G::NDOF + i];
      const size_t o = off + (size_t)c * G::NDOF;
      if (EPI == EPI_STORE)
        du[o] = -s;
      else
        stage_update<EPI>(epi, o, -s, epi.u[o], epi.stage > 0 ? (EPI == EPI_RK4 ? epi.acc[o] : epi.y[o]) : 0.0);
    }
  }
}

// ---------------------------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------------------------
namespace {
template <int N>
GaussOps<N> make_ops(int p) {
  const GaussTables& g = gauss_tables(p);
  GaussOps<N> op;
  for (int i = 0; i < N; ++i) {
    for (int k = 0; k < N; ++k)
      op.S8[i * N + k] = 0.125 * (g.ref.w[i] * g.ref.D[i * N + k] - g.ref.w[k] * g.ref.D[k * N + i]);
    op.lm[i] = g.lm[i];
    op.lp[i] = g.lp[i];
    op.lm8[i] = 0.125 * g.lm[i];
    op.lp8[i] = 0.125 * g.lp[i];
    op.winv[i] = 1.0 / g.ref.w[i];
  }
  return op;
}

template <int ND, int N>
size_t volume_smem() {
  constexpr int EPB = gauss_epb<ND, N>();
  using G = Geo<ND, N>;
  return sizeof(double) * EPB * (NodeQ<ND>::NQ * (G::NDOF + ND * 2 * G::NL) + ND * G::NV * G::NDOF);
}

// One instantiation per epilogue, each with its own one-time opt-in to the dynamic shared memory it needs.
template <int ND, int N, int EPI>
cudaError_t launch_gauss_volume(const GaussLaunch& L, const GaussOps<N>& op, int blocks) {
  constexpr int EPB = gauss_epb<ND, N>();
  const size_t smem = volume_smem<ND, N>();
  auto kern = gauss_volume_kernel<ND, N, EPB, EPI>;
  static PerDeviceCache cache;  // the shared-memory opt-in, once per device
  long long done = 0;
  const cudaError_t a = per_device(cache, &done, [&](long long* v) {
    *v = 1;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (a != cudaSuccess) return a;
  const Epilogue epi = L.epi ? *L.epi : Epilogue{};
  kern<<<blocks, EPB * Geo<ND, N>::TPE, smem, L.s>>>(L.u, L.gface, L.fstar, L.du, L.md, op, L.c[0], L.c[1], L.c[2],
                                                     L.gamma, L.flag, epi);
  return cudaGetLastError();
}

template <int ND, int N>
cudaError_t gauss_rhs_n(const GaussLaunch& L) {
  constexpr int EPB = gauss_epb<ND, N>();
  using G = Geo<ND, N>;
  const MeshDims md = L.md;
  const GaussOps<N> op = make_ops<N>(N - 1);
  const int blocks = (md.E + EPB - 1) / EPB;
  cudaError_t e = cudaSuccess;
  if (L.part == 0) {
    gauss_project_kernel<ND, N, EPB><<<blocks, EPB * G::TPE, 0, L.s>>>(L.u, L.gface, md, op, L.gamma, L.flag);
    e = cudaGetLastError();
  } else if (L.part == 1) {
    const long long total = (long long)ND * md.E * G::NL;
    const unsigned nb = (unsigned)((total + 255) / 256);
    if (L.llf)
      gauss_interface_kernel<ND, N, true><<<nb, 256, 0, L.s>>>(L.gface, L.fstar, md, L.c[0], L.c[1], L.c[2],
                                                               L.gamma, L.flag);
    else
      gauss_interface_kernel<ND, N, false><<<nb, 256, 0, L.s>>>(L.gface, L.fstar, md, L.c[0], L.c[1], L.c[2],
                                                                L.gamma, L.flag);
    e = cudaGetLastError();
  } else {
    if (!L.epi || L.epi->mode == EPI_STORE)
      e = launch_gauss_volume<ND, N, EPI_STORE>(L, op, blocks);
    else if (L.epi->mode == EPI_RK4)
      e = launch_gauss_volume<ND, N, EPI_RK4>(L, op, blocks);
    else
      e = launch_gauss_volume<ND, N, EPI_CK45>(L, op, blocks);
  }
  return e;
}

template <int ND>
cudaError_t gauss_rhs_nd(const GaussLaunch& L) {
  switch (L.p) {
    case 1: return gauss_rhs_n<ND, 2>(L);
    case 2: return gauss_rhs_n<ND, 3>(L);
    case 3: return gauss_rhs_n<ND, 4>(L);
    case 4: return gauss_rhs_n<ND, 5>(L);
    case 5: return gauss_rhs_n<ND, 6>(L);
    case 6: return gauss_rhs_n<ND, 7>(L);
    case 7: return gauss_rhs_n<ND, 8>(L);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_gauss(const GaussLaunch& L) {
  if (L.md.E <= 0) return cudaSuccess;
  return L.nd == 2 ? gauss_rhs_nd<2>(L) : gauss_rhs_nd<3>(L);
}

}  // namespace dgk
