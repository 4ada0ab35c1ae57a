// Vector-Jacobian product of the RHS: ubar = (d RHS/du)^T gbar (FP64), the adjoint of dg_rhs.
//
// The RHS is du_i = -(1/J_i) tot_i with tot_i = sum over pairs Dt8_ik F(q_i, q_k, n2_ik) + lifted interface
// fluxes (Eq. fluxdiff-SBP-opDsplit). Its adjoint runs the same structure backwards:
//   tbar_i = -gbar_i / J_i                               (adjoint of tot at every node)
//   interface kernel: fbar* = winv (tbar at the lower element's face node - tbar at the upper element's),
//     back through the LLF dissipation, Ranocha's flux and the node quantities of both states; the two u-space
//     contributions go to a face buffer (no write conflicts);
//   volume kernel: per pair Fbar = Dt8_ik tbar_i + Dt8_ki tbar_k, back through the flux to the node quantities
//     of i and k (accumulated per line in registers, summed over directions in shared memory), then back
//     through the node quantities to u, plus the face contributions of the element's face nodes.
#include <new>

#include "kernels.cuh"

namespace dgk {
namespace {

// face adjoint buffer layout: [n][E][side][NV][NL], side 0 = lower element (face node i_n = N-1),
// side 1 = upper element (face node i_n = 0)
template <int ND, int N, bool LLF>
__global__ void __launch_bounds__(256) interface_vjp_kernel(const double* __restrict__ u, const double* __restrict__ Ja,
                                                            const double* __restrict__ invJ,
                                                            const double* __restrict__ gbar,
                                                            double* __restrict__ fadj, MeshDims md, double gamma) {
  using G = Geo<ND, N>;
  using Q = NodeQ<ND>;
  const long long total = (long long)ND * md.E * G::NL;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int fn = (int)(idx % G::NL);
  const long long t = idx / G::NL;
  const int e = (int)(t % md.E);
  const int n = (int)(t / md.E);
  const int eR = neighbor(md, e, n, +1);
  const int st = G::stride(n);
  const int lo = fn % st, hi = fn / st;
  const int nodeL = lo + (N - 1) * st + hi * st * N;
  const int nodeR = lo + hi * st * N;
  double uL[G::NV], uR[G::NV], fb[G::NV];
  const double winv = 0.5 * (N - 1) * N;  // 1/w_0 = p(p+1)/2
  const double sL = -invJ[(size_t)e * G::NDOF + nodeL], sR = -invJ[(size_t)eR * G::NDOF + nodeR];
#pragma unroll
  for (int c = 0; c < G::NV; ++c) {
    uL[c] = u[((size_t)e * G::NV + c) * G::NDOF + nodeL];
    uR[c] = u[((size_t)eR * G::NV + c) * G::NDOF + nodeR];
    // f* enters tot of the lower element with +winv and of the upper element with -winv
    fb[c] = winv * (sL * gbar[((size_t)e * G::NV + c) * G::NDOF + nodeL] -
                    sR * gbar[((size_t)eR * G::NV + c) * G::NDOF + nodeR]);
  }
  double m[ND], m2[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    m[j] = Ja[(((size_t)e * ND + n) * ND + j) * G::NDOF + nodeL];
    m2[j] = m[j] + m[j];
  }
  const double gm1 = gamma - 1.0, tg = 2.0 / gm1;
  double qL[Q::NQ], qR[Q::NQ], qLb[Q::NQ], qRb[Q::NQ], uLb[G::NV], uRb[G::NV], Fb[G::NV];
  node_quantities<ND, double>(uL, gm1, tg, qL);
  node_quantities<ND, double>(uR, gm1, tg, qR);
#pragma unroll
  for (int c = 0; c < Q::NQ; ++c) qLb[c] = qRb[c] = 0.0;
#pragma unroll
  for (int c = 0; c < G::NV; ++c) {
    Fb[c] = 0.125 * fb[c];  // f* = F/8 - ...
    uLb[c] = uRb[c] = 0.0;
  }
  if (LLF) {
    double mm = m[0] * m[0], vnL = qL[1] * m[0], vnR = qR[1] * m[0];
#pragma unroll
    for (int j = 1; j < ND; ++j) {
      mm += m[j] * m[j];
      vnL += qL[1 + j] * m[j];
      vnR += qR[1 + j] * m[j];
    }
    const double hg = 0.5 * gamma;
    const double mn = sqrt(mm);
    const double wL = hg * qL[Q::PP] / qL[0], wR = hg * qR[Q::PP] / qR[0];
    const double cL = sqrt(wL), cR = sqrt(wR);
    const double lamL = fabs(vnL) + cL * mn, lamR = fabs(vnR) + cR * mn;
    const bool pickL = lamL > lamR;  // the forward kernel keeps lamR at ties
    const double half_lam = 0.5 * (pickL ? lamL : lamR);
    double lamb = 0.0;
#pragma unroll
    for (int c = 0; c < G::NV; ++c) {  // f*_c -= half_lam (uR_c - uL_c)
      uLb[c] += half_lam * fb[c];
      uRb[c] -= half_lam * fb[c];
      lamb -= 0.5 * fb[c] * (uR[c] - uL[c]);
    }
    // lambda_X = |vn_X| + c_X |m|, c_X = sqrt(w_X), w_X = hg pp_X / rho_X, vn_X = v_X . m
    const double vn = pickL ? vnL : vnR, cx = pickL ? cL : cR, w = pickL ? wL : wR;
    double* qb = pickL ? qLb : qRb;
    const double* qx = pickL ? qL : qR;
    const double vnb = lamb * (vn < 0.0 ? -1.0 : 1.0);
    const double wb = lamb * mn / (2.0 * cx);
    qb[Q::PP] += wb * hg / qx[0];
    qb[0] -= wb * w / qx[0];
#pragma unroll
    for (int j = 0; j < ND; ++j) qb[1 + j] += vnb * m[j];
  }
  ranocha_flux8_adjoint<ND, double>(qL, qR, m2, Fb, qLb, qRb);
  double ua[G::NV], ub[G::NV];
  node_quantities_adjoint<ND, double>(uL, gm1, tg, qLb, ua);
  node_quantities_adjoint<ND, double>(uR, gm1, tg, qRb, ub);
  double* fo = fadj + ((size_t)n * md.E + e) * 2 * G::NV * G::NL + fn;
#pragma unroll
  for (int c = 0; c < G::NV; ++c) {
    fo[c * G::NL] = ua[c] + uLb[c];
    fo[(G::NV + c) * G::NL] = ub[c] + uRb[c];
  }
}

template <int ND, int N>
struct VjpSmem {
  using G = Geo<ND, N>;
  static constexpr int kQ = NodeQ<ND>::NQ * G::NDOF;
  static constexpr int kJa = ND * ND * G::NDOF;
  static constexpr int kT = G::NV * G::NDOF;
  static constexpr int kQb = ND * NodeQ<ND>::NQ * G::NDOF;
  static constexpr size_t bytes(int epb) { return (size_t)epb * (kQ + kJa + kT + kQb) * sizeof(double); }
};

template <int ND, int N, int EPB>
__global__ void __launch_bounds__(EPB* Geo<ND, N>::TPE)
    volume_vjp_kernel(const double* __restrict__ u, const double* __restrict__ Ja, const double* __restrict__ invJ,
                      const double* __restrict__ gbar, const double* __restrict__ fadj, double* __restrict__ ubar,
                      MeshDims md, OpTable<N, double> op, double gamma) {
  using G = Geo<ND, N>;
  using Q = NodeQ<ND>;
  using S = VjpSmem<ND, N>;
  constexpr int NQ = Q::NQ;
  constexpr int kThreads = EPB * G::TPE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_q = reinterpret_cast<double*>(smem_raw);  // [EPB][NQ][NDOF]
  double* s_ja = s_q + EPB * S::kQ;                    // [EPB][ND][ND][NDOF]
  double* s_t = s_ja + EPB * S::kJa;                   // [EPB][NV][NDOF]  tbar = -gbar/J
  double* s_qb = s_t + EPB * S::kT;                    // [EPB][ND][NQ][NDOF] qbar per direction
  const int tid = threadIdx.x;
  const int e0 = blockIdx.x * EPB;
  const int nel = min(EPB, md.E - e0);
  const double gm1 = gamma - 1.0, tg = 2.0 / gm1;

  for (int idx = tid; idx < nel * G::NDOF; idx += kThreads) {
    const int el = idx / G::NDOF, i = idx - el * G::NDOF;
    const size_t base = (size_t)(e0 + el) * G::NV * G::NDOF + i;
    double uc[G::NV], q[NQ];
#pragma unroll
    for (int c = 0; c < G::NV; ++c) uc[c] = u[base + c * G::NDOF];
    node_quantities<ND, double>(uc, gm1, tg, q);
#pragma unroll
    for (int c = 0; c < NQ; ++c) s_q[(el * NQ + c) * G::NDOF + i] = q[c];
    const double sj = -invJ[(size_t)(e0 + el) * G::NDOF + i];
#pragma unroll
    for (int c = 0; c < G::NV; ++c) s_t[(el * G::NV + c) * G::NDOF + i] = sj * gbar[base + c * G::NDOF];
  }
  {
    const double* jae = Ja + (size_t)e0 * S::kJa;
    for (int idx = tid; idx < nel * S::kJa; idx += kThreads) s_ja[idx] = jae[idx];
  }
  __syncthreads();

  if (tid < nel * G::TPE) {
    const int el = tid / G::TPE, r = tid - el * G::TPE;
    const int n = r / G::NL, l = r - n * G::NL;
    const int st = G::stride(n), base = G::line_base(n, l);
    const double* sq = s_q + el * S::kQ + base;
    const double* sj = s_ja + (el * ND + n) * ND * G::NDOF + base;
    const double* stb = s_t + el * S::kT + base;
    double qb[N][NQ];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int c = 0; c < NQ; ++c) qb[i][c] = 0.0;
#pragma unroll
    for (int i = 0; i < N - 1; ++i) {
      double a[NQ], ja_i[ND], ti[G::NV];
#pragma unroll
      for (int c = 0; c < NQ; ++c) a[c] = sq[c * G::NDOF + i * st];
#pragma unroll
      for (int j = 0; j < ND; ++j) ja_i[j] = sj[j * G::NDOF + i * st];
#pragma unroll
      for (int c = 0; c < G::NV; ++c) ti[c] = stb[c * G::NDOF + i * st];
#pragma unroll
      for (int k = i + 1; k < N; ++k) {
        double b[NQ], n2[ND], Fb[G::NV];
#pragma unroll
        for (int c = 0; c < NQ; ++c) b[c] = sq[c * G::NDOF + k * st];
#pragma unroll
        for (int j = 0; j < ND; ++j) n2[j] = ja_i[j] + sj[j * G::NDOF + k * st];
        const double dik = op.Dt8[i * N + k], dki = op.Dt8[k * N + i];
#pragma unroll
        for (int c = 0; c < G::NV; ++c) Fb[c] = dik * ti[c] + dki * stb[c * G::NDOF + k * st];
        ranocha_flux8_adjoint<ND, double>(a, b, n2, Fb, qb[i], qb[k]);
      }
    }
    double* sqb = s_qb + (el * ND + n) * NQ * G::NDOF + base;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int c = 0; c < NQ; ++c) sqb[c * G::NDOF + i * st] = qb[i][c];
  }
  __syncthreads();

  for (int idx = tid; idx < nel * G::NDOF; idx += kThreads) {
    const int el = idx / G::NDOF, i = idx - el * G::NDOF;
    const int ge = e0 + el;
    const size_t base = (size_t)ge * G::NV * G::NDOF + i;
    double qbs[NQ], uc[G::NV], ub[G::NV];
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
      double s = 0.0;
#pragma unroll
      for (int n = 0; n < ND; ++n) s += s_qb[((el * ND + n) * NQ + c) * G::NDOF + i];
      qbs[c] = s;
    }
#pragma unroll
    for (int c = 0; c < G::NV; ++c) uc[c] = u[base + c * G::NDOF];
    node_quantities_adjoint<ND, double>(uc, gm1, tg, qbs, ub);
#pragma unroll
    for (int n = 0; n < ND; ++n) {
      const int in = (i / G::stride(n)) % N;
      if (in == N - 1 || in == 0) {
        const int fn = G::face_index(n, i);
        const int fe = in == N - 1 ? ge : neighbor(md, ge, n, -1);
        const int side = in == N - 1 ? 0 : 1;
        const double* fp = fadj + (((size_t)n * md.E + fe) * 2 + side) * G::NV * G::NL + fn;
#pragma unroll
        for (int c = 0; c < G::NV; ++c) ub[c] += fp[c * G::NL];
      }
    }
#pragma unroll
    for (int c = 0; c < G::NV; ++c) ubar[base + c * G::NDOF] = ub[c];
  }
}

template <int ND, int N>
constexpr int vjp_epb() {
  return Geo<ND, N>::TPE >= 192 ? 1 : 192 / Geo<ND, N>::TPE;
}

template <int ND, int N>
cudaError_t launch_vjp_t(int llf, MeshDims md, const double* u, const double* Ja, const double* invJ,
                         const double* gbar, double* fadj, double* ubar, double gamma, cudaStream_t s) {
  using G = Geo<ND, N>;
  const long long total = (long long)ND * md.E * G::NL;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (llf)
    interface_vjp_kernel<ND, N, true><<<blocks, 256, 0, s>>>(u, Ja, invJ, gbar, fadj, md, gamma);
  else
    interface_vjp_kernel<ND, N, false><<<blocks, 256, 0, s>>>(u, Ja, invJ, gbar, fadj, md, gamma);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  constexpr int EPB = vjp_epb<ND, N>();
  const size_t smem = VjpSmem<ND, N>::bytes(EPB);
  auto kern = volume_vjp_kernel<ND, N, EPB>;
  static PerDeviceCache cache;  // the shared-memory opt-in, once per device
  long long done = 0;
  e = per_device(cache, &done, [&](long long* v) {
    *v = 1;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  OpTable<N, double> op;
  const RefTables& t = ref_tables(N - 1);
  for (int i = 0; i < N * N; ++i) {
    op.Dt8[i] = 0.125 * t.Dt[i];
    op.D0[i] = 0.25 * t.Dt[i];
  }
  op.winv = 1.0 / t.w[0];
  op.lift8 = 0.125 / t.w[0];
  kern<<<(md.E + EPB - 1) / EPB, EPB * G::TPE, smem, s>>>(u, Ja, invJ, gbar, fadj, ubar, md, op, gamma);
  return cudaGetLastError();
}

template <int ND>
cudaError_t dispatch_vjp(int p, int llf, MeshDims md, const double* u, const double* Ja, const double* invJ,
                         const double* gbar, double* fadj, double* ubar, double gamma, cudaStream_t s) {
  switch (p) {
    case 1: return launch_vjp_t<ND, 2>(llf, md, u, Ja, invJ, gbar, fadj, ubar, gamma, s);
    case 2: return launch_vjp_t<ND, 3>(llf, md, u, Ja, invJ, gbar, fadj, ubar, gamma, s);
    case 3: return launch_vjp_t<ND, 4>(llf, md, u, Ja, invJ, gbar, fadj, ubar, gamma, s);
    case 4: return launch_vjp_t<ND, 5>(llf, md, u, Ja, invJ, gbar, fadj, ubar, gamma, s);
    case 5: return launch_vjp_t<ND, 6>(llf, md, u, Ja, invJ, gbar, fadj, ubar, gamma, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace dgk

extern "C" dg_status dg_vjp(dg_ctx* c, const double* u, const double* gbar, double* ubar, dg_stream_t stream) {
  if (!c || !u || !gbar || !ubar) return DG_ERR_ARG;
  if (c->precision != DG_FP64 || c->p > 5 || c->volume_flux != DG_VOL_RANOCHA ||
      c->var.lm != 0 || c->nodes != DG_NODES_LGL || c->layer != 0)
    return DG_ERR_UNSUPPORTED;
  if (((uintptr_t)u | (uintptr_t)gbar | (uintptr_t)ubar) & 7) return DG_ERR_ARG;
  const size_t bytes = (size_t)c->state_len * sizeof(double);
  const char* ob = (const char*)ubar;
  const char* in[2] = {(const char*)u, (const char*)gbar};
  for (const char* ib : in)
    if (ib < ob + bytes && ob < ib + bytes) return DG_ERR_ARG;  // ubar overlaps an input
  if (!c->d_fadj) {
    const size_t n = (size_t)c->nd * c->E * 2 * c->nv * (c->nd == 3 ? c->N * c->N : c->N);
    cudaError_t e = cudaMalloc(&c->d_fadj, n * sizeof(double));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  c->launches += 2;
  const int llf = c->surface_flux == DG_SURF_EC_LLF;
  cudaError_t e = c->nd == 3 ? dgk::dispatch_vjp<3>(c->p, llf, c->md, u, c->d_Ja, c->d_invJ, gbar, c->d_fadj, ubar,
                                                    c->gamma, s)
                             : dgk::dispatch_vjp<2>(c->p, llf, c->md, u, c->d_Ja, c->d_invJ, gbar, c->d_fadj, ubar,
                                                    c->gamma, s);
  return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}
