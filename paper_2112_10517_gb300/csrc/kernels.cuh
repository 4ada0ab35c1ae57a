// Device code of the RHS: primitive variables, logarithmic means, Ranocha's two-point flux and the kernel
// templates. Included by the translation units that instantiate the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_internal.h"

namespace dgk {

// ---------------------------------------------------------------------------------------------------
// Precision traits
// ---------------------------------------------------------------------------------------------------
template <typename T>
struct Num;

template <>
struct Num<double> {
  __device__ static __forceinline__ double rcp(double x) { return __drcp_rn(x); }
  __device__ static __forceinline__ double log(double x) { return ::log(x); }
  __device__ static __forceinline__ double sqrt(double x) { return ::sqrt(x); }
  __device__ static __forceinline__ double abs(double x) { return ::fabs(x); }
  // threshold of the series branch of Algorithms 2 and 3 (Sec. 3.1; the value stated for 64-bit floats)
  static constexpr double kLogMeanEps = 1e-4;
};

template <>
struct Num<float> {
  __device__ static __forceinline__ float rcp(float x) { return __frcp_rn(x); }
  __device__ static __forceinline__ float log(float x) { return ::logf(x); }
  __device__ static __forceinline__ float sqrt(float x) { return ::sqrtf(x); }
  __device__ static __forceinline__ float abs(float x) { return ::fabsf(x); }
  // The paper states the threshold for 64-bit floats only. In FP32 the truncated series is accurate to
  // about 0.03 u^4 relative, and the log branch loses about eps32/(2 sqrt(u)): 1e-2 keeps both near 1 ulp.
  static constexpr float kLogMeanEps = 1e-2f;
};

// ---------------------------------------------------------------------------------------------------
// Logarithmic means (Sec. 3.1). With s = a+b and f = (b-a)/s, u = f^2 is the quantity of Algorithms 2 and 3
// (their numerator and denominator are (b-a)^2 and (b+a)^2); it is formed here from one reciprocal 1/s,
// which the series branches reuse. The series of Algorithm 2 uses the polynomial form of 1/log given in
// Sec. 3.1 (multiplication instead of division); the series of Algorithm 3 is used as printed.
// ---------------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ln_mean(T a, T b) {
  const T s = a + b, d = b - a;
  const T r = Num<T>::rcp(s);
  const T f = d * r;
  const T u = f * f;
  if (u < T(Num<T>::kLogMeanEps))
    return s * (T(0.5) + u * (T(-1.0 / 6.0) + u * (T(-2.0 / 45.0) + u * T(-22.0 / 945.0))));
  return d / Num<T>::log(b / a);
}

template <typename T>
__device__ __forceinline__ T inv_ln_mean(T a, T b) {
  const T s = a + b, d = b - a;
  const T r = Num<T>::rcp(s);
  const T f = d * r;
  const T u = f * f;
  if (u < T(Num<T>::kLogMeanEps)) return r * (T(2.0) + u * (T(2.0 / 3.0) + u * (T(2.0 / 5.0) + u * T(2.0 / 7.0))));
  return Num<T>::log(b / a) / d;
}

// ---------------------------------------------------------------------------------------------------
// Primitive variables (Sec. 7.1: computed once per node, not once per pair). P = (rho, v_1..v_d, p).
// Returns false for rho <= 0, p <= 0 or NaN.
// ---------------------------------------------------------------------------------------------------
template <int ND, typename T>
__device__ __forceinline__ bool cons_to_prim(const double* uc, T gm1, T* P) {
  const T rho = (T)uc[0];
  const T ir = Num<T>::rcp(rho);
  T ke = T(0);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const T m = (T)uc[1 + j];
    const T v = m * ir;
    P[1 + j] = v;
    ke += m * v;
  }
  const T p = gm1 * ((T)uc[ND + 1] - T(0.5) * ke);
  P[0] = rho;
  P[ND + 1] = p;
  return rho > T(0) && p > T(0);
}

// ---------------------------------------------------------------------------------------------------
// Ranocha's EC/KEP/PEP flux in directional form (Sec. 3.2, Eq. flux_ranocha) for a direction n of any length
// (the flux is linear in n; Sec. 2.3 uses the averaged contravariant vector). 1/{{rho/p}}_log is evaluated as
// p_a p_b / {{rho_a p_b, rho_b p_a}}_log (division-free rewrite of Sec. 3.2) and 1/(gamma-1) is a factor.
//   f_rho  = {{rho}}_log {{v.n}}
//   f_rhov = f_rho {{v}} + {{p}} n
//   f_rhoe = f_rho (v_a.v_b/2 + 1/({{rho/p}}_log (gamma-1))) + ((p; v.n))
// ---------------------------------------------------------------------------------------------------
template <int ND, typename T>
__device__ __forceinline__ void ranocha_flux(const T* a, const T* b, const T* n, T inv_gm1, T* f) {
  T vna = a[1] * n[0], vnb = b[1] * n[0], vv = a[1] * b[1];
#pragma unroll
  for (int j = 1; j < ND; ++j) {
    vna += a[1 + j] * n[j];
    vnb += b[1 + j] * n[j];
    vv += a[1 + j] * b[1 + j];
  }
  const T pa = a[ND + 1], pb = b[ND + 1];
  const T rho_mean = ln_mean<T>(a[0], b[0]);
  const T inv_rho_p_mean = pa * pb * inv_ln_mean<T>(a[0] * pb, b[0] * pa);
  const T p_avg = T(0.5) * (pa + pb);
  const T f_rho = rho_mean * T(0.5) * (vna + vnb);
  f[0] = f_rho;
#pragma unroll
  for (int j = 0; j < ND; ++j) f[1 + j] = f_rho * T(0.5) * (a[1 + j] + b[1 + j]) + p_avg * n[j];
  f[ND + 1] = f_rho * (T(0.5) * vv + inv_rho_p_mean * inv_gm1) + T(0.5) * (pa * vnb + pb * vna);
}

// ---------------------------------------------------------------------------------------------------
// Geometry of an element: N nodes per line, NL = N^(ND-1) lines per direction, NDOF = N^ND nodes.
// Node index i = i1 + N i2 + N^2 i3. Direction n has stride N^n. A line along n is identified by the index
// l in [0, NL) of its remaining coordinates (in increasing direction order); so is a face node on a face
// normal to n.
// ---------------------------------------------------------------------------------------------------
template <int ND, int N>
struct Geo {
  static constexpr int NL = (ND == 3) ? N * N : N;
  static constexpr int NDOF = NL * N;
  static constexpr int NV = ND + 2;
  static constexpr int TPE = ND * NL;  // threads per element in the pair phase: one per (direction, line)

  __device__ static __forceinline__ int stride(int n) { return n == 0 ? 1 : (n == 1 ? N : N * N); }
  // first node of line l along direction n (node index with i_n = 0)
  __device__ static __forceinline__ int line_base(int n, int l) {
    if (ND == 2) return n == 0 ? l * N : l;
    return n == 0 ? l * N : (n == 1 ? (l % N) + (l / N) * N * N : l);
  }
  // face-node index of node i on a face normal to n
  __device__ static __forceinline__ int face_index(int n, int i) {
    if (ND == 2) return n == 0 ? i / N : i % N;
    return n == 0 ? i / N : (n == 1 ? (i % N) + N * (i / (N * N)) : i % (N * N));
  }
};

// element neighbour across direction n (dir = +1 or -1), periodic
__device__ __forceinline__ int neighbor(const MeshDims& md, int e, int n, int dir) {
  int e1 = e % md.n1, t = e / md.n1, e2 = t % md.n2, e3 = t / md.n2;
  if (n == 0) e1 = (e1 + dir + md.n1) % md.n1;
  if (n == 1) e2 = (e2 + dir + md.n2) % md.n2;
  if (n == 2) e3 = (e3 + dir + md.n3) % md.n3;
  return e1 + md.n1 * (e2 + md.n2 * e3);
}

template <int N, typename T>
struct OpTable {
  T Dt[N * N];  // flux-differencing matrix 2D - M^{-1}B (Eq. opDsplit)
  T winv;       // 1/w_0 = 1/w_p = p(p+1)/2: the lift M^{-1} R^T B at the end nodes
};

// ---------------------------------------------------------------------------------------------------
// Interface flux (Sec. 2.4: one surface flux per interface node, shared by both elements).
// Thread per (direction n, lower element e, face node fn). The upper neighbour across +n is e+.
// f* = f_Ranocha(u_L, u_R, m) - [llf] lambda/2 (u_R - u_L), m = Ja^n at the lower element's face node,
// lambda = max(|v_L.m| + c_L|m|, |v_R.m| + c_R|m|), c = sqrt(gamma p/rho).
// face layout [n][E][NV][NL].
// ---------------------------------------------------------------------------------------------------
template <int ND, int N, typename T, bool LLF>
__global__ void __launch_bounds__(256) interface_kernel(const double* __restrict__ u, const T* __restrict__ Ja,
                                                        T* __restrict__ face, MeshDims md, T gamma, int* flag) {
  using G = Geo<ND, N>;
  const long long total = (long long)ND * md.E * G::NL;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int fn = (int)(idx % G::NL);
  const long long t = idx / G::NL;
  const int e = (int)(t % md.E);
  const int n = (int)(t / md.E);
  const int eR = neighbor(md, e, n, +1);
  // node with i_n = N-1 (lower element) and i_n = 0 (upper element) for face node fn
  const int st = G::stride(n);
  const int lo = fn % st, hi = fn / st;
  const int nodeL = lo + (N - 1) * st + hi * st * N;
  const int nodeR = lo + hi * st * N;
  double uL[G::NV], uR[G::NV];
#pragma unroll
  for (int c = 0; c < G::NV; ++c) {
    uL[c] = u[((size_t)e * G::NV + c) * G::NDOF + nodeL];
    uR[c] = u[((size_t)eR * G::NV + c) * G::NDOF + nodeR];
  }
  T m[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) m[j] = Ja[(((size_t)e * ND + n) * ND + j) * G::NDOF + nodeL];
  const T gm1 = gamma - T(1);
  T PL[G::NV], PR[G::NV], f[G::NV];
  const bool ok = cons_to_prim<ND, T>(uL, gm1, PL) & cons_to_prim<ND, T>(uR, gm1, PR);
  if (!ok) atomicOr(flag, 1);
  ranocha_flux<ND, T>(PL, PR, m, T(1) / gm1, f);
  if (LLF) {
    T mm = m[0] * m[0], vnL = PL[1] * m[0], vnR = PR[1] * m[0];
#pragma unroll
    for (int j = 1; j < ND; ++j) {
      mm += m[j] * m[j];
      vnL += PL[1 + j] * m[j];
      vnR += PR[1 + j] * m[j];
    }
    const T mn = Num<T>::sqrt(mm);
    const T lamL = Num<T>::abs(vnL) + Num<T>::sqrt(gamma * PL[ND + 1] / PL[0]) * mn;
    const T lamR = Num<T>::abs(vnR) + Num<T>::sqrt(gamma * PR[ND + 1] / PR[0]) * mn;
    const T half_lam = T(0.5) * (lamL > lamR ? lamL : lamR);
#pragma unroll
    for (int c = 0; c < G::NV; ++c) f[c] -= half_lam * (T)(uR[c] - uL[c]);
  }
  T* fo = face + ((size_t)n * md.E + e) * G::NV * G::NL + fn;
#pragma unroll
  for (int c = 0; c < G::NV; ++c) fo[c * G::NL] = f[c];
}

// ---------------------------------------------------------------------------------------------------
// Volume term + surface lift + Jacobian scaling (Eq. fluxdiff-SBP-opDsplit with Eq. curvilinear-rearrange):
//   du_i = -(1/J_i) [ sum_n sum_{k on i's line along n} Dt_{i_n k_n} f(u_i, u_k, (Ja^n_i + Ja^n_k)/2)
//                   + sum_n ([i_n = p] f*_up - [i_n = 0] f*_down) / w_0 ].
// Each CTA handles EPB elements.
//   A. stage primitive variables and metric terms of the elements in shared memory (coalesced loads);
//   B. one thread per (element, direction n, line): every pair i < k of the line is evaluated ONCE
//      (Sec. 2.2: Dt has zero diagonal and M Dt is skew-symmetric; f is symmetric) and added to both nodes
//      with Dt_ik and Dt_ki; the line's sums stay in registers and go to shared memory per direction;
//   C. one thread per node: sum the directions, add the lifted interface fluxes, scale by -1/J, store.
// ---------------------------------------------------------------------------------------------------
template <int ND, int N, typename T>
struct VolumeSmem {
  using G = Geo<ND, N>;
  static constexpr int kPrim = G::NV * G::NDOF;            // per element
  static constexpr int kJa = ND * ND * G::NDOF;            // per element
  static constexpr int kAcc = ND * G::NV * G::NDOF;        // per element
  static constexpr int kPerElem = kPrim + kJa + kAcc;      // elements of T
  static constexpr size_t bytes(int epb) { return (size_t)epb * kPerElem * sizeof(T); }
};

template <int ND, int N, typename T, int EPB>
__global__ void __launch_bounds__(EPB* Geo<ND, N>::TPE)
    volume_kernel(const double* __restrict__ u, const T* __restrict__ Ja, const double* __restrict__ invJ,
                  const T* __restrict__ face, double* __restrict__ du, MeshDims md, OpTable<N, T> op, T gamma,
                  int* flag) {
  using G = Geo<ND, N>;
  using S = VolumeSmem<ND, N, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_prim = reinterpret_cast<T*>(smem_raw);  // [EPB][NV][NDOF]
  T* s_ja = s_prim + EPB * S::kPrim;           // [EPB][ND][ND][NDOF]
  T* s_acc = s_ja + EPB * S::kJa;              // [EPB][ND][NV][NDOF]
  const int tid = threadIdx.x;
  constexpr int kThreads = EPB * G::TPE;
  const int e0 = blockIdx.x * EPB;
  const int nel = min(EPB, md.E - e0);
  const T gm1 = gamma - T(1);

  // ---- A: primitives and metric terms -> shared memory
  bool ok = true;
  for (int idx = tid; idx < nel * G::NDOF; idx += kThreads) {
    const int el = idx / G::NDOF, i = idx - el * G::NDOF;
    const double* ue = u + (size_t)(e0 + el) * G::NV * G::NDOF + i;
    double uc[G::NV];
#pragma unroll
    for (int c = 0; c < G::NV; ++c) uc[c] = ue[c * G::NDOF];
    T P[G::NV];
    ok &= cons_to_prim<ND, T>(uc, gm1, P);
#pragma unroll
    for (int c = 0; c < G::NV; ++c) s_prim[(el * G::NV + c) * G::NDOF + i] = P[c];
  }
  if (!ok) atomicOr(flag, 1);
  {
    const T* jae = Ja + (size_t)e0 * S::kJa;
    for (int idx = tid; idx < nel * S::kJa; idx += kThreads) s_ja[idx] = jae[idx];
  }
  __syncthreads();

  // ---- B: pairs along lines
  if (tid < nel * G::TPE) {
    const int el = tid / G::TPE, r = tid - el * G::TPE;
    const int n = r / G::NL, l = r - n * G::NL;
    const int st = G::stride(n), base = G::line_base(n, l);
    const T* sp = s_prim + el * S::kPrim + base;
    const T* sj = s_ja + (el * ND + n) * ND * G::NDOF + base;
    const T inv_gm1 = T(1) / gm1;
    T acc[N][G::NV];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int c = 0; c < G::NV; ++c) acc[i][c] = T(0);
#pragma unroll
    for (int i = 0; i < N - 1; ++i) {
      T a[G::NV], ja_i[ND];
#pragma unroll
      for (int c = 0; c < G::NV; ++c) a[c] = sp[c * G::NDOF + i * st];
#pragma unroll
      for (int j = 0; j < ND; ++j) ja_i[j] = sj[j * G::NDOF + i * st];
#pragma unroll
      for (int k = i + 1; k < N; ++k) {
        T b[G::NV], nrm[ND], f[G::NV];
#pragma unroll
        for (int c = 0; c < G::NV; ++c) b[c] = sp[c * G::NDOF + k * st];
#pragma unroll
        for (int j = 0; j < ND; ++j) nrm[j] = T(0.5) * (ja_i[j] + sj[j * G::NDOF + k * st]);
        ranocha_flux<ND, T>(a, b, nrm, inv_gm1, f);
        const T dik = op.Dt[i * N + k], dki = op.Dt[k * N + i];
#pragma unroll
        for (int c = 0; c < G::NV; ++c) {
          acc[i][c] += dik * f[c];
          acc[k][c] += dki * f[c];
        }
      }
    }
    T* sa = s_acc + (el * ND + n) * G::NV * G::NDOF + base;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int c = 0; c < G::NV; ++c) sa[c * G::NDOF + i * st] = acc[i][c];
  }
  __syncthreads();

  // ---- C: sum directions, lift interface fluxes, scale by -1/J
  for (int idx = tid; idx < nel * G::NDOF; idx += kThreads) {
    const int el = idx / G::NDOF, i = idx - el * G::NDOF;
    const int ge = e0 + el;
    T tot[G::NV];
#pragma unroll
    for (int c = 0; c < G::NV; ++c) {
      T s = T(0);
#pragma unroll
      for (int n = 0; n < ND; ++n) s += s_acc[((el * ND + n) * G::NV + c) * G::NDOF + i];
      tot[c] = s;
    }
#pragma unroll
    for (int n = 0; n < ND; ++n) {
      const int in = (i / G::stride(n)) % N;
      if (in == N - 1 || in == 0) {
        const int fn = G::face_index(n, i);
        const int fe = in == N - 1 ? ge : neighbor(md, ge, n, -1);
        const T sgn = in == N - 1 ? op.winv : -op.winv;
        const T* fp = face + ((size_t)n * md.E + fe) * G::NV * G::NL + fn;
#pragma unroll
        for (int c = 0; c < G::NV; ++c) tot[c] += sgn * fp[c * G::NL];
      }
    }
    const double sj = -invJ[(size_t)ge * G::NDOF + i];
    double* d = du + (size_t)ge * G::NV * G::NDOF + i;
#pragma unroll
    for (int c = 0; c < G::NV; ++c) d[c * G::NDOF] = sj * (double)tot[c];
  }
}

}  // namespace dgk
