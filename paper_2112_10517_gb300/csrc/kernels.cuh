// Device code of the RHS: primitive variables, logarithmic means, Ranocha's two-point flux and the kernel
// templates. Included by the translation units that instantiate the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_internal.h"
#include "dgmath.cuh"

namespace dgk {

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

// Ja^n_n of a Cartesian mesh for direction n (selects, no dynamic indexing of the parameter struct)
__device__ __forceinline__ double cart_jn(const Variant& v, int n) { return n == 0 ? v.jn[0] : (n == 1 ? v.jn[1] : v.jn[2]); }

// element neighbour across direction n (dir = +1 or -1), periodic
__device__ __forceinline__ int neighbor(const MeshDims& md, int e, int n, int dir) {
  int e1 = e % md.n1, t = e / md.n1, e2 = t % md.n2, e3 = t / md.n2;
  if (n == 0) e1 = (e1 + dir + md.n1) % md.n1;
  if (n == 1) e2 = (e2 + dir + md.n2) % md.n2;
  if (n == 2) e3 = (e3 + dir + md.n3) % md.n3;
  return e1 + md.n1 * (e2 + md.n2 * e3);
}

// upper neighbour of element e across direction n (periodic), with one or two divisions
__device__ __forceinline__ int upper_neighbor(const MeshDims& md, int e, int n) {
  if (n == 0) {
    const int e1 = e % md.n1;
    return e1 == md.n1 - 1 ? e - e1 : e + 1;
  }
  const int s = n == 1 ? md.n1 : md.n1 * md.n2;  // element stride along n
  const int c = n == 1 ? (e / md.n1) % md.n2 : e / s;  // coordinate along n
  const int len = n == 1 ? md.n2 : md.n3;
  return c == len - 1 ? e - c * s : e + s;
}

// Programmatic dependent launch (the kernels that a stream runs back to back may overlap): pdl_wait blocks until
// the kernels before this one in the stream have completed and their writes are visible (at once when the kernel
// was launched without the attribute); a kernel reads nothing those kernels write, and writes nothing, before it.
// A dependent grid is scheduled as the CTAs of the one before it exit (or signal, griddepcontrol.launch_dependents),
// and its CTAs set up and copy their first tile's geometry while that grid's writes are made visible. Only the FP64
// pipelined volume kernel signals early, at the start of each CTA's last tile, so that the next interface kernel's
// CTAs take the SMs its last round leaves idle (16^3 RK4 step -0.2 %, graph replay -0.4 %; 32^3 unchanged). The
// dependents still wait (pdl_wait) for the whole grid before reading its results. Other early signals measured
// slower: volume CTAs placed on SMs in the order the interface kernel freed them lose the round-robin balance of
// their tiles (16^3 FP64: +9 %), and interface CTAs resident during the FP32 volume kernel's last tiles slowed it
// (32^3 FP32: +7 %).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#ifndef DG_VOLUME_EARLY_TRIGGER
#define DG_VOLUME_EARLY_TRIGGER 1
#endif

// Launch of `kern`; with `overlap`, as a programmatic dependent of the kernel before it in stream s (the kernel
// calls pdl_wait before its first read of data written by the stream's earlier work).
template <typename... P, typename... A>
inline cudaError_t launch_kernel(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                 bool overlap, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = overlap ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

template <int N, typename T>
struct OpTable {
  T Dt8[N * N];  // flux-differencing matrix 2D - M^{-1}B (Eq. opDsplit), divided by 8 (fluxes come scaled by 8)
  T D0[N * N];   // 2 Dt8: the coefficients of the mass flux, which the volume sums take halved (exact)
  T winv;        // 1/w_0 = 1/w_p = p(p+1)/2: the lift M^{-1} R^T B at the end nodes
  T lift8;       // winv / 8 (the face buffer holds the interface fluxes already lifted: f* / w_0)
};

// ---------------------------------------------------------------------------------------------------
// Interface flux (Sec. 2.4: one surface flux per interface node, shared by both elements).
// Thread per (lower element e, direction n, face node fn). The upper neighbour across +n is e+.
// f* = f_Ranocha(u_L, u_R, m) - [llf] lambda/2 (u_R - u_L), m = Ja^n at the lower element's face node,
// lambda = max(|v_L.m| + c_L|m|, |v_R.m| + c_R|m|), c = sqrt(gamma p/rho).
// face layout [n][E][NV][NL], holding the lifted flux f* / w_0 (the surface term of the volume kernel: +f* / w_p
// at i_n = p, -f* / w_0 at i_n = 0, Eq. opDsplit). f* is linear in m (both the two-point flux and the LLF term are
// homogeneous of degree 1 in m), so the factor 1/w_0 = p(p+1)/2 rides on the metric vector at no cost.
// ---------------------------------------------------------------------------------------------------
// Interface flux at face node `idx` of a mesh, idx = (e * ND + n) * NL + fn: the faces on an element's upper side
// in all directions are neighbours in the launch, so the element's data are fetched once for them and its lower
// neighbours' visits follow closely. FLUX: 0 Ranocha, 1 Shima et al.
// cart: metric terms are the Cartesian constants of `var` (Ja is not read).
template <int ND, int N, typename T, bool LLF, int FLUX>
__device__ __forceinline__ void interface_node(const double* __restrict__ u, const T* __restrict__ Ja,
                                               T* __restrict__ face, const MeshDims& md, T gamma, int* flag,
                                               int idx, const Variant& var) {
  using G = Geo<ND, N>;
  const int fn = idx % G::NL;
  const int t = idx / G::NL;
  const int n = t % ND;
  const int e = t / ND;
  const int eR = upper_neighbor(md, e, n);
  // node with i_n = N-1 (lower element) and i_n = 0 (upper element) for face node fn
  const int st = G::stride(n);
  const int lo = fn % st, hi = fn / st;
  const int nodeL = lo + (N - 1) * st + hi * st * N;
  const int nodeR = lo + hi * st * N;
  // the pair flux takes 2 m and returns 8 f: with 2 m scaled by lift8 = N(N-1)/16 the result is f / w_0
  constexpr double kLift8 = N * (N - 1) / 16.0;
  T m[ND], m2[ND], gm2 = T(0);
  // FP64 curvilinear contexts: m2 and gamma |m2|^2 / 2 precomputed per interface node (Variant::fgeo)
  const bool pre = sizeof(T) == 8 && var.fgeo != nullptr;
  const T jn = var.cart ? to_flux<T>(cart_jn(var, n)) : T(0);  // (integer-pipe conversion in FP32 mode)
  if (pre) {
    const double* g = var.fgeo + (size_t)t * 4 * G::NL + fn;  // [E][ND][4][NL], t = e ND + n
#pragma unroll
    for (int j = 0; j < ND; ++j) m2[j] = (T)g[j * G::NL];
    gm2 = (T)g[3 * G::NL];
  } else {
#pragma unroll
    for (int j = 0; j < ND; ++j)  // the metric terms are written once, at set-up: read before the wait
      m[j] = var.cart ? (j == n ? jn : T(0)) : Ja[(((size_t)e * ND + n) * ND + j) * G::NDOF + nodeL];
  }
  pdl_wait();  // the state comes from the kernel before (a stage update)
  double uL[G::NV], uR[G::NV];
#pragma unroll
  for (int c = 0; c < G::NV; ++c) {
    uL[c] = u[((size_t)e * G::NV + c) * G::NDOF + nodeL];
    uR[c] = u[((size_t)eR * G::NV + c) * G::NDOF + nodeR];
  }
  if (!pre) {
#pragma unroll
    for (int j = 0; j < ND; ++j) m2[j] = m[j] * T(2.0 * kLift8);
  }
  const T gm1 = gamma - T(1);
  // the states in the flux precision, converted once (FP32 mode: also the LLF jump below); with a reference
  // pressure (FP32 mode) the energies relative to that of p_ref, so that their jump, and the pressure terms of the
  // momentum flux, carry the rounding of the small differences
  T uLt[G::NV], uRt[G::NV];
#pragma unroll
  for (int c = 0; c < G::NV - 1; ++c) {
    uLt[c] = to_flux<T>(uL[c]);
    uRt[c] = to_flux<T>(uR[c]);
  }
  uLt[G::NV - 1] = energy_rel<T>(uL[G::NV - 1], var.sh_eh, var.sh_el);
  uRt[G::NV - 1] = energy_rel<T>(uR[G::NV - 1], var.sh_eh, var.sh_el);
  const T pp0 = T(var.sh_pp);  // 2 p_ref (FP32 mode), else 0
  T qL[NodeQ<ND>::NQ], qR[NodeQ<ND>::NQ], f[G::NV], irL, irR;
  if constexpr (sizeof(T) == 8) {  // one reciprocal for both densities: 1/rho_L = rho_R R, R = 1/(rho_L rho_R)
    const T R = Num<T>::rcp(uLt[0] * uRt[0]);
    irL = uRt[0] * R;
    irR = uLt[0] * R;
  } else {
    irL = Num<T>::rcp(uLt[0]);
    irR = Num<T>::rcp(uRt[0]);
  }
  const bool ok = node_quantities_ir<ND, T>(uLt, irL, gm1, T(2) / gm1, qL, pp0) &
                  node_quantities_ir<ND, T>(uRt, irR, gm1, T(2) / gm1, qR, pp0);
  if (!ok) atomicOr(flag, 1);
  pair_flux8<ND, T, FLUX>(qL, qR, m2, f, LogRef<T>{nullptr, nullptr, 0}, pp0);  // f(u_L, u_R, m) / w_0
  if (LLF) {
    // with the precomputed geometry the speeds come out scaled like m2 (by p(p+1)/8), which the last factor undoes
    T vnL, vnR, hgm;
    if (pre) {
      vnL = qL[1] * m2[0];
      vnR = qR[1] * m2[0];
#pragma unroll
      for (int j = 1; j < ND; ++j) {
        vnL += qL[1 + j] * m2[j];
        vnR += qR[1 + j] * m2[j];
      }
      hgm = gm2;
    } else {
      T mm = m[0] * m[0];
      vnL = qL[1] * m[0];
      vnR = qR[1] * m[0];
#pragma unroll
      for (int j = 1; j < ND; ++j) {
        mm += m[j] * m[j];
        vnL += qL[1 + j] * m[j];
        vnR += qR[1 + j] * m[j];
      }
      hgm = T(0.5) * gamma * mm;
    }
    // c |m| = sqrt(gamma p |m|^2 / rho) with p = pp/2: one root per side (FP64: to about 46 bits, sqrt_wave_f64)
    const T aL = hgm * unshift_pp(qL[NodeQ<ND>::PP], pp0) * irL, aR = hgm * unshift_pp(qR[NodeQ<ND>::PP], pp0) * irR;
    T cL, cR;
    if constexpr (sizeof(T) == 8) {
      cL = sqrt_wave_f64(aL);
      cR = sqrt_wave_f64(aR);
    } else {
      cL = Num<T>::sqrt(aL);
      cR = Num<T>::sqrt(aR);
    }
    const T lamL = Num<T>::abs(vnL) + cL;
    const T lamR = Num<T>::abs(vnR) + cR;
    const T lmax = Num<T>::maxnn(lamL, lamR);
    const T lam4 = pre ? lmax + lmax : T(4.0 * kLift8) * lmax;  // (lambda / 2) / w_0
#pragma unroll
    for (int c = 0; c < G::NV; ++c) {
      // FP64: the jump in FP64; FP32 mode: both states rounded to FP32 first (no FP64 arithmetic)
      const T jump = uRt[c] - uLt[c];
      f[c] -= lam4 * jump;
    }
  }
  T* fo = face + ((size_t)n * md.E + e) * G::NV * G::NL + fn;
#pragma unroll
  for (int c = 0; c < G::NV; ++c) fo[c * G::NL] = f[c];
}

// The interface kernel's body: one face node per thread (see interface_node); kernels below by precision.
template <int ND, int N, typename T, bool LLF>
__device__ __forceinline__ void interface_items(const double* __restrict__ u, const T* __restrict__ Ja,
                                                T* __restrict__ face, const MeshDims& md, T gamma, int* flag,
                                                const Variant& var) {
  // the faces of elements [if_e0, if_e1) (all when if_e1 = 0; past E wrapping around to element 0);
  // ND E NL < 2^31 (checked at dg_init)
  const long long total = (long long)ND * md.E * Geo<ND, N>::NL;
  const long long end = (long long)ND * (var.if_e1 > 0 ? var.if_e1 : md.E) * Geo<ND, N>::NL;
  long long idx = (long long)ND * var.if_e0 * Geo<ND, N>::NL + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= end) return;
  if (idx >= total) idx -= total;
  if (var.ghost) {  // a partition's ghost layer: only its faces along the last direction (the lower boundary)
    const int t = (int)(idx / Geo<ND, N>::NL);
    if (t / ND < var.ghost && t % ND != ND - 1) return;
  }
  if (var.flux == 0)
    interface_node<ND, N, T, LLF, 0>(u, Ja, face, md, gamma, flag, (int)idx, var);
  else
    interface_node<ND, N, T, LLF, 1>(u, Ja, face, md, gamma, flag, (int)idx, var);
}

template <int ND, int N, typename T, bool LLF>
__global__ void __launch_bounds__(256) interface_kernel(const double* __restrict__ u, const T* __restrict__ Ja,
                                                        T* __restrict__ face, MeshDims md, T gamma, int* flag,
                                                        Variant var) {
  interface_items<ND, N, T, LLF>(u, Ja, face, md, gamma, flag, var);
}

// FP32: at most 40 registers (6 CTAs of 256 threads): 12 of the launcher's 128-thread CTAs fit per SM instead of
// 10 at 50 registers, for the memory-latency-bound kernel (32^3 launch 38.5 -> 37.8 us; 16^3 unchanged at 10.5 us,
// where the launch's fixed latency dominates)
#ifndef DG_INTERFACE_F32_MIN_BLOCKS
#define DG_INTERFACE_F32_MIN_BLOCKS 6
#endif
template <int ND, int N, bool LLF>
__global__ void __launch_bounds__(256, DG_INTERFACE_F32_MIN_BLOCKS)
    interface_kernel_f32(const double* __restrict__ u, const float* __restrict__ Ja, float* __restrict__ face,
                         MeshDims md, float gamma, int* flag, Variant var) {
  interface_items<ND, N, float, LLF>(u, Ja, face, md, gamma, flag, var);
}

// ---------------------------------------------------------------------------------------------------
// Volume term + surface lift + Jacobian scaling (Eq. fluxdiff-SBP-opDsplit with Eq. curvilinear-rearrange):
//   du_i = -(1/J_i) [ sum_n sum_{k on i's line along n} Dt_{i_n k_n} f(u_i, u_k, (Ja^n_i + Ja^n_k)/2)
//                   + sum_n ([i_n = p] f*_up - [i_n = 0] f*_down) / w_0 ].
// Each CTA handles EPB elements.
//   A. stage the node quantities (rho, v, 2p, 2p/(gamma-1)) and metric terms of the elements in shared memory
//      (coalesced loads);
//   B. one thread per (element, direction n, line): every pair i < k of the line is evaluated ONCE
//      (Sec. 2.2: Dt has zero diagonal and M Dt is skew-symmetric; f is symmetric) and added to both nodes
//      with Dt_ik and Dt_ki; the line's sums stay in registers and go to shared memory per direction;
//   C. one thread per node: sum the directions, add the lifted interface fluxes, scale by -1/J, store.
// ---------------------------------------------------------------------------------------------------
// The Runge-Kutta stage update at state offset o with the RHS value k (FP64), given the values of u (uo) and of
// the stage register yo (RK4: acc, CK45: K; read only after stage 0):
//   classical RK4, low storage: acc accumulates sum b_s dt k_s, y is the next stage state, u is updated last;
//   CK(5,4) 2N: K = A_s K + dt k, u = u + B_s K (Sec. 4.1).
template <int EPI>
__device__ __forceinline__ void stage_update(const Epilogue& epi, size_t o, double k, double uo, double yo) {
  if (EPI == EPI_RK4) {
    // weights: ca = dt/6, dt/3, dt/3, dt/6 and cy = dt/2, dt/2, dt for stages 0..3 (set by the host)
    if (epi.stage == 0) {
      epi.acc[o] = epi.ca * k;
      epi.y[o] = uo + epi.cy * k;
    } else if (epi.stage < 3) {
      epi.acc[o] = yo + epi.ca * k;
      epi.y[o] = uo + epi.cy * k;
    } else {
      epi.uw[o] = uo + yo + epi.ca * k;
    }
  } else {
    const double kk = (epi.stage == 0 ? 0.0 : epi.a * yo) + epi.dt * k;
    epi.y[o] = kk;
    epi.uw[o] = uo + epi.b * kk;
  }
}

// The same update with the node's Jacobian factor s = -1/J folded into the weights (k = s tot; FP64 flux
// arithmetic): w1 = s b_s dt (RK4: the weight of k in acc, or in u at the last stage) or s dt (CK45), w2 = s c dt
// (RK4: the weight of k in the next stage state). Two products per node replace one per value.
template <int EPI>
__device__ __forceinline__ void stage_weights(const Epilogue& epi, double s, double& w1, double& w2) {
  if (EPI == EPI_RK4) {
    w1 = epi.ca * s;
    w2 = epi.cy * s;
  } else {
    w1 = epi.dt * s;
    w2 = 0.0;
  }
}

template <int EPI>
__device__ __forceinline__ void stage_update_w(const Epilogue& epi, size_t o, double tot, double w1, double w2,
                                               double uo, double yo) {
  if (EPI == EPI_RK4) {
    if (epi.stage == 0) {
      epi.acc[o] = w1 * tot;
      epi.y[o] = uo + w2 * tot;
    } else if (epi.stage < 3) {
      epi.acc[o] = yo + w1 * tot;
      epi.y[o] = uo + w2 * tot;
    } else {
      epi.uw[o] = uo + yo + w1 * tot;
    }
  } else {
    const double kk = (epi.stage == 0 ? 0.0 : epi.a * yo) + w1 * tot;
    epi.y[o] = kk;
    epi.uw[o] = uo + epi.b * kk;
  }
}

// Positive floating-point values order like their bit patterns read as unsigned integers: shared-memory integer
// atomicMin/atomicMax then give a tile's value range.
template <typename T>
struct RangeBits;
template <>
struct RangeBits<double> {
  using type = unsigned long long;
  __device__ static __forceinline__ type bits(double x) { return (type)__double_as_longlong(x); }
  __device__ static __forceinline__ double value(type b) { return __longlong_as_double((long long)b); }
};
template <>
struct RangeBits<float> {
  using type = unsigned int;
  __device__ static __forceinline__ type bits(float x) { return __float_as_uint(x); }
  __device__ static __forceinline__ float value(type b) { return __uint_as_float(b); }
};

template <int ND, int N, typename T>
struct VolumeSmem {
  using G = Geo<ND, N>;
  static constexpr int kPrim = NodeQ<ND>::NQ * G::NDOF;    // per element: node quantities
  static constexpr int kJa = ND * ND * G::NDOF;            // per element
  static constexpr int kAcc = ND * G::NV * G::NDOF;        // per element
  static constexpr int kPerElem = kPrim + kJa + kAcc;      // elements of T
  static constexpr int kState = G::NV * G::NDOF;           // doubles per element of one state array
  // per element with precomputed logarithms: [2][NDOF] logs, then (with the whole tile's logs first) 4 range slots
  static constexpr int kLog = 2 * G::NDOF + 4;
  // with a fused stage update, two FP64 state arrays of the CTA's elements are prefetched into shared memory
  static constexpr size_t bytes(int epb, bool fused, bool logs = false) {
    return (size_t)epb * (kPerElem + (logs ? kLog : 0)) * sizeof(T) +
           (fused ? (size_t)2 * epb * kState * sizeof(double) : 0);
  }
};

// Asynchronous 8-byte global -> shared copies (cp.async): issued early, completed before the values are used.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// EPI selects the epilogue: store du, or apply a Runge-Kutta stage update (in place of a separate kernel). With a
// stage update the kernel writes arrays that alias its input u (the CTA has read its own elements before the
// barrier; no other CTA reads them).
// The pairs i < k of one line (Sec. 2.2): sp/sj point at the line's first node in the node-quantity and metric
// arrays (stride st), sa at its accumulator slots (node k at so[k] = k st from sp and sa); each pair's flux is
// evaluated once and added to both nodes.
// With LM == LM_PRELOG, sl points at the line's first node in the per-node logarithm array [2][NDOF].
// fu, fl (optional): the lifted interface fluxes (f* / w_0, component stride NL) of the line's upper and lower face
// point; the surface term then starts the end nodes' sums (+fu at node N-1, -fl at node 0) instead of being added
// in the epilogue.
// pp0: 2 p_ref of the FP32 mode's reference pressure (the node quantities' pp is shifted by it), else 0.
// Ranocha's flux with the default log mean takes its beta form in FP64 (the node quantities' PG slot holds rho/p;
// c2 = 2/(gamma-1)): three FP64 products per pair less for one reciprocal per node, -3 % of the FP64 volume kernel.
// FP32 keeps pg (its FP32 pipe is not the bound, and the reciprocal lengthens phase A: +1.8 % at 16^3); so do
// Shima's flux and the log-mean variants.
template <int ND, int N, typename T, int FLUX, bool CART, int LM = LM_SHARED_RCP>
__device__ __forceinline__ void line_pairs(const T* sp, const int (&so)[N], const T* sj, const T* sl, int st, int n, T n2n,
                                           const OpTable<N, T>& op, T* sa, const T* fu = nullptr,
                                           const T* fl = nullptr, T pp0 = T(0), T c2 = T(0)) {
  constexpr bool kBeta = FLUX == 0 && LM == LM_SHARED_RCP && sizeof(T) == 8;
  using G = Geo<ND, N>;
  constexpr int NQ = NodeQ<ND>::NQ;
  T acc[N][G::NV];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < G::NV; ++c) acc[i][c] = T(0);
  if (fu) {
#pragma unroll
    for (int c = 0; c < G::NV; ++c) {
      acc[N - 1][c] = fu[c * G::NL];
      acc[0][c] = -fl[c * G::NL];
    }
  }
#pragma unroll
  for (int i = 0; i < N - 1; ++i) {
    T a[NQ], ja_i[ND], va_n = T(0);
#pragma unroll
    for (int c = 0; c < NQ; ++c) a[c] = sp[c * G::NDOF + so[i]];
    if (CART) {
      va_n = sp[(1 + n) * G::NDOF + so[i]];
    } else {
#pragma unroll
      for (int j = 0; j < ND; ++j) ja_i[j] = sj[j * G::NDOF + i * st];
    }
#pragma unroll
    for (int k = i + 1; k < N; ++k) {
      T b[NQ], f[G::NV];
#pragma unroll
      for (int c = 0; c < NQ; ++c) b[c] = sp[c * G::NDOF + so[k]];
      const LogRef<T> lg{sl + i * st, sl + k * st, G::NDOF};
      if (CART) {
        pair_flux8_cart<ND, T, FLUX, LM, true, kBeta>(a, b, va_n, sp[(1 + n) * G::NDOF + so[k]], n2n, n, f, lg,
                                                       pp0, c2);
      } else {
        T n2[ND];
#pragma unroll
        for (int j = 0; j < ND; ++j) n2[j] = ja_i[j] + sj[j * G::NDOF + k * st];
        pair_flux8<ND, T, FLUX, LM, true, kBeta>(a, b, n2, f, lg, pp0, c2);
      }
      const T dik = op.Dt8[i * N + k], dki = op.Dt8[k * N + i];
      // f[0] is the halved mass flux: 2 dik (f[0]) equals dik (2 f[0]) exactly
      acc[i][0] += op.D0[i * N + k] * f[0];
      acc[k][0] += op.D0[k * N + i] * f[0];
#pragma unroll
      for (int c = 1; c < G::NV; ++c) {
        acc[i][c] += dik * f[c];
        acc[k][c] += dki * f[c];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < G::NV; ++c) sa[c * G::NDOF + so[i]] = acc[i][c];
}

// One tile of EPB elements starting at element e0, computed by the kThreads threads of a CTA (kThreads >=
// EPB * TPE; threads beyond EPB * TPE only join the cooperative loops). smem_raw holds VolumeSmem::bytes(EPB).
template <int ND, int N, typename T, int EPB, int EPI, int kThreads, int LMK = LM_SHARED_RCP>
__device__ __forceinline__ void volume_tile(const double* u, const T* __restrict__ Ja, const double* __restrict__ invJ,
                                            const T* __restrict__ face, double* du, const MeshDims& md,
                                            const OpTable<N, T>& op, T gamma, int* flag, const Epilogue& epi, int e0,
                                            unsigned char* smem_raw, const Variant& var) {
  using G = Geo<ND, N>;
  using S = VolumeSmem<ND, N, T>;
  static_assert(kThreads >= EPB * G::TPE, "a tile needs one thread per element line");
  constexpr bool kFused = EPI != EPI_STORE;
  double* s_eu = reinterpret_cast<double*>(smem_raw);      // [EPB][NV][NDOF] fused update: u
  double* s_ey = s_eu + (kFused ? EPB * S::kState : 0);     // [EPB][NV][NDOF] fused update: acc (RK4) / K (CK45)
  T* s_prim = reinterpret_cast<T*>(s_ey + (kFused ? EPB * S::kState : 0));  // [EPB][NQ][NDOF]
  T* s_ja = s_prim + EPB * S::kPrim;                       // [EPB][ND][ND][NDOF]
  T* s_acc = s_ja + EPB * S::kJa;                          // [EPB][ND][NV][NDOF]
  T* s_log = s_acc + EPB * S::kAcc;                        // [EPB][2][NDOF], then [EPB][4] (LM_PRELOG only)
  const int tid = threadIdx.x;
  const int nel = min(EPB, md.E - e0);
  const T gm1 = gamma - T(1);

  // ---- prefetch the FP64 arrays the fused stage update reads, so that they arrive during the pair phase
  if (kFused) {
    const size_t base = (size_t)e0 * S::kState;
    const int cnt = nel * S::kState;
    const bool need_y = (EPI == EPI_RK4) ? epi.stage > 0 : epi.stage > 0;  // acc / K are read after stage 0
    const double* gy = EPI == EPI_RK4 ? epi.acc : epi.y;
    for (int idx = tid; idx < cnt; idx += kThreads) {
      cp_async8(s_eu + idx, epi.u + base + idx);
      if (need_y) cp_async8(s_ey + idx, gy + base + idx);
    }
    cp_async_commit();
  }

  // ---- A: node quantities and metric terms -> shared memory
  constexpr int NQ = NodeQ<ND>::NQ;
  typename RangeBits<T>::type* s_rng =  // [EPB][4]: min/max of rho and pp/rho per element (precomputed logs)
      reinterpret_cast<typename RangeBits<T>::type*>(s_log + EPB * 2 * G::NDOF);
  if constexpr (LMK == LM_PRELOG) {
    for (int idx = tid; idx < nel * 4; idx += kThreads) s_rng[idx] = (idx & 1) ? 0 : ~(typename RangeBits<T>::type)0;
    __syncthreads();
  }
  bool ok = true;
  for (int idx = tid; idx < nel * G::NDOF; idx += kThreads) {
    const int el = idx / G::NDOF, i = idx - el * G::NDOF;
    const double* ue = u + (size_t)(e0 + el) * G::NV * G::NDOF + i;
    double uc[G::NV];
#pragma unroll
    for (int c = 0; c < G::NV; ++c) uc[c] = ue[c * G::NDOF];
    T q[NQ];
    ok &= node_quantities<ND, T>(uc, gm1, T(2) / gm1, q, nullptr, var.sh_eh, var.sh_el, var.sh_pp,
                                 sizeof(T) == 8 && LMK == LM_SHARED_RCP && var.flux == 0);  // line_pairs' kBeta
#pragma unroll
    for (int c = 0; c < NQ; ++c) s_prim[(el * NQ + c) * G::NDOF + i] = q[c];
    if constexpr (LMK == LM_PRELOG) {  // the element's range of rho and w = pp/rho (positive floats order as integers)
      const T w = q[NodeQ<ND>::PP] * Num<T>::rcp(q[NodeQ<ND>::RHO]);
      atomicMin(&s_rng[el * 4 + 0], RangeBits<T>::bits(q[NodeQ<ND>::RHO]));
      atomicMax(&s_rng[el * 4 + 1], RangeBits<T>::bits(q[NodeQ<ND>::RHO]));
      atomicMin(&s_rng[el * 4 + 2], RangeBits<T>::bits(w));
      atomicMax(&s_rng[el * 4 + 3], RangeBits<T>::bits(w));
    }
  }
  if (!ok) atomicOr(flag, 1);
  if (!var.cart) {
    const T* jae = Ja + (size_t)e0 * S::kJa;
    for (int idx = tid; idx < nel * S::kJa; idx += kThreads) s_ja[idx] = jae[idx];
  }
  __syncthreads();

  // ---- A2 (precomputed logarithms): per-node logs of the elements where a pair can reach a log branch. The
  // mean of rho compares rho_b/rho_a, the inverse mean compares (rho_b pp_a)/(rho_a pp_b) = w_a/w_b with w = pp/rho.
  // If rho_max <= r rho_min and w_max <= r w_min (r = Num<T>::series_range()), every pair of the element takes
  // both series branches and the element needs no logarithm.
  if constexpr (LMK == LM_PRELOG) {
    for (int idx = tid; idx < nel * G::NDOF; idx += kThreads) {
      const int el = idx / G::NDOF, i = idx - el * G::NDOF;
      const T rmin = RangeBits<T>::value(s_rng[el * 4 + 0]), rmax = RangeBits<T>::value(s_rng[el * 4 + 1]);
      const T wmin = RangeBits<T>::value(s_rng[el * 4 + 2]), wmax = RangeBits<T>::value(s_rng[el * 4 + 3]);
      if (rmax <= Num<T>::series_range() * rmin && wmax <= Num<T>::series_range() * wmin) continue;
      const T* qe = s_prim + el * S::kPrim;
      T q[NQ];
#pragma unroll
      for (int c = 0; c < NQ; ++c) q[c] = qe[c * G::NDOF + i];
      T lr, lb;  // relative to the element's first node
      node_logs<ND, T>(q, qe[NodeQ<ND>::RHO * G::NDOF], qe[NodeQ<ND>::PP * G::NDOF], lr, lb);
      s_log[(el * 2 + 0) * G::NDOF + i] = lr;
      s_log[(el * 2 + 1) * G::NDOF + i] = lb;
    }
    __syncthreads();
  }

  // ---- B: pairs along lines (the flux and the Cartesian specialisation select one of four loop bodies)
  if (tid < nel * G::TPE) {
    const int el = tid / G::TPE, r = tid - el * G::TPE;
    const int n = r / G::NL, l = r - n * G::NL;
    const int st = G::stride(n), base = G::line_base(n, l);
    const T* sp = s_prim + el * S::kPrim + base;
    const T* sj = s_ja + (el * ND + n) * ND * G::NDOF + base;
    const T* sl = s_log + el * 2 * G::NDOF + base;
    T* sa = s_acc + (el * ND + n) * G::NV * G::NDOF + base;
    int so[N];
#pragma unroll
    for (int k = 0; k < N; ++k) so[k] = k * st;
    const T n2n = T(2) * to_flux<T>(cart_jn(var, n));
    if constexpr (LMK == LM_SHARED_RCP) {
      const T pp0 = T(var.sh_pp), c2 = T(2) / gm1;
      switch (var.flux * 2 + var.cart) {
        case 0: line_pairs<ND, N, T, 0, false>(sp, so, sj, sl, st, n, n2n, op, sa, nullptr, nullptr, pp0, c2); break;
        case 1: line_pairs<ND, N, T, 0, true>(sp, so, sj, sl, st, n, n2n, op, sa, nullptr, nullptr, pp0, c2); break;
        case 2: line_pairs<ND, N, T, 1, false>(sp, so, sj, sl, st, n, n2n, op, sa, nullptr, nullptr, pp0); break;
        default: line_pairs<ND, N, T, 1, true>(sp, so, sj, sl, st, n, n2n, op, sa, nullptr, nullptr, pp0); break;
      }
    } else if constexpr (LMK == LM_PRELOG) {
      if (var.cart)
        line_pairs<ND, N, T, 0, true, LM_PRELOG>(sp, so, sj, sl, st, n, n2n, op, sa);
      else
        line_pairs<ND, N, T, 0, false, LM_PRELOG>(sp, so, sj, sl, st, n, n2n, op, sa);
    } else {
      line_pairs<ND, N, T, 0, false, LMK>(sp, so, sj, sl, st, n, n2n, op, sa);
    }
  }
  __syncthreads();

  // ---- C: sum directions, lift interface fluxes, scale by -1/J
  if (kFused) {
    cp_async_wait_all();
    __syncthreads();
  }
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
        const T* fp = face + ((size_t)n * md.E + fe) * G::NV * G::NL + fn;  // lifted: f* / w_0
        if (in == N - 1) {
#pragma unroll
          for (int c = 0; c < G::NV; ++c) tot[c] += fp[c * G::NL];
        } else {
#pragma unroll
          for (int c = 0; c < G::NV; ++c) tot[c] -= fp[c * G::NL];
        }
      }
    }
    const double ij = var.cart ? var.invJ : invJ[(size_t)ge * G::NDOF + i];
    const double sj = -ij;
    const T sjT = sizeof(T) == 8 ? T(0) : -to_flux<T>(ij);
    const size_t off = (size_t)ge * G::NV * G::NDOF + i;
    if constexpr (sizeof(T) == 8 && EPI != EPI_STORE) {  // FP64: -1/J folded into the stage weights
      double w1, w2;
      stage_weights<EPI>(epi, sj, w1, w2);
#pragma unroll
      for (int c = 0; c < G::NV; ++c) {
        const int so = (el * G::NV + c) * G::NDOF + i;
        stage_update_w<EPI>(epi, off + (size_t)c * G::NDOF, (double)tot[c], w1, w2, s_eu[so], s_ey[so]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < G::NV; ++c) {
        const size_t o = off + (size_t)c * G::NDOF;
        const int so = (el * G::NV + c) * G::NDOF + i;  // same value, prefetched into shared memory
        // FP64: k = -(1/J) tot in FP64. FP32 mode: the scaling in FP32 and an exact integer-pipe widening, so the
        // FP64 pipe only carries the RK accumulation below.
        const double k = sizeof(T) == 8 ? sj * (double)tot[c] : f2d_int((float)(sjT * tot[c]));
        if (EPI == EPI_STORE)
          du[o] = k;
        else
          stage_update<EPI>(epi, o, k, s_eu[so], s_ey[so]);
      }
    }
  }
}

// LMK, the log-mean variant, is a template parameter so that each variant's kernel has its own register
// allocation (the default kernels do not carry the registers of the ablation variants); the flux and the
// Cartesian specialisation are selected at run time inside the default kernel.
template <int ND, int N, typename T, int EPB, int EPI, int LMK>
__global__ void __launch_bounds__(EPB* Geo<ND, N>::TPE)
    volume_kernel(const double* u, const T* __restrict__ Ja, const double* __restrict__ invJ,
                  const T* __restrict__ face, double* du, MeshDims md, OpTable<N, T> op, T gamma, int* flag,
                  Epilogue epi, Variant var) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  volume_tile<ND, N, T, EPB, EPI, EPB * Geo<ND, N>::TPE, LMK>(u, Ja, invJ, face, du, md, op, gamma, flag, epi,
                                                              var.ghost + blockIdx.x * EPB, smem_raw, var);
}

}  // namespace dgk
