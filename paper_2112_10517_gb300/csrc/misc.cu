// Runge-Kutta coefficients and the entropy-rate diagnostic (FP64). The stage updates themselves run in the
// volume kernel's epilogue.
#include "kernels.cuh"
#include "volume_pipe.cuh"

namespace dgk {
namespace {

// Carpenter-Kennedy five-stage fourth-order 2N-storage coefficients (Sec. 4.1; Carpenter and Kennedy 1994).
constexpr double kCkAh[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                             -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
constexpr double kCkBh[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                             1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                             2277821191437.0 / 14882151754819.0};
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1024;

// Entropy rate (Sec. 2): sum_nodes J W w(u) . du with w = ((gamma - s)/(gamma-1) - rho|v|^2/(2p), rho v/p, -rho/p),
// s = log p - gamma log rho. Each thread walks a fixed node subset; blocks reduce in a fixed tree order, so the
// result does not depend on scheduling.
template <int ND>
__global__ void __launch_bounds__(kRedThreads)
    entropy_partial_kernel(const double* __restrict__ u, const double* __restrict__ du, const double* __restrict__ JW,
                           long long nodes, int ndof, double gamma, double* __restrict__ partial) {
  constexpr int NV = ND + 2;
  double s = 0.0, sa = 0.0;
  for (long long g = (long long)blockIdx.x * kRedThreads + threadIdx.x; g < nodes; g += (long long)gridDim.x * kRedThreads) {
    const long long e = g / ndof;
    const int i = (int)(g - e * ndof);
    const double* ue = u + (size_t)e * NV * ndof + i;
    const double* de = du + (size_t)e * NV * ndof + i;
    const double rho = ue[0];
    double m2 = 0.0;
#pragma unroll
    for (int j = 0; j < ND; ++j) m2 += ue[(1 + j) * ndof] * ue[(1 + j) * ndof];
    const double p = (gamma - 1.0) * (ue[(ND + 1) * ndof] - 0.5 * m2 / rho);
    const double ent = log(p) - gamma * log(rho);
    const double beta = rho / p;
    const double jw = JW[g];
    double t = jw * ((gamma - ent) / (gamma - 1.0) - 0.5 * beta * m2 / (rho * rho)) * de[0];
    double ta = fabs(t);
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const double tj = jw * (ue[(1 + j) * ndof] / p) * de[(1 + j) * ndof];
      t += tj;
      ta += fabs(tj);
    }
    const double te = -jw * beta * de[(ND + 1) * ndof];
    t += te;
    ta += fabs(te);
    s += t;
    sa += ta;
  }
  __shared__ double sh[2][kRedThreads];
  sh[0][threadIdx.x] = s;
  sh[1][threadIdx.x] = sa;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sh[0][0];
    partial[2 * blockIdx.x + 1] = sh[1][0];
  }
}

__global__ void __launch_bounds__(kRedThreads) reduce_pairs_kernel(const double* __restrict__ partial, int nb,
                                                                   double* __restrict__ out) {
  __shared__ double sh[2][kRedThreads];
  double s = 0.0, sa = 0.0;
  for (int b = threadIdx.x; b < nb; b += kRedThreads) {
    s += partial[2 * b];
    sa += partial[2 * b + 1];
  }
  sh[0][threadIdx.x] = s;
  sh[1][threadIdx.x] = sa;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sh[0][0];
    out[1] = sh[1][0];
  }
}

// Conserved totals (the c scalars of discrete conservation, Sec. 2): sum over nodes of J W q per variable; the same
// fixed-order reduction as the entropy rate.
template <int NV>
__global__ void __launch_bounds__(kRedThreads)
    totals_partial_kernel(const double* __restrict__ q, const double* __restrict__ JW, long long nodes, int ndof,
                          double* __restrict__ partial) {
  double s[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) s[c] = 0.0;
  for (long long g = (long long)blockIdx.x * kRedThreads + threadIdx.x; g < nodes; g += (long long)gridDim.x * kRedThreads) {
    const long long e = g / ndof;
    const int i = (int)(g - e * ndof);
    const double jw = JW[g];
#pragma unroll
    for (int c = 0; c < NV; ++c) s[c] += jw * q[((size_t)e * NV + c) * ndof + i];
  }
  __shared__ double sh[NV][kRedThreads];
#pragma unroll
  for (int c = 0; c < NV; ++c) sh[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int c = 0; c < NV; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) partial[(size_t)blockIdx.x * NV + c] = sh[c][0];
  }
}

template <int NV>
__global__ void __launch_bounds__(kRedThreads) reduce_totals_kernel(const double* __restrict__ partial, int nb,
                                                                    double* __restrict__ out) {
  __shared__ double sh[NV][kRedThreads];
  double s[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) s[c] = 0.0;
  for (int b = threadIdx.x; b < nb; b += kRedThreads) {
#pragma unroll
    for (int c = 0; c < NV; ++c) s[c] += partial[(size_t)b * NV + c];
  }
#pragma unroll
  for (int c = 0; c < NV; ++c) sh[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int c = 0; c < NV; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) out[c] = sh[c][0];
  }
}

// Halo planes of a partitioned context (the cut runs along the last direction, whose node stride is NL = N^(ND-1)):
// plane k of element e holds the nodes k NL .. k NL + NL - 1 of each variable. A halo buffer is [layer][NV][NL] for
// the `layer` elements of one element layer (consecutive in the element order).
//   pack:   send_lo <- plane 0 of the first owned layer, send_hi <- plane N-1 of the last owned layer
//   unpack: plane N-1 of the ghost layer <- recv_lo (the lower neighbour's last layer's plane N-1),
//           plane 0 of the ghost layer <- recv_hi (the upper neighbour's first layer's plane 0)
__global__ void halo_kernel(double* u, const double* recv_lo, const double* recv_hi, double* send_lo,
                            double* send_hi, int layer, int nv, int nl, int ndof, long long first_owned,
                            long long last_owned, int pack) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long count = (long long)layer * nv * nl;
  pdl_wait();  // the state comes from the kernel before (a stage update), the ghost layer is read after this one
  if (g >= count) return;
  const int fn = (int)(g % nl);
  const long long t = g / nl;
  const int c = (int)(t % nv);
  const long long pos = t / nv;
  const int top = (ndof / nl - 1) * nl;  // first node of plane N-1
  if (pack) {
    send_lo[g] = u[((first_owned + pos) * nv + c) * ndof + fn];
    send_hi[g] = u[((last_owned + pos) * nv + c) * ndof + top + fn];
  } else {
    u[(pos * nv + c) * ndof + top + fn] = recv_lo[g];
    u[(pos * nv + c) * ndof + fn] = recv_hi[g];
  }
}

}  // namespace

cudaError_t launch_halo(int nd, int p, int layer, long long first_owned, long long last_owned, double* u,
                        const double* recv_lo, const double* recv_hi, double* send_lo, double* send_hi, bool pack,
                        bool overlap, cudaStream_t s) {
  const int N = p + 1, nv = nd + 2;
  const int nl = nd == 3 ? N * N : N;
  const long long count = (long long)layer * nv * nl;
  if (count <= 0) return cudaSuccess;
  const int threads = 256;
  const cudaError_t e = launch_kernel(halo_kernel, dim3((unsigned)((count + threads - 1) / threads)), dim3(threads), 0,
                                      s, overlap, u, recv_lo, recv_hi, send_lo, send_hi, layer, nv, nl, nl * N,
                                      first_owned, last_owned, pack ? 1 : 0);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_totals(int nd, int p, long long nelem, const double* q, const double* JW, double* partial,
                          int nblocks, double* out, cudaStream_t s) {
  const int N = p + 1;
  const int ndof = nd == 3 ? N * N * N : N * N;
  const long long nodes = nelem * ndof;
  cudaError_t e;
  if (nd == 2) {
    totals_partial_kernel<4><<<nblocks, kRedThreads, 0, s>>>(q, JW, nodes, ndof, partial);
    e = cudaGetLastError();
    if (e == cudaSuccess) reduce_totals_kernel<4><<<1, kRedThreads, 0, s>>>(partial, nblocks, out);
  } else {
    totals_partial_kernel<5><<<nblocks, kRedThreads, 0, s>>>(q, JW, nodes, ndof, partial);
    e = cudaGetLastError();
    if (e == cudaSuccess) reduce_totals_kernel<5><<<1, kRedThreads, 0, s>>>(partial, nblocks, out);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

int entropy_rate_blocks() { return kRedBlocks; }

void ck45_coefficients(int stage, double* a, double* b) {
  *a = kCkAh[stage];
  *b = kCkBh[stage];
}

cudaError_t launch_entropy_rate(int nd, int p, MeshDims md, const double* u, const double* du, const double* JW,
                                double gamma, double* partial, int nblocks, double* out, cudaStream_t s) {
  const int N = p + 1;
  const int ndof = nd == 3 ? N * N * N : N * N;
  const long long nodes = (long long)md.E * ndof;
  if (nd == 2)
    entropy_partial_kernel<2><<<nblocks, kRedThreads, 0, s>>>(u, du, JW, nodes, ndof, gamma, partial);
  else
    entropy_partial_kernel<3><<<nblocks, kRedThreads, 0, s>>>(u, du, JW, nodes, ndof, gamma, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_pairs_kernel<<<1, kRedThreads, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}

// One thread waits on an mbarrier that expects one arrival and gets none: mbar_wait_bounded gives up and the flag
// records the timeout, as in the pipelined volume kernel.
__global__ void wait_probe_kernel(int* flag) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
    if (!mbar_wait_bounded(&bar, 0u)) atomicOr(flag, FLAG_WAIT_TIMEOUT);
  }
}

cudaError_t launch_wait_probe(int* flag, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(flag);
  return cudaGetLastError();
}

}  // namespace dgk
