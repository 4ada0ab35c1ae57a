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

}  // namespace

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
