// Batched RHS: many independent meshes of uneven size and polynomial degree in one persistent launch.
//
// Every instance is a dg_ctx (its own mesh, metrics and interface-flux workspace). A plan binds the instances
// and their state buffers; dg_batch_rhs then queues one memset and two launches on a stream:
//   1. one interface-flux launch over the face nodes of all instances (the instance is found by binary search
//      in the prefix sums of the face-node counts),
//   2. one persistent volume launch per polynomial degree present: each CTA repeatedly takes the next element
//      tile of its degree from a global work counter and runs the volume/lift/Jacobian code. A kernel per degree
//      keeps each degree's register allocation (one kernel over all degrees would carry the largest). With the
//      default log mean and pipelined staging (the contexts' dg_opts.staging) the kernel is the pipelined one of
//      volume_pipe.cuh: a CTA takes its next tile from the counter while the current one computes and copies
//      that tile's data from its instance's arrays with asynchronous copies.
// The work is the same per element as dg_rhs (Eq. fluxdiff-SBP-opDsplit); only the scheduling differs.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "volume_pipe.cuh"

namespace dgk {
namespace {

constexpr int kBatchMaxP = 5;  // degrees 1..5 in a batch
const int kThreadChoices[] = {128, 192, 256};
constexpr int kNumThreadChoices = 3;

struct BatchInst {
  const double* u;
  double* du;
  const void* Ja;
  const double* invJ;
  void* face;
  int* flag;
  MeshDims md;
  int p;
  long long face_begin;  // first face node of this instance in the flattened interface launch
};

struct BatchTile {
  int inst;
  int e0;
};

// flux-differencing tables of every degree in constant memory (one copy per device, uploaded at plan creation)
#define DG_BATCH_CONST_OP(NN)                                                       \
  __constant__ OpTable<NN, double> c_opd_##NN;                                      \
  __constant__ OpTable<NN, float> c_opf_##NN;
DG_BATCH_CONST_OP(2)
DG_BATCH_CONST_OP(3)
DG_BATCH_CONST_OP(4)
DG_BATCH_CONST_OP(5)
DG_BATCH_CONST_OP(6)

template <int N, typename T>
struct ConstOp;
#define DG_BATCH_CONST_GET(NN)                                                                           \
  template <>                                                                                            \
  struct ConstOp<NN, double> {                                                                           \
    __device__ static __forceinline__ const OpTable<NN, double>& get() { return c_opd_##NN; }           \
  };                                                                                                     \
  template <>                                                                                            \
  struct ConstOp<NN, float> {                                                                            \
    __device__ static __forceinline__ const OpTable<NN, float>& get() { return c_opf_##NN; }            \
  };
DG_BATCH_CONST_GET(2)
DG_BATCH_CONST_GET(3)
DG_BATCH_CONST_GET(4)
DG_BATCH_CONST_GET(5)
DG_BATCH_CONST_GET(6)

// elements per tile for degree N at a CTA size: as many element line sets as fit, capped by shared memory
template <int N, typename T, int THREADS, int LMK = LM_SHARED_RCP>
struct BatchEpb {
  static constexpr int kByThreads = THREADS / Geo<3, N>::TPE;
  static constexpr int kBySmem = (int)(200 * 1024 / VolumeSmem<3, N, T>::bytes(1, false, LMK == LM_PRELOG));
  static constexpr int value = kByThreads < kBySmem ? kByThreads : kBySmem;
  static_assert(value >= 1, "CTA too small for this degree");
};

// shared memory per element of the volume tile (node quantities, metric terms, accumulators; with precomputed
// logarithms two more values per node and four range slots), as VolumeSmem<3, N, T>::bytes(1, false, logs)
size_t batch_smem_per_elem(int p, int precision, bool logs) {
  const int N = p + 1;
  return (size_t)((6 + 9 + 15) * N * N * N + (logs ? 2 * N * N * N + 4 : 0)) * (precision == DG_FP32 ? 4 : 8);
}

int batch_epb(int p, int precision, int threads, bool logs) {
  const int N = p + 1;
  const int tpe = 3 * N * N;
  const int by_t = threads / tpe, by_s = (int)(200 * 1024 / batch_smem_per_elem(p, precision, logs));
  return std::max(1, std::min(by_t, by_s));
}

size_t batch_smem(int p, int precision, int threads, bool logs) {
  return batch_smem_per_elem(p, precision, logs) * batch_epb(p, precision, threads, logs);
}

// batches use Ranocha's flux on the instances' metric arrays (a compile-time variant, so only that loop is built)
__device__ __forceinline__ Variant general_variant(int lm = LM_SHARED_RCP) {
  Variant v;
  v.flux = 0;
  v.cart = 0;
  v.lm = lm;
  v.jn[0] = v.jn[1] = v.jn[2] = 0.0;
  v.invJ = 0.0;
  v.sh_eh = v.sh_el = v.sh_pp = 0.0f;  // batches take no reference pressure
  v.ghost = 0;                         // nor partitioned contexts
  v.fgeo = nullptr;                    // the interface kernel forms the geometry from the instances' metric terms
  v.if_e0 = v.if_e1 = 0;
  v.tiles = nullptr;
  return v;
}

template <typename T, bool LLF>
__global__ void __launch_bounds__(256) batch_interface_kernel(const BatchInst* __restrict__ insts, int n,
                                                              long long total, T gamma) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = n - 1;  // last instance with face_begin <= g
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (insts[mid].face_begin <= g) lo = mid;
    else hi = mid - 1;
  }
  const BatchInst& in = insts[lo];
  const int idx = (int)(g - in.face_begin);  // < 3 E NL < 2^31 per instance
  const double* u = in.u;
  const T* ja = static_cast<const T*>(in.Ja);
  T* face = static_cast<T*>(in.face);
  switch (in.p) {
    case 1: interface_node<3, 2, T, LLF, 0>(u, ja, face, in.md, gamma, in.flag, idx, general_variant()); break;
    case 2: interface_node<3, 3, T, LLF, 0>(u, ja, face, in.md, gamma, in.flag, idx, general_variant()); break;
    case 3: interface_node<3, 4, T, LLF, 0>(u, ja, face, in.md, gamma, in.flag, idx, general_variant()); break;
    case 4: interface_node<3, 5, T, LLF, 0>(u, ja, face, in.md, gamma, in.flag, idx, general_variant()); break;
    case 5: interface_node<3, 6, T, LLF, 0>(u, ja, face, in.md, gamma, in.flag, idx, general_variant()); break;
    default: break;
  }
}

template <int N, typename T, int THREADS, int LMK>
__device__ __forceinline__ void batch_tile(const BatchInst& in, int e0, T gamma, unsigned char* smem) {
  constexpr int EPB = BatchEpb<N, T, THREADS, LMK>::value;
  Epilogue none{};
  none.mode = EPI_STORE;
  volume_tile<3, N, T, EPB, EPI_STORE, THREADS, LMK>(in.u, static_cast<const T*>(in.Ja), in.invJ,
                                                     static_cast<const T*>(in.face), in.du, in.md,
                                                     ConstOp<N, T>::get(), gamma, in.flag, none, e0, smem,
                                                     general_variant(LMK));
}

// Persistent volume kernel of one degree (N nodes per line): CTAs take tiles of that degree from the counter.
// LMK: the log-mean variant of the batch's contexts (the default, or logarithms precomputed per node).
template <int N, typename T, int THREADS, int LMK>
__global__ void __launch_bounds__(THREADS) batch_volume_kernel(const BatchInst* __restrict__ insts,
                                                               const BatchTile* __restrict__ tiles, int ntiles,
                                                               int* counter, T gamma) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const BatchTile tl = tiles[t];
    batch_tile<N, T, THREADS, LMK>(insts[tl.inst], tl.e0, gamma, smem);
    __syncthreads();  // the next tile reuses shared memory and s_tile
  }
}

// The batch's tiles for the pipelined kernel: taken from the degree's work counter one ahead (thread 0 fetches the
// next index while the current tile computes), each tile from its instance's arrays. (The batch kernel is launched
// without the programmatic-dependence attribute, so the counter it takes before pdl_wait is already reset.)
template <typename T>
struct BatchTileSource {
  const BatchInst* insts;
  const BatchTile* tiles;
  int ntiles;
  int* counter;
  __device__ __forceinline__ int first() const { return atomicAdd(counter, 1); }
  __device__ __forceinline__ int next(int) const { return atomicAdd(counter, 1); }
  __device__ __forceinline__ bool valid(int t) const { return t < ntiles; }
  __device__ __forceinline__ PipeTile<T> tile(int t) const {
    const BatchTile bt = tiles[t];
    const BatchInst& in = insts[bt.inst];
    return PipeTile<T>{in.u, static_cast<const T*>(in.Ja), in.invJ, static_cast<const T*>(in.face), in.du,
                       in.flag, in.md, bt.e0, 1 << 30};  // bounded by the kernel's tile size and the instance's end
  }
  __device__ __forceinline__ void finish() const {}  // the counter is reset before each launch
};

// The pipelined batch kernel of degree N at a CTA size: the tile of the direct kernel (elements per tile of the
// tile table), one thread per element line set.
template <int N, typename T, int THREADS>
struct BatchPipe {
  static constexpr int EPB = BatchEpb<N, T, THREADS, LM_SHARED_RCP>::value;
  static constexpr int kThreads = EPB * Geo<3, N>::TPE;
  static constexpr size_t kSmem = PipeSmem<3, N, T>::bytes(EPB, false);
  static constexpr bool kFits = kSmem <= 227 * 1024;
};

template <int N, typename T, int THREADS>
__global__ void __launch_bounds__(BatchPipe<N, T, THREADS>::kThreads,
                                  pipe_min_ctas<3, N, T, BatchPipe<N, T, THREADS>::EPB>())
    batch_pipe_kernel(const BatchInst* __restrict__ insts, const BatchTile* __restrict__ tiles, int ntiles,
                      int* counter, T gamma) {
  const BatchTileSource<T> src{insts, tiles, ntiles, counter};
  Epilogue none{};
  none.mode = EPI_STORE;
  pipe_tiles<3, N, T, BatchPipe<N, T, THREADS>::EPB, EPI_STORE>(src, ConstOp<N, T>::get(), gamma, none,
                                                                general_variant());
}

template <typename T>
cudaError_t upload_const_ops() {
  cudaError_t e = cudaSuccess;
#define DG_BATCH_UPLOAD(NN, SYM)                                               \
  if (e == cudaSuccess) {                                                      \
    OpTable<NN, T> op;                                                         \
    const RefTables& t = ref_tables(NN - 1);                                   \
    for (int i = 0; i < NN * NN; ++i) {                                        \
      op.Dt8[i] = (T)(0.125 * t.Dt[i]);                                        \
      op.D0[i] = (T)(0.25 * t.Dt[i]);                                          \
    }                                                                          \
    op.winv = (T)(1.0 / t.w[0]);                                               \
    op.lift8 = (T)(0.125 / t.w[0]);                                            \
    e = cudaMemcpyToSymbol(SYM, &op, sizeof(op));                              \
  }
  if (sizeof(T) == 8) {
    DG_BATCH_UPLOAD(2, c_opd_2) DG_BATCH_UPLOAD(3, c_opd_3) DG_BATCH_UPLOAD(4, c_opd_4)
    DG_BATCH_UPLOAD(5, c_opd_5) DG_BATCH_UPLOAD(6, c_opd_6)
  } else {
    DG_BATCH_UPLOAD(2, c_opf_2) DG_BATCH_UPLOAD(3, c_opf_3) DG_BATCH_UPLOAD(4, c_opf_4)
    DG_BATCH_UPLOAD(5, c_opf_5) DG_BATCH_UPLOAD(6, c_opf_6)
  }
#undef DG_BATCH_UPLOAD
  return e;
}

std::mutex g_upload_mutex;
bool g_uploaded[64] = {false};

cudaError_t ensure_const_ops(int device) {
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_upload_mutex);
  if (g_uploaded[device]) return cudaSuccess;
  cudaError_t e = upload_const_ops<double>();
  if (e == cudaSuccess) e = upload_const_ops<float>();
  if (e == cudaSuccess) g_uploaded[device] = true;
  return e;
}

// One entry point per (degree, precision, CTA size): its occupancy at a shared-memory size, or its launch.
// The kernel's dynamic shared-memory opt-in is raised once to the largest size asked for, so that launches issue
// no attribute call (a batch's launches can then be captured in a CUDA graph after a first call outside it).
// (Function attributes are per device: the largest size set so far is kept per device.)
template <int N, typename T, int THREADS, int LMK>
cudaError_t batch_volume_optin(size_t smem) {
  static std::mutex m;
  static size_t done[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(m);
  if (smem <= done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(batch_volume_kernel<N, T, THREADS, LMK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e == cudaSuccess) done[dev] = smem;
  return e;
}

template <int N, typename T, int THREADS>
cudaError_t batch_pipe_optin() {
  static PerDeviceCache cache;
  long long done = 0;
  return per_device(cache, &done, [](long long* v) {
    *v = 1;
    return cudaFuncSetAttribute(batch_pipe_kernel<N, T, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)BatchPipe<N, T, THREADS>::kSmem);
  });
}

// pipe: the pipelined kernel (its own CTA size and shared memory); else the per-tile kernel with `smem`.
template <int N, typename T, int THREADS>
cudaError_t batch_volume_call(int lm, bool pipe, bool launch, const BatchInst* insts, const BatchTile* tiles,
                              int ntiles, int* counter, double gamma, size_t smem, int grid, cudaStream_t s,
                              int* occupancy) {
  if (pipe) {
    using BP = BatchPipe<N, T, THREADS>;
    if constexpr (BP::kFits) {
      cudaError_t e = batch_pipe_optin<N, T, THREADS>();
      if (e != cudaSuccess) return e;
      if (!launch)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, batch_pipe_kernel<N, T, THREADS>,
                                                             BP::kThreads, BP::kSmem);
      batch_pipe_kernel<N, T, THREADS><<<grid, BP::kThreads, BP::kSmem, s>>>(insts, tiles, ntiles, counter, (T)gamma);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  auto kern = lm == LM_PRELOG ? batch_volume_kernel<N, T, THREADS, LM_PRELOG>
                              : batch_volume_kernel<N, T, THREADS, LM_SHARED_RCP>;
  cudaError_t e = lm == LM_PRELOG ? batch_volume_optin<N, T, THREADS, LM_PRELOG>(smem)
                                  : batch_volume_optin<N, T, THREADS, LM_SHARED_RCP>(smem);
  if (e != cudaSuccess) return e;
  if (!launch) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, kern, THREADS, smem);
  kern<<<grid, THREADS, smem, s>>>(insts, tiles, ntiles, counter, (T)gamma);
  return cudaGetLastError();
}

// The arguments of one degree's persistent launch (or of its occupancy query).
struct BatchCall {
  int lm;
  bool pipe;
  bool launch;
  const BatchInst* insts;
  const BatchTile* tiles;
  int ntiles;
  int* counter;
  double gamma;
  size_t smem;
  int grid;
  cudaStream_t s;
  int* occupancy;
};

template <typename T, int THREADS>
cudaError_t batch_volume_p(int p, const BatchCall& c) {
#define DG_BATCH_CALL(NN)                                                                                        \
  batch_volume_call<NN, T, THREADS>(c.lm, c.pipe, c.launch, c.insts, c.tiles, c.ntiles, c.counter, c.gamma, c.smem, \
                                    c.grid, c.s, c.occupancy)
  switch (p) {
    case 1: return DG_BATCH_CALL(2);
    case 2: return DG_BATCH_CALL(3);
    case 3: return DG_BATCH_CALL(4);
    case 4: return DG_BATCH_CALL(5);
    case 5: return DG_BATCH_CALL(6);
    default: return cudaErrorInvalidValue;
  }
#undef DG_BATCH_CALL
}

cudaError_t batch_volume(int precision, int threads, int p, const BatchCall& c) {
  if (precision == DG_FP32) {
    if (threads == 128) return batch_volume_p<float, 128>(p, c);
    if (threads == 192) return batch_volume_p<float, 192>(p, c);
    return batch_volume_p<float, 256>(p, c);
  }
  if (threads == 128) return batch_volume_p<double, 128>(p, c);
  if (threads == 192) return batch_volume_p<double, 192>(p, c);
  return batch_volume_p<double, 256>(p, c);
}

// Whether the pipelined kernel fits degree p's tile at a CTA size (its shared memory within the opt-in limit).
template <typename T, int THREADS>
bool batch_pipe_fits_t(int p) {
  switch (p) {
    case 1: return BatchPipe<2, T, THREADS>::kFits;
    case 2: return BatchPipe<3, T, THREADS>::kFits;
    case 3: return BatchPipe<4, T, THREADS>::kFits;
    case 4: return BatchPipe<5, T, THREADS>::kFits;
    case 5: return BatchPipe<6, T, THREADS>::kFits;
    default: return false;
  }
}

bool batch_pipe_fits(int precision, int threads, int p) {
  if (precision == DG_FP32)
    return threads == 128 ? batch_pipe_fits_t<float, 128>(p)
                          : (threads == 192 ? batch_pipe_fits_t<float, 192>(p) : batch_pipe_fits_t<float, 256>(p));
  return threads == 128 ? batch_pipe_fits_t<double, 128>(p)
                        : (threads == 192 ? batch_pipe_fits_t<double, 192>(p) : batch_pipe_fits_t<double, 256>(p));
}

int occupancy_for(int precision, int threads, int p, int lm, bool pipe, size_t smem) {
  int occ = 0;
  const BatchCall c{lm, pipe, false, nullptr, nullptr, 0, nullptr, 0.0, smem, 0, 0, &occ};
  if (batch_volume(precision, threads, p, c) != cudaSuccess) return 0;
  return occ;
}

}  // namespace
}  // namespace dgk

// ---------------------------------------------------------------------------------------------------------
// The plan
// ---------------------------------------------------------------------------------------------------------
struct dg_batch {
  int device = 0, n = 0, precision = 0, llf = 0, sms = 0, lm = 0;
  double gamma = 1.4;
  long long total_face_nodes = 0;
  dgk::BatchInst* d_inst = nullptr;
  // element tiles per CTA size and degree (index p), and the shared memory of that degree's kernel
  dgk::BatchTile* d_tiles[dgk::kNumThreadChoices][dgk::kBatchMaxP + 1] = {};
  int ntiles[dgk::kNumThreadChoices][dgk::kBatchMaxP + 1] = {};
  size_t smem[dgk::kNumThreadChoices][dgk::kBatchMaxP + 1] = {};
  int* d_counter = nullptr;  // one work counter per degree
  // the per-degree kernels run concurrently: forked from the caller's stream after the interface launch, joined
  // before dg_batch_rhs returns (in a captured graph these become parallel branches)
  cudaStream_t streams[dgk::kBatchMaxP + 1] = {};
  cudaEvent_t fork = nullptr, join[dgk::kBatchMaxP + 1] = {};
  int occ[dgk::kNumThreadChoices][dgk::kBatchMaxP + 1];  // occupancy limits, -1 until queried
  bool pipe[dgk::kNumThreadChoices][dgk::kBatchMaxP + 1] = {};  // the pipelined kernel for this CTA size and degree
  int threads_idx = 1;  // 192 threads per CTA until tuned
  int ctas_per_sm = 0;  // 0: the occupancy limit
  std::string signature;
};

namespace {

void batch_release(dg_batch* b) {
  if (!b) return;
  cudaFree(b->d_inst);
  for (int i = 0; i < dgk::kNumThreadChoices; ++i)
    for (int p = 0; p <= dgk::kBatchMaxP; ++p) cudaFree(b->d_tiles[i][p]);
  cudaFree(b->d_counter);
  for (int p = 0; p <= dgk::kBatchMaxP; ++p) {
    if (b->streams[p]) cudaStreamDestroy(b->streams[p]);
    if (b->join[p]) cudaEventDestroy(b->join[p]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

dg_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return DG_OK;
  return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
}

// persistent grid of degree p's kernel: CTAs per SM (tuned, capped by the occupancy limit) times SMs, at most the
// number of tiles
int occupancy_of(dg_batch* b, int ti, int p) {
  if (b->occ[ti][p] < 0)
    b->occ[ti][p] = dgk::occupancy_for(b->precision, dgk::kThreadChoices[ti], p, b->lm, b->pipe[ti][p],
                                       b->smem[ti][p]);
  return b->occ[ti][p];
}

int grid_for(dg_batch* b, int ti, int p) {
  const int occ = occupancy_of(b, ti, p);
  if (occ <= 0) return 0;
  const int per_sm = b->ctas_per_sm > 0 ? std::min(b->ctas_per_sm, occ) : occ;
  return std::max(1, std::min(per_sm * b->sms, b->ntiles[ti][p]));
}

dg_status batch_launch(dg_batch* b, int ti, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int) * (dgk::kBatchMaxP + 1), s);
  if (e != cudaSuccess) return to_status(e);
  if (b->total_face_nodes > 0) {
    const long long blocks = (b->total_face_nodes + 255) / 256;
    if (b->precision == DG_FP32) {
      if (b->llf)
        dgk::batch_interface_kernel<float, true><<<(unsigned)blocks, 256, 0, s>>>(b->d_inst, b->n, b->total_face_nodes,
                                                                                 (float)b->gamma);
      else
        dgk::batch_interface_kernel<float, false><<<(unsigned)blocks, 256, 0, s>>>(b->d_inst, b->n,
                                                                                  b->total_face_nodes, (float)b->gamma);
    } else {
      if (b->llf)
        dgk::batch_interface_kernel<double, true><<<(unsigned)blocks, 256, 0, s>>>(b->d_inst, b->n,
                                                                                  b->total_face_nodes, b->gamma);
      else
        dgk::batch_interface_kernel<double, false><<<(unsigned)blocks, 256, 0, s>>>(b->d_inst, b->n,
                                                                                   b->total_face_nodes, b->gamma);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return to_status(e);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, s);
  for (int p = 1; p <= dgk::kBatchMaxP && e == cudaSuccess; ++p) {
    if (b->ntiles[ti][p] == 0) continue;
    const int grid = grid_for(b, ti, p);
    if (grid <= 0) return DG_ERR_CUDA;
    e = cudaStreamWaitEvent(b->streams[p], b->fork, 0);
    const dgk::BatchCall c{b->lm,  b->pipe[ti][p], true, b->d_inst, b->d_tiles[ti][p], b->ntiles[ti][p],
                           b->d_counter + p, b->gamma, b->smem[ti][p], grid, b->streams[p], nullptr};
    if (e == cudaSuccess) e = dgk::batch_volume(b->precision, dgk::kThreadChoices[ti], p, c);
    if (e == cudaSuccess) e = cudaEventRecord(b->join[p], b->streams[p]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join[p], 0);
  }
  return to_status(e);
}

}  // namespace

extern "C" {

dg_status dg_batch_create(dg_batch** out, dg_ctx* const* ctxs, int n, const double* const* u, double* const* du) {
  if (!out || !ctxs || !u || !du || n < 1 || n > 65536) return DG_ERR_ARG;
  *out = nullptr;
  const dg_ctx* c0 = ctxs[0];
  if (!c0) return DG_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    const dg_ctx* c = ctxs[i];
    if (!c || !u[i] || !du[i]) return DG_ERR_ARG;
    if (c->device != c0->device || c->precision != c0->precision || c->surface_flux != c0->surface_flux ||
        c->gamma != c0->gamma || c->var.lm != c0->var.lm || (c->var.pipe != 0) != (c0->var.pipe != 0))
      return DG_ERR_ARG;
    if (c->nd != 3 || c->p > dgk::kBatchMaxP || c->volume_flux != DG_VOL_RANOCHA || c->var.sh_pp != 0.0f ||
        c->var.ghost != 0 ||
        (c->var.lm != dgk::LM_SHARED_RCP && c->var.lm != dgk::LM_PRELOG) || c->nodes != DG_NODES_LGL)
      return DG_ERR_UNSUPPORTED;
    if (((uintptr_t)u[i] | (uintptr_t)du[i]) & 7) return DG_ERR_ARG;
    const size_t bytes = (size_t)c->state_len * sizeof(double);
    const char *ub = (const char*)u[i], *db = (const char*)du[i];
    if (ub < db + bytes && db < ub + bytes) return DG_ERR_ARG;
  }
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != c0->device) return DG_ERR_ARG;
  dg_batch* b = new (std::nothrow) dg_batch();
  if (!b) return DG_ERR_OOM;
  for (int ti = 0; ti < dgk::kNumThreadChoices; ++ti)
    for (int p = 0; p <= dgk::kBatchMaxP; ++p) b->occ[ti][p] = -1;
  b->device = c0->device;
  b->n = n;
  b->precision = c0->precision;
  b->llf = c0->surface_flux == DG_SURF_EC_LLF;
  b->gamma = c0->gamma;
  b->lm = c0->var.lm;
  cudaError_t e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) e = dgk::ensure_const_ops(b->device);
  if (e != cudaSuccess) {
    batch_release(b);
    return to_status(e);
  }
  std::vector<dgk::BatchInst> inst(n);
  int hist[dgk::kBatchMaxP + 1] = {0};
  long long elems = 0;
  for (int i = 0; i < n; ++i) {
    const dg_ctx* c = ctxs[i];
    dgk::BatchInst& bi = inst[i];
    bi.u = u[i];
    bi.du = du[i];
    bi.Ja = c->precision == DG_FP32 ? (const void*)c->d_Ja32 : (const void*)c->d_Ja;
    bi.invJ = c->d_invJ;
    bi.face = c->d_face;
    bi.flag = c->d_flag;
    bi.md = c->md;
    bi.p = c->p;
    bi.face_begin = b->total_face_nodes;
    b->total_face_nodes += 3LL * c->E * c->N * c->N;
    hist[c->p]++;
    elems += c->E;
  }
  char sig[256];
  snprintf(sig, sizeof(sig), "%s%s n=%d E=%lld p1-5=%d,%d,%d,%d,%d", c0->precision == DG_FP32 ? "fp32" : "fp64",
           b->lm == dgk::LM_PRELOG ? " logs" : "", n, elems, hist[1], hist[2], hist[3], hist[4], hist[5]);
  b->signature = sig;
  // tile lists per CTA size and degree; full tiles first, the instances' ragged last tiles at the end
  for (int ti = 0; ti < dgk::kNumThreadChoices && e == cudaSuccess; ++ti) {
    const int threads = dgk::kThreadChoices[ti];
    for (int p = 1; p <= dgk::kBatchMaxP && e == cudaSuccess; ++p) {
      if (hist[p] == 0) continue;
      const bool logs = b->lm == dgk::LM_PRELOG;
      const int epb = dgk::batch_epb(p, b->precision, threads, logs);
      std::vector<dgk::BatchTile> full, ragged;
      for (int i = 0; i < n; ++i) {
        if (ctxs[i]->p != p) continue;
        for (int e0 = 0; e0 < ctxs[i]->md.E; e0 += epb)
          (ctxs[i]->md.E - e0 >= epb ? full : ragged).push_back(dgk::BatchTile{i, e0});
      }
      full.insert(full.end(), ragged.begin(), ragged.end());
      b->ntiles[ti][p] = (int)full.size();
      b->smem[ti][p] = dgk::batch_smem(p, b->precision, threads, logs);
      // the pipelined kernel with the default log mean and pipelined staging, except FP32 at p = 2 (slower there)
      b->pipe[ti][p] = c0->var.pipe != 0 && !logs && !(b->precision == DG_FP32 && p == 2) &&
                       dgk::batch_pipe_fits(b->precision, threads, p);
      e = cudaMalloc(&b->d_tiles[ti][p], full.size() * sizeof(dgk::BatchTile));
      if (e == cudaSuccess)
        e = cudaMemcpy(b->d_tiles[ti][p], full.data(), full.size() * sizeof(dgk::BatchTile), cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->d_inst, n * sizeof(dgk::BatchInst));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_inst, inst.data(), n * sizeof(dgk::BatchInst), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int) * (dgk::kBatchMaxP + 1));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int p = 1; p <= dgk::kBatchMaxP && e == cudaSuccess; ++p) {
    if (hist[p] == 0) continue;
    e = cudaStreamCreateWithFlags(&b->streams[p], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[p], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    batch_release(b);
    return to_status(e);
  }
  *out = b;
  return DG_OK;
}

dg_status dg_batch_rhs(dg_batch* b, dg_stream_t stream) {
  if (!b) return DG_ERR_ARG;
  return batch_launch(b, b->threads_idx, (cudaStream_t)stream);
}

dg_status dg_batch_autotune(dg_batch* b, const char* cache_path, dg_stream_t stream, int* threads_out,
                            int* ctas_per_sm_out) {
  if (!b) return DG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  char devname[256] = "device";
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, b->device) == cudaSuccess) snprintf(devname, sizeof(devname), "%s", prop.name);
  const std::string key = std::string(devname) + " | " + b->signature;
  // cached choice: lines "key<TAB>threads<TAB>ctas_per_sm"
  if (cache_path) {
    FILE* f = fopen(cache_path, "r");
    if (f) {
      char line[1024];
      while (fgets(line, sizeof(line), f)) {
        char* tab = strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        int th = 0, cps = 0;
        if (key == line && sscanf(tab + 1, "%d\t%d", &th, &cps) == 2) {
          for (int ti = 0; ti < dgk::kNumThreadChoices; ++ti)
            if (dgk::kThreadChoices[ti] == th) {
              b->threads_idx = ti;
              b->ctas_per_sm = cps;
            }
          fclose(f);
          if (threads_out) *threads_out = dgk::kThreadChoices[b->threads_idx];
          if (ctas_per_sm_out) *ctas_per_sm_out = b->ctas_per_sm;
          return DG_OK;
        }
      }
      fclose(f);
    }
  }
  cudaEvent_t t0, t1;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e != cudaSuccess) return to_status(e);
  float best = 1e30f;
  int best_ti = b->threads_idx, best_cps = b->ctas_per_sm;
  dg_status st = DG_OK;
  for (int ti = 0; ti < dgk::kNumThreadChoices && st == DG_OK; ++ti) {
    int occ = 0;  // the largest occupancy limit over the degrees present (cps is capped per degree)
    for (int p = 1; p <= dgk::kBatchMaxP; ++p)
      if (b->ntiles[ti][p] > 0)
        occ = std::max(occ, occupancy_of(b, ti, p));
    for (int cps = 1; cps <= occ && st == DG_OK; ++cps) {
      b->ctas_per_sm = cps;
      st = batch_launch(b, ti, s);  // warm-up
      cudaEventRecord(t0, s);
      for (int r = 0; r < 3 && st == DG_OK; ++r) st = batch_launch(b, ti, s);
      cudaEventRecord(t1, s);
      if (st != DG_OK) break;
      if (cudaEventSynchronize(t1) != cudaSuccess) {
        st = DG_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (ms < best) {
        best = ms;
        best_ti = ti;
        best_cps = cps;
      }
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  b->threads_idx = best_ti;
  b->ctas_per_sm = best_cps;
  if (st != DG_OK) return st;
  if (cache_path) {
    FILE* f = fopen(cache_path, "a");
    if (f) {
      fprintf(f, "%s\t%d\t%d\n", key.c_str(), dgk::kThreadChoices[best_ti], best_cps);
      fclose(f);
    }
  }
  if (threads_out) *threads_out = dgk::kThreadChoices[best_ti];
  if (ctas_per_sm_out) *ctas_per_sm_out = best_cps;
  return DG_OK;
}

dg_status dg_batch_set_tuning(dg_batch* b, int threads, int ctas_per_sm) {
  if (!b || ctas_per_sm < 0) return DG_ERR_ARG;
  for (int ti = 0; ti < dgk::kNumThreadChoices; ++ti)
    if (dgk::kThreadChoices[ti] == threads) {
      b->threads_idx = ti;
      b->ctas_per_sm = ctas_per_sm;
      return DG_OK;
    }
  return DG_ERR_ARG;
}

void dg_batch_free(dg_batch* b) { batch_release(b); }

}  // extern "C"
