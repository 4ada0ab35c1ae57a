// Pipelined volume kernel (Eq. fluxdiff-SBP-opDsplit, the same arithmetic as volume_tile):
// persistent CTAs take element tiles round-robin, t = blockIdx.x, blockIdx.x + gridDim.x, ... (or, FP64 where the
// launcher predicts an earlier end, from a counter with a half-tile last round: MeshTileSource); one thread copies the tiles'
// data into shared memory with bulk asynchronous copies (cp.async.bulk, the TMA engine), each group of arrays
// completing on its own mbarrier. A tile runs in three phases -- A: node quantities from the stage input,
// B: the two-point fluxes along lines, whose sums start from the lifted interface fluxes (metric terms, faces),
// C: -1/J, store or stage update (1/J, the Runge-Kutta operands) -- and each group is copied for the NEXT tile as soon as the
// phase that reads it has finished: the stage input during phases B and C, the metric terms during C and the next
// A, the phase-C group during the next A and B. One buffer per group keeps the shared memory per CTA, and so the
// number of resident CTAs, close to that of the per-tile kernel, while the loads overlap computation: the FP32
// kernel is bound by their latency, the FP64 kernel by its FP64 pipe, which then also runs through phases A and C.
//
// With an even number of nodes per line every element block of every array is a multiple of 16 bytes, and thread
// 0 moves each group with a few bulk copies (16-byte-aligned arrays, checked by the launcher). With an odd number
// every thread copies part of the group with 4- or 8-byte asynchronous copies (cp.async), which the same
// mbarrier tracks (cp.async.mbarrier.arrive, one arrival per thread). The default log mean only. Waits on the
// mbarriers are bounded: on a timeout the CTA raises FLAG_WAIT_TIMEOUT, waits (bounded again, or for its own
// copies) for the copies in flight and returns.
#pragma once

#include "kernels.cuh"
#include "tile_plan.h"

namespace dgk {

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the asynchronous proxy (the bulk-copy engine)
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// arrive once (the barrier's expected count is 1) and add `bytes` to the transaction count of the current phase
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// 4-byte asynchronous copy (cp.async; the 8-byte form is cp_async8)
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}

// the executing thread's cp.async copies issued so far arrive on `bar` once complete (the barrier's expected
// count includes this thread)
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// global -> shared bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned), completing on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// true once the phase of parity `parity` has completed (acquire: the copied data are then visible)
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Polls `bar` for the phase of parity `parity` at most kPolls times, about 64 ns apart (about half a second).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  constexpr int kPolls = 1 << 23;
  for (int i = 0; i < kPolls; ++i) {
    if (mbar_test(bar, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

// Shared memory of the pipelined kernel, for EPB elements: the copied groups
//   IN [EPB][NV][NDOF] f64 (stage input)                                         mbarrier 0
//   JA [EPB][ND][ND][NDOF] T (metric terms; not copied on Cartesian meshes), FC [2][ND][EPB][NV][NL] T (the
//   lifted interface fluxes; side 0: the upper face of the lower neighbour, side 1: the element's own)
//                                                                                  mbarrier 1
//   IJ [EPB][NDOF] f64 (1/J; not on Cartesian meshes), EU, EY [EPB][NV][NDOF] f64
//   (fused stage update: u, and acc (RK4) / K (CK45) after stage 0)              mbarrier 2
// then the tile scratch, node quantities [EPB][NQ][NDOF] T and per-direction sums [EPB][ND][NV][NDOF] T (each
// element's block followed by kElemPad bytes), then the three mbarriers. Each region starts on a 16-byte boundary (for even N every element block is a multiple of 16
// bytes already).
template <int ND, int N, typename T>
struct PipeSmem {
  using G = Geo<ND, N>;
  static constexpr bool kBulk = N % 2 == 0;  // bulk (TMA) copies; else per-thread cp.async
  __host__ __device__ static constexpr size_t r16(size_t x) { return (x + 15) / 16 * 16; }
  static constexpr size_t kIn = (size_t)G::NV * G::NDOF * sizeof(double);
  static constexpr size_t kJa = (size_t)ND * ND * G::NDOF * sizeof(T);
  static constexpr size_t kInvJ = (size_t)G::NDOF * sizeof(double);
  static constexpr size_t kFace = (size_t)G::NV * G::NL * sizeof(T);  // one face of one element
  // 5 words between the scratch blocks of consecutive elements (4-byte T, ND = 3, N = 4): a phase-B warp holds
  // lines of one direction for two elements, and the pad moves the second element's plane onto other banks
  static constexpr size_t kElemPad = (ND == 3 && N == 4 && sizeof(T) == 4) ? 20 : 0;
  static constexpr size_t kPrim = (size_t)NodeQ<ND>::NQ * G::NDOF * sizeof(T) + kElemPad;
  static constexpr size_t kAcc = (size_t)ND * G::NV * G::NDOF * sizeof(T) + kElemPad;
  static constexpr int kPrimT = (int)(kPrim / sizeof(T)), kAccT = (int)(kAcc / sizeof(T));  // element strides
  // byte offsets of the regions for EPB elements
  __host__ __device__ static constexpr size_t off_ja(int epb) { return r16((size_t)epb * kIn); }
  __host__ __device__ static constexpr size_t off_ij(int epb) { return off_ja(epb) + r16((size_t)epb * kJa); }
  __host__ __device__ static constexpr size_t off_eu(int epb) { return off_ij(epb) + r16((size_t)epb * kInvJ); }
  __host__ __device__ static constexpr size_t off_ey(int epb, bool fused) { return off_eu(epb) + (fused ? r16(epb * kIn) : 0); }
  __host__ __device__ static constexpr size_t off_fc(int epb, bool fused) { return off_ey(epb, fused) + (fused ? r16(epb * kIn) : 0); }
  __host__ __device__ static constexpr size_t off_prim(int epb, bool fused) { return off_fc(epb, fused) + r16((size_t)2 * ND * epb * kFace); }
  __host__ __device__ static constexpr size_t off_acc(int epb, bool fused) { return off_prim(epb, fused) + r16((size_t)epb * kPrim); }
  __host__ __device__ static constexpr size_t off_bar(int epb, bool fused) { return off_acc(epb, fused) + r16((size_t)epb * kAcc); }
  __host__ __device__ static constexpr size_t bytes(int epb, bool fused) { return off_bar(epb, fused) + 32; }
  static_assert(!kBulk || (kIn % 16 == 0 && kJa % 16 == 0 && kInvJ % 16 == 0 && kFace % 16 == 0),
                "bulk copies move multiples of 16 bytes");
};

// True when the lower neighbours across direction n of the consecutive elements e0 .. e0+nel-1 are consecutive
// too. An element's neighbour is e - s_n (s_n the element stride along n) when its coordinate c_n > 0 and
// e + (len_n - 1) s_n when c_n = 0: the map is one translation when all elements share the group e / s_n, when
// len_n = 1, or when no element of the range has c_n = 0.
__device__ __forceinline__ bool lower_neighbors_consecutive(const MeshDims& md, int e0, int nel, int n) {
  if (nel == 1) return true;
  const int s = n == 0 ? 1 : (n == 1 ? md.n1 : md.n1 * md.n2);
  const int len = n == 0 ? md.n1 : (n == 1 ? md.n2 : md.n3);
  const int g0 = e0 / s, g1 = (e0 + nel - 1) / s;
  return g0 == g1 || len == 1 || (g0 % len != 0 && g0 / len == g1 / len);
}

// Waits (bounded) for the last of `fills` fills of `bar`, if any: the drain of the copies in flight on a timeout.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, int fills) {
  if (fills > 0) mbar_wait_bounded(bar, (unsigned)((fills - 1) & 1));
}

// Resident CTAs per SM that the register budget is set for (65536 / (CTAs x threads) registers per thread): as
// many as the shared memory of a fused-update kernel admits (228 KB per SM, 1 KB of it reserved per CTA), at most
// 2048 threads.
template <int ND, int N, typename T, int EPB>
constexpr int pipe_min_ctas() {
  constexpr size_t smem = PipeSmem<ND, N, T>::bytes(EPB, true) + 1024;
  constexpr int by_smem = (int)((228 * 1024) / smem);
  constexpr int by_threads = 2048 / (EPB * Geo<ND, N>::TPE);
  constexpr int n = by_smem < by_threads ? by_smem : by_threads;
  return n < 1 ? 1 : n;
}

// Where a tile's data live: the arrays of its mesh and its first element.
template <typename T>
struct PipeTile {
  const double* in;   // stage input [E][NV][NDOF]
  const T* Ja;        // metric terms [E][ND][ND][NDOF]
  const double* invJ;  // 1/J [E][NDOF]
  const T* face;      // lifted interface fluxes [ND][E][NV][NL]
  double* du;         // output (stored RHS)
  int* flag;          // the mesh's status flag
  MeshDims md;
  int e0;
  int nel;  // elements in the tile (at most EPB; the mesh's last tile may hold fewer still)
};

// The tiles of one mesh (first and next are called by thread 0, which passes the index on through shared memory).
// Tiles t < nfull hold EPB elements from element mesh.e0 + t EPB (mesh.e0: the first element computed, past a
// partition's ghost layer), the tiles after them EPB/2 elements each (the mesh's last round).
// dyn == nullptr: round-robin over the persistent grid, t = blockIdx.x, blockIdx.x + gridDim.x, ...
// dyn != nullptr: each CTA's first tile is blockIdx.x, the following ones are taken from the counter dyn[0] (one
// tile ahead), so that SMs whose CTAs finish early take more tiles; with the half-size tiles of the last round the
// SMs finish within about a half tile of one another. The round-robin grid instead finishes with whole tiles on some
// SMs only (the time of ceil(tiles / SM) rounds). The last CTA to finish resets dyn[0] and its count dyn[1].
template <typename T, int EPB>
struct MeshTileSource {
  PipeTile<T> mesh;
  int ntiles;
  int nfull;
  int* dyn;
  __device__ __forceinline__ int first() const { return blockIdx.x; }
  __device__ __forceinline__ int next(int t) const { return dyn ? (int)gridDim.x + atomicAdd(dyn, 1) : t + gridDim.x; }
  __device__ __forceinline__ bool valid(int t) const { return t < ntiles; }
  __device__ __forceinline__ PipeTile<T> tile(int t) const {
    PipeTile<T> r = mesh;
    int first;
    tile_range(nfull, EPB, mesh.md.E - mesh.e0, t, first, r.nel);
    r.e0 = mesh.e0 + first;
    return r;
  }
  // by thread 0 of each CTA after its last fetch: the counter's fetches are ordered before the count of finished
  // CTAs, so the last CTA resets the counter after every fetch of this launch
  __device__ __forceinline__ void finish() const {
    if (!dyn) return;
    __threadfence();
    if (atomicAdd(dyn + 1, 1) == (int)gridDim.x - 1) {
      atomicExch(dyn, 0);
      atomicExch(dyn + 1, 0);
    }
  }
};

// The tile loop of the pipelined kernel over the tiles of `src` (MeshTileSource, or the batch's dynamic source).
template <int ND, int N, typename T, int EPB, int EPI, class Src>
__device__ __forceinline__ void pipe_tiles(const Src& src, const OpTable<N, T>& op, T gamma, const Epilogue& epi,
                                           const Variant& var) {
  using G = Geo<ND, N>;
  using S = PipeSmem<ND, N, T>;
  constexpr int NQ = NodeQ<ND>::NQ;
  constexpr bool kFused = EPI != EPI_STORE;
  constexpr int kThreads = EPB * G::TPE;
  constexpr int kFaceT = G::NV * G::NL;  // elements of T in one face block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // s_ok[j]: thread 0's wait before the j-th barrier of a tile succeeded (0: stage input, at the barrier that
  // closes the previous tile; 1: metric terms; 2: phase-C group). A slot is rewritten only after every thread has
  // passed the two barriers that follow its read.
  __shared__ int s_ok[3];
  __shared__ int s_tile[2];  // thread 0's tile indices: [0] the first, [1] the next (read after the tile's first
                             // barrier, rewritten after its third)
  double* s_in = reinterpret_cast<double*>(smem_raw);
  T* s_ja = reinterpret_cast<T*>(smem_raw + S::off_ja(EPB));
  double* s_ij = reinterpret_cast<double*>(smem_raw + S::off_ij(EPB));
  double* s_eu = reinterpret_cast<double*>(smem_raw + S::off_eu(EPB));
  double* s_ey = reinterpret_cast<double*>(smem_raw + S::off_ey(EPB, kFused));
  T* s_fc = reinterpret_cast<T*>(smem_raw + S::off_fc(EPB, kFused));
  T* s_prim = reinterpret_cast<T*>(smem_raw + S::off_prim(EPB, kFused));
  T* s_acc = reinterpret_cast<T*>(smem_raw + S::off_acc(EPB, kFused));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + S::off_bar(EPB, kFused));
  const int tid = threadIdx.x;
  const T gm1 = gamma - T(1);
  const bool has_ja = !var.cart;
  const bool need_y = kFused && epi.stage > 0;  // acc (RK4) / K (CK45) are read after stage 0
  const double* gy = EPI == EPI_RK4 ? epi.acc : epi.y;
  int fill_in = 0, fill_ja = 0, fill_c = 0;  // issuing threads: fills issued per mbarrier

  // The copies of one group for the tile t: bulk mode, by thread 0 (byte count first, then the copies); cp.async
  // mode, by every thread (its share of each array, then its arrival on the group's barrier). Captures by value:
  // a kernel parameter captured by reference would be copied to local memory.
  auto copy = [=](auto* dst, const auto* src, int count, uint64_t* bar) {  // count values of src's type
    if constexpr (S::kBulk) {
      bulk_g2s(dst, src, (unsigned)(count * sizeof(*src)), bar);
    } else {
      for (int w = tid; w < count; w += kThreads) {
        if constexpr (sizeof(*src) == 8)
          cp_async8(dst + w, src + w);
        else
          cp_async4(dst + w, src + w);
      }
    }
  };
  auto tile_nel = [](const PipeTile<T>& tt) { return min(min(EPB, tt.nel), tt.md.E - tt.e0); };
  auto issue_in = [=](const PipeTile<T>& tt) {
    const int e0 = tt.e0, nel = tile_nel(tt);
    if constexpr (S::kBulk) mbar_expect_tx(&bars[0], (unsigned)(nel * S::kIn));
    copy(s_in, tt.in + (size_t)e0 * G::NV * G::NDOF, nel * G::NV * G::NDOF, &bars[0]);
    if constexpr (!S::kBulk) cp_async_arrive(&bars[0]);
  };
  // The metric group in two parts: the metric terms (curvilinear meshes; written once, at set-up), with the byte
  // count of the whole group, then the faces' lifted fluxes (written by the interface kernel before this one).
  auto issue_ja_geo = [=](const PipeTile<T>& tt) {
    const int e0 = tt.e0, nel = tile_nel(tt);
    if constexpr (S::kBulk)
      mbar_expect_tx(&bars[1], (has_ja ? (unsigned)(nel * S::kJa) : 0u) + 2u * ND * (unsigned)(nel * S::kFace));
    if (has_ja) copy(s_ja, tt.Ja + (size_t)e0 * ND * ND * G::NDOF, nel * ND * ND * G::NDOF, &bars[1]);
  };
  auto issue_ja_dep = [=](const PipeTile<T>& tt) {
    const int e0 = tt.e0, nel = tile_nel(tt);
    const MeshDims& md = tt.md;
#pragma unroll
    for (int n = 0; n < ND; ++n) {
      // the tile's own upper faces along n are consecutive in the face array; the lower neighbours' mostly are
      const T* fn = tt.face + (size_t)n * md.E * kFaceT;
      copy(s_fc + ((1 * ND + n) * EPB) * kFaceT, fn + (size_t)e0 * kFaceT, nel * kFaceT, &bars[1]);
      if (lower_neighbors_consecutive(md, e0, nel, n)) {
        copy(s_fc + (n * EPB) * kFaceT, fn + (size_t)neighbor(md, e0, n, -1) * kFaceT, nel * kFaceT, &bars[1]);
      } else {
        for (int el = 0; el < nel; ++el)
          copy(s_fc + (n * EPB + el) * kFaceT, fn + (size_t)neighbor(md, e0 + el, n, -1) * kFaceT, kFaceT,
               &bars[1]);
      }
    }
    if constexpr (!S::kBulk) cp_async_arrive(&bars[1]);
  };
  // The phase-C group (may be empty), likewise: 1/J (curvilinear meshes) with the group's byte count, then the
  // stage update's operands.
  auto issue_c_geo = [=](const PipeTile<T>& tt) {
    const int e0 = tt.e0, nel = tile_nel(tt);
    if constexpr (S::kBulk)
      mbar_expect_tx(&bars[2], (has_ja ? (unsigned)(nel * S::kInvJ) : 0u) + (kFused ? (unsigned)(nel * S::kIn) : 0u) +
                                   (need_y ? (unsigned)(nel * S::kIn) : 0u));
    if (has_ja) copy(s_ij, tt.invJ + (size_t)e0 * G::NDOF, nel * G::NDOF, &bars[2]);
  };
  auto issue_c_dep = [=](const PipeTile<T>& tt) {
    const int e0 = tt.e0, nel = tile_nel(tt);
    const int nin = nel * G::NV * G::NDOF;
    const size_t so = (size_t)e0 * G::NV * G::NDOF;
    if (kFused) copy(s_eu, epi.u + so, nin, &bars[2]);
    if (need_y) copy(s_ey, gy + so, nin, &bars[2]);
    if constexpr (!S::kBulk) cp_async_arrive(&bars[2]);
  };
  auto issue_ja = [=](const PipeTile<T>& tt) {
    issue_ja_geo(tt);
    issue_ja_dep(tt);
  };
  auto issue_c = [=](const PipeTile<T>& tt) {
    issue_c_geo(tt);
    issue_c_dep(tt);
  };
  // the threads that issue copies: thread 0 in bulk mode, all in cp.async mode
  const bool issuer = S::kBulk ? tid == 0 : true;

  if (tid == 0) {
    for (int j = 0; j < 3; ++j) mbar_init(&bars[j], S::kBulk ? 1 : kThreads);
    mbar_init_fence();
    s_tile[0] = src.first();
  }
  __syncthreads();
  int t = s_tile[0];
  // The first tile: its geometry is copied before the wait for the kernels before this one in the stream (with a
  // programmatic launch, while the interface kernel's writes are made visible), its state and fluxes after it.
  if (issuer && src.valid(t)) {
    const PipeTile<T> ft = src.tile(t);
    issue_ja_geo(ft);
    issue_c_geo(ft);
  }
  pdl_wait();
  if (issuer && src.valid(t)) {
    const PipeTile<T> ft = src.tile(t);
    issue_in(ft);
    issue_ja_dep(ft);
    issue_c_dep(ft);
    fill_in = fill_ja = fill_c = 1;
  }
  if (tid == 0 && src.valid(t)) s_ok[0] = mbar_wait_bounded(&bars[0], 0u) ? 1 : 0;
  __syncthreads();
  bool failed = false;
  int* flag = nullptr;  // the current tile's mesh flag (a wait that ran out is reported there)
  for (int k = 0; src.valid(t); ++k) {
    const unsigned par = (unsigned)(k & 1);  // every group is copied once per tile
    const PipeTile<T> cur = src.tile(t);
    const int e0 = cur.e0, nel = tile_nel(cur);
    flag = cur.flag;
    if (tid == 0) s_tile[1] = src.next(t);
    if (!s_ok[0]) {  // all threads read the same slot: the whole CTA leaves the loop
      failed = true;
      break;
    }
    mbar_test(&bars[0], par);  // completed: each thread's own acquire of the copied data

    // ---- A: node quantities from the staged input (a partial last round falls to the last warps, not to warp 0,
    // which also issues the copies)
    bool ok = true;
    for (int idx = kThreads - 1 - tid; idx < nel * G::NDOF; idx += kThreads) {
      const int el = idx / G::NDOF, i = idx - el * G::NDOF;
      double uc[G::NV];
#pragma unroll
      for (int c = 0; c < G::NV; ++c) uc[c] = s_in[(el * G::NV + c) * G::NDOF + i];
      T q[NQ];
      ok &= node_quantities<ND, T>(uc, gm1, T(2) / gm1, q, nullptr, var.sh_eh, var.sh_el, var.sh_pp,
                                   sizeof(T) == 8 && var.flux == 0);  // beta = rho/p as line_pairs' kBeta
#pragma unroll
      for (int c = 0; c < NQ; ++c) s_prim[el * S::kPrimT + c * G::NDOF + i] = q[c];
    }
    if (!ok) atomicOr(flag, FLAG_NONPHYSICAL);
    if (tid == 0) s_ok[1] = mbar_wait_bounded(&bars[1], par) ? 1 : 0;
    __syncthreads();
    if (!s_ok[1]) {  // all threads read the same slot: the whole CTA leaves the loop
      failed = true;
      break;
    }
    mbar_test(&bars[1], par);
    const int tn = s_tile[1];
    const bool has_next = src.valid(tn);
    if constexpr (DG_VOLUME_EARLY_TRIGGER && sizeof(T) == 8)
      if (!has_next) pdl_trigger();  // this CTA's last tile: the dependent grid may be scheduled
    const PipeTile<T> nxt = src.tile(has_next ? tn : t);
    if (issuer && has_next) {  // the stage input has been read
      issue_in(nxt);
      ++fill_in;
    }

    // ---- B: the pairs i < k of each line, as in volume_tile; the end nodes' sums start from the lifted fluxes of
    // the line's two face points (face node l of the faces normal to n)
    // direction-major threads: n = tid / (EPB NL), then the element, then the line
    const int n = tid / (EPB * G::NL), r = tid - n * (EPB * G::NL);
    const int el = r / G::NL, l = r - el * G::NL;
    if (el < nel) {
      const int st = G::stride(n), lb = G::line_base(n, l);
      int so[N];
#pragma unroll
      for (int k = 0; k < N; ++k) so[k] = k * st;
      const T* sp = s_prim + el * S::kPrimT + lb;
      const T* sj = s_ja + (el * ND + n) * ND * G::NDOF + lb;
      T* sa = s_acc + el * S::kAccT + n * G::NV * G::NDOF + lb;
      const T* fu = s_fc + ((1 * ND + n) * EPB + el) * kFaceT + l;
      const T* fl = s_fc + ((0 * ND + n) * EPB + el) * kFaceT + l;
      const T n2n = T(2) * to_flux<T>(cart_jn(var, n));
      const T pp0 = T(var.sh_pp), c2 = T(2) / gm1;
      switch (var.flux * 2 + var.cart) {
        case 0: line_pairs<ND, N, T, 0, false>(sp, so, sj, nullptr, st, n, n2n, op, sa, fu, fl, pp0, c2); break;
        case 1: line_pairs<ND, N, T, 0, true>(sp, so, sj, nullptr, st, n, n2n, op, sa, fu, fl, pp0, c2); break;
        case 2: line_pairs<ND, N, T, 1, false>(sp, so, sj, nullptr, st, n, n2n, op, sa, fu, fl, pp0); break;
        default: line_pairs<ND, N, T, 1, true>(sp, so, sj, nullptr, st, n, n2n, op, sa, fu, fl, pp0); break;
      }
    }
    if (tid == 0) s_ok[2] = mbar_wait_bounded(&bars[2], par) ? 1 : 0;
    __syncthreads();
    if (!s_ok[2]) {  // all threads read the same slot: the whole CTA leaves the loop
      failed = true;
      break;
    }
    mbar_test(&bars[2], par);
    if (issuer && has_next) {  // the metric terms and face fluxes have been read
      issue_ja(nxt);
      ++fill_ja;
    }

    // ---- C: sum the directions, scale by -1/J, store or update (reversed thread order as in phase A)
    for (int idx = kThreads - 1 - tid; idx < nel * G::NDOF; idx += kThreads) {
      const int el = idx / G::NDOF, i = idx - el * G::NDOF;
      T tot[G::NV];
#pragma unroll
      for (int c = 0; c < G::NV; ++c) {
        T s = T(0);
#pragma unroll
        for (int n = 0; n < ND; ++n) s += s_acc[el * S::kAccT + (n * G::NV + c) * G::NDOF + i];
        tot[c] = s;
      }
      const double ij = var.cart ? var.invJ : s_ij[el * G::NDOF + i];
      const double sj = -ij;
      const T sjT = sizeof(T) == 8 ? T(0) : -to_flux<T>(ij);
      const size_t off = (size_t)(e0 + el) * G::NV * G::NDOF + i;
      if constexpr (sizeof(T) == 8 && EPI != EPI_STORE) {  // FP64: -1/J folded into the stage weights
        double w1, w2;
        stage_weights<EPI>(epi, sj, w1, w2);
#pragma unroll
        for (int c = 0; c < G::NV; ++c) {
          const int so = (el * G::NV + c) * G::NDOF + i;
          stage_update_w<EPI>(epi, off + (size_t)c * G::NDOF, (double)tot[c], w1, w2, s_eu[so],
                              need_y ? s_ey[so] : 0.0);
        }
      } else {
#pragma unroll
        for (int c = 0; c < G::NV; ++c) {
          const size_t o = off + (size_t)c * G::NDOF;
          const int so = (el * G::NV + c) * G::NDOF + i;
          // as in volume_tile: FP64 scaling, or the FP32 scaling and an exact integer-pipe widening
          const double kv = sizeof(T) == 8 ? sj * (double)tot[c] : f2d_int((float)(sjT * tot[c]));
          if (EPI == EPI_STORE)
            cur.du[o] = kv;
          else
            stage_update<EPI>(epi, o, kv, s_eu[so], need_y ? s_ey[so] : 0.0);
        }
      }
    }
    if (tid == 0 && has_next) s_ok[0] = mbar_wait_bounded(&bars[0], par ^ 1u) ? 1 : 0;
    __syncthreads();
    if (issuer && has_next) {  // the phase-C group has been read
      issue_c(nxt);
      ++fill_c;
    }
    t = tn;
  }
  if (failed) {  // a wait ran out: raise the flag, wait (bounded, or for the own copies) for the copies in flight
    if (tid == 0 && flag) atomicOr(flag, FLAG_WAIT_TIMEOUT);
    if constexpr (S::kBulk) {
      if (tid == 0) {
        mbar_drain(&bars[0], fill_in);
        mbar_drain(&bars[1], fill_ja);
        mbar_drain(&bars[2], fill_c);
      }
    } else {
      cp_async_wait_all();
    }
  }
  if (tid == 0) src.finish();
}

template <int ND, int N, typename T, int EPB, int EPI>
__global__ void __launch_bounds__(EPB* Geo<ND, N>::TPE, pipe_min_ctas<ND, N, T, EPB>())
    volume_pipe_kernel(const double* __restrict__ in, const T* __restrict__ Ja, const double* __restrict__ invJ,
                       const T* __restrict__ face, double* du, MeshDims md, OpTable<N, T> op, T gamma, int* flag,
                       Epilogue epi, Variant var, int ntiles, int nfull, int* dyn) {
  const MeshTileSource<T, EPB> src{{in, Ja, invJ, face, du, flag, md, var.ghost, EPB}, ntiles, nfull, dyn};
  pipe_tiles<ND, N, T, EPB, EPI>(src, op, gamma, epi, var);
}

}  // namespace dgk
