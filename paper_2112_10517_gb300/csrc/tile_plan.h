// Tile schedule of the pipelined volume kernel: which elements each tile holds and in which order the persistent
// CTAs take the tiles. Plain C++ (no CUDA types), shared by the launcher (host), the kernel (device) and a host
// test that compiles this header alone.
//
// Round-robin: tile t holds elements [e0 + t EPB, e0 + (t + 1) EPB) (the last one fewer), and CTA b takes tiles b,
// b + grid, b + 2 grid, ... Counter: the first `grid` tiles are taken round-robin (each CTA's first tile, whose
// metric terms it copies before the wait for the kernel ahead of it), the rest one ahead from a per-context counter;
// tiles t < nfull hold EPB elements, the tiles after them EPB/2 (the mesh's last round, cut in half tiles).
//
// The kernel ends when its busiest SM does. Round-robin gives an SM up to ceil(tiles / SMs) full tiles; the counter
// lets SMs whose CTAs finish early take more tiles and balances the SMs to about a half tile, ceil(half tiles / SMs).
// Each schedule's efficiency is its mean load per SM over that maximum; the counter is taken where it is higher by
// more than the counter's own cost (the atomic fetches and the half tiles' barriers: about 1 % of a launch), where
// every CTA has at least two full tiles, and where the caller allows it (`allowed`: half tiles that fill whole
// warps, a counter present).
#pragma once

#if defined(__CUDACC__)
#define DG_TILE_PLAN_FN __host__ __device__ __forceinline__
#else
#define DG_TILE_PLAN_FN inline
#endif

namespace dgk {

struct TilePlan {
  int ntiles;    // tiles of the launch
  int nfull;     // tiles of EPB elements before the half tiles (ntiles: none)
  bool counter;  // tiles after the first `grid` from the counter
};

// elems: elements computed (from the first one on); epb: elements per full tile; grid: persistent CTAs; sms: SMs.
DG_TILE_PLAN_FN TilePlan tile_plan(int elems, int epb, int grid, int sms, bool allowed) {
  TilePlan p;
  p.ntiles = (elems + epb - 1) / epb;
  p.nfull = p.ntiles;
  p.counter = false;
  if (!allowed || epb < 2 || grid < 1 || sms < 1 || elems / epb < 2 * grid) return p;
  const int half = epb / 2;
  const int halves = (elems + half - 1) / half;
  const double eff_rr = (double)p.ntiles / ((double)sms * ((p.ntiles + sms - 1) / sms));
  const double eff_counter = (double)halves / ((double)sms * ((halves + sms - 1) / sms));
  if (eff_counter > eff_rr + 0.01) {
    p.nfull = elems / epb - grid;
    p.ntiles = p.nfull + (elems - p.nfull * epb + half - 1) / half;
    p.counter = true;
  }
  return p;
}

// The elements of tile t: the first, relative to the first element computed, and the count (at most epb; the last
// tile may hold fewer, up to `elems`).
DG_TILE_PLAN_FN void tile_range(int nfull, int epb, int elems, int t, int& first, int& count) {
  const int half = epb / 2 > 0 ? epb / 2 : 1;
  int n;
  if (t < nfull) {
    first = t * epb;
    n = epb;
  } else {
    first = nfull * epb + (t - nfull) * half;
    n = half;
  }
  count = elems - first < n ? elems - first : n;
}

}  // namespace dgk
