// Host check of the pipelined volume kernel's tile schedule (paper_2112_10517_gb300/csrc/tile_plan.h, compiled
// alone): for each case read from stdin, "elems epb grid sms allowed", one JSON line with the plan and whether its
// tiles cover elements 0 .. elems-1 once each, in order, with at most epb elements per tile and, under the counter
// schedule, full first tiles for the grid's CTAs.
#include <cstdio>
#include <vector>

#include "tile_plan.h"

int main() {
  int elems, epb, grid, sms, allowed;
  while (std::scanf("%d %d %d %d %d", &elems, &epb, &grid, &sms, &allowed) == 5) {
    const dgk::TilePlan p = dgk::tile_plan(elems, epb, grid, sms, allowed != 0);
    std::vector<int> seen(elems > 0 ? elems : 0, 0);
    int next = 0, in_order = 1, sizes_ok = 1, first_full = 1;
    for (int t = 0; t < p.ntiles; ++t) {
      int first = -1, count = -1;
      dgk::tile_range(p.nfull, epb, elems, t, first, count);
      if (first != next) in_order = 0;
      if (count < 1 || count > epb || first < 0 || first + count > elems) {
        sizes_ok = 0;
        break;
      }
      for (int e = first; e < first + count; ++e) ++seen[e];
      if (p.counter && t < grid && count != epb) first_full = 0;
      next = first + count;
    }
    int once = next == elems;
    for (int e = 0; e < elems; ++e)
      if (seen[e] != 1) once = 0;
    std::printf("{\"elems\": %d, \"epb\": %d, \"grid\": %d, \"sms\": %d, \"allowed\": %d, \"ntiles\": %d, "
                "\"nfull\": %d, \"counter\": %d, \"once\": %d, \"in_order\": %d, \"sizes_ok\": %d, "
                "\"first_full\": %d}\n",
                elems, epb, grid, sms, allowed, p.ntiles, p.nfull, p.counter ? 1 : 0, once, in_order, sizes_ok,
                first_full);
  }
  return 0;
}
