// Sweep tiles of the batched form (host code): the lines a sweep of one level processes,
// cut into runs, and the greedy packing of the runs into tiles of the sweep kernel.
//
// A sweep along x processes, for every patch, rows j of the patch (interior lines, whose
// edges count toward the CFL reduction and the interface fluxes) and, where the step needs
// them, ghost rows beside the patch: the two rows on each side on a refined level of the
// dimensionally split step (the y sweep reads the x sweep's state there) or one row on each
// side for the edge passes of the unsplit step. Along the line, the patch's extent is cut
// into parts of the tile length. A run is one part of all consecutive lines of one kind
// (ghost before, interior, ghost after) of one patch.
#include <algorithm>
#include <vector>
#include "mlswe_internal.h"

namespace mlswe {

void patch_segments(const Box& b, int dir, int tile_len, int g0, int g1, int desc, std::vector<SweepItem>& out) {
  const int a0 = dir == 0 ? b.i0 : b.j0, a1 = dir == 0 ? b.i1 : b.j1;  // along the lines
  const int lo = dir == 0 ? b.j0 : b.i0, hi = dir == 0 ? b.j1 : b.i1;  // across
  const int runs[3][3] = {{g0, lo, 0}, {lo, hi, 1}, {hi, g1, 0}};
  for (const auto& run : runs) {
    if (run[1] <= run[0]) continue;
    for (int a = a0; a < a1; a += tile_len) {
      SweepItem it;
      it.desc = desc;
      it.len = std::min(tile_len, a1 - a);
      if (dir == 0) { it.i0 = a; it.j0 = run[0]; } else { it.i0 = run[0]; it.j0 = a; }
      it.nlines = run[1] - run[0];
      it.flags = run[2] | (a + it.len == a1 ? 2 : 0);
      out.push_back(it);
    }
  }
}

bool pack_tiles(const std::vector<SweepItem>& segs, int dir, std::vector<SweepItem>& items, std::vector<int>& toff) {
  items.clear();
  toff.assign(1, 0);
  int used_e = 0, used_c = 0, ng = 0, desc = -1;
  auto close = [&]() {
    if (ng > 0) toff.push_back((int)items.size());
    used_e = used_c = ng = 0;
    desc = -1;
  };
  for (const SweepItem& sgm : segs) {
    if (sgm.len < 1 || sgm.len + 3 > kMaxEdges || sgm.len + 4 > kMaxCells) return false;  // a line fits no tile
    int left = sgm.nlines, first = 0;
    while (left > 0) {
      const int room = std::min((kMaxEdges - used_e) / (sgm.len + 3), (kMaxCells - used_c) / (sgm.len + 4));
      const int take = std::min(left, room);
      if (take < 1 || ng == kMaxGroups || (ng > 0 && sgm.desc != desc)) {
        close();
        continue;
      }
      SweepItem g = sgm;
      if (dir == 0) g.j0 = sgm.j0 + first; else g.i0 = sgm.i0 + first;
      g.nlines = take;
      items.push_back(g);
      ++ng;
      desc = sgm.desc;
      used_e += take * (sgm.len + 3);
      used_c += take * (sgm.len + 4);
      left -= take;
      first += take;
    }
  }
  close();
  return true;
}

}  // namespace mlswe
