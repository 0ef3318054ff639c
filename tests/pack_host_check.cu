// Host-side wrapper around the library's sweep-tile packing (compiled as host code by the
// test, no GPU needed) so that its runs and tiles can be checked from Python.
#include <vector>
#include "../paper_1803_01450_gb300/csrc/mlswe_internal.h"

extern "C" {

// Runs of one patch (i0, j0, i1, j1) for a sweep along dir: 6 ints per run (desc, i0, j0,
// len, nlines, flags) into out; returns the number of runs (at most cap written).
int pk_segments(int i0, int j0, int i1, int j1, int dir, int tile_len, int g0, int g1, int desc, int* out, int cap) {
  std::vector<mlswe::SweepItem> v;
  mlswe::patch_segments(mlswe::Box{i0, j0, i1, j1}, dir, tile_len, g0, g1, desc, v);
  for (int k = 0; k < (int)v.size() && k < cap; ++k) {
    const mlswe::SweepItem& s = v[k];
    int* o = out + 6 * k;
    o[0] = s.desc; o[1] = s.i0; o[2] = s.j0; o[3] = s.len; o[4] = s.nlines; o[5] = s.flags;
  }
  return (int)v.size();
}

// Packs n runs (6 ints each, as above): groups into items (6 ints each), tile offsets into
// toff; counts into counts[0] (groups) and counts[1] (tiles). Returns 0 when pack_tiles
// refuses the runs, -1 when the output arrays are too small, 1 otherwise.
int pk_pack(const int* segs, int n, int dir, int* items, int icap, int* toff, int tcap, int* counts) {
  std::vector<mlswe::SweepItem> in(n), out;
  for (int k = 0; k < n; ++k) {
    const int* s = segs + 6 * k;
    in[k].desc = s[0]; in[k].i0 = s[1]; in[k].j0 = s[2]; in[k].len = s[3]; in[k].nlines = s[4]; in[k].flags = s[5];
  }
  std::vector<int> off;
  if (!mlswe::pack_tiles(in, dir, out, off)) return 0;
  counts[0] = (int)out.size();
  counts[1] = (int)off.size() - 1;
  if ((int)out.size() > icap || (int)off.size() > tcap) return -1;
  for (int k = 0; k < (int)out.size(); ++k) {
    int* o = items + 6 * k;
    o[0] = out[k].desc; o[1] = out[k].i0; o[2] = out[k].j0; o[3] = out[k].len; o[4] = out[k].nlines;
    o[5] = out[k].flags;
  }
  for (int k = 0; k < (int)off.size(); ++k) toff[k] = off[k];
  return 1;
}
}
