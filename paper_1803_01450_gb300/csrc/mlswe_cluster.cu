// Host-side flag dilation and deterministic Berger-Rigoutsos clustering.
//
// The paper leaves flagging and clustering to GeoClaw's AMR (Sec. 2). This is
// the library's deterministic reading (integer arithmetic only, so any correct
// implementation of the same rules yields the same boxes):
//  * flags dilated by n_buf cells (Chebyshev distance);
//  * regions: level 0 -> the domain; refined level -> each patch shrunk by
//    n_nest cells on sides not on the domain boundary; each region alone;
//  * in a box: bounding box of its flags grown to min_len per side inside the
//    box (upper side first); accepted if flags/area >= eff and sides <= max_len;
//  * else split at the first signature hole (longer dimension first, x on
//    ties), else at the strongest sign change of the signature's second
//    difference (ties: dimension order, then lowest position), else at the
//    middle of the longer side; no part shorter than min_len; unsplittable
//    boxes are accepted;
//  * output sorted by (j0, i0).
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <vector>
#include "mlswe_internal.h"

namespace mlswe {

void dilate_flags(const uint8_t* in, int nx, int ny, int n, std::vector<uint8_t>& out) {
  // Separable max filter (a cell is set when its (2n + 1) x (2n + 1) window holds a flag):
  // along each row, the OR of the row shifted by -n .. n, then down the columns, the OR of
  // rows j - n .. j + n; every inner loop is a straight byte OR over a row (vectorised), and
  // both passes read memory in row order.
  std::vector<uint8_t> tmp((size_t)nx * ny, 0);
  out.assign((size_t)nx * ny, 0);
  for (int j = 0; j < ny; ++j) {
    const uint8_t* row = in + (size_t)j * nx;
    uint8_t* t = &tmp[(size_t)j * nx];
    for (int k = -n; k <= n; ++k) {
      const int i0 = std::max(0, -k), i1 = std::min(nx, nx - k);
      for (int i = i0; i < i1; ++i) t[i] |= row[i + k];
    }
  }
  for (int j = 0; j < ny; ++j) {
    uint8_t* o = &out[(size_t)j * nx];
    for (int k = std::max(0, j - n); k <= std::min(ny - 1, j + n); ++k) {
      const uint8_t* a = &tmp[(size_t)k * nx];
      for (int i = 0; i < nx; ++i) o[i] |= a[i];
    }
    for (int i = 0; i < nx; ++i) o[i] = o[i] != 0;
  }
}

namespace {

struct Grid {
  const uint8_t* f;
  int nx;
  bool at(int i, int j) const { return f[(size_t)j * nx + i] != 0; }
};

void cluster_box(const Grid& G, Box b, int min_len, int max_len, double eff, std::vector<Box>& out) {
  // bounding box of the flags in b
  int ti0 = b.i1, tj0 = b.j1, ti1 = b.i0 - 1, tj1 = b.j0 - 1;
  for (int j = b.j0; j < b.j1; ++j)
    for (int i = b.i0; i < b.i1; ++i)
      if (G.at(i, j)) {
        ti0 = std::min(ti0, i); tj0 = std::min(tj0, j);
        ti1 = std::max(ti1, i); tj1 = std::max(tj1, j);
      }
  if (ti1 < ti0) return;
  int t[4] = {ti0, tj0, ti1 + 1, tj1 + 1};
  const int bb[4] = {b.i0, b.j0, b.i1, b.j1};
  for (int d = 0; d < 2; ++d) {
    int lo = t[d], hi = t[d + 2];
    int need = min_len - (hi - lo);
    if (need > 0) {
      const int up = std::min(need, bb[d + 2] - hi);
      hi += up;
      need -= up;
      lo -= std::min(need, lo - bb[d]);
    }
    t[d] = lo; t[d + 2] = hi;
  }
  const Box T{t[0], t[1], t[2], t[3]};
  const int w = T.w(), h = T.h();
  std::vector<long long> sx(w, 0), sy(h, 0);
  long long nflag = 0;
  for (int j = T.j0; j < T.j1; ++j)
    for (int i = T.i0; i < T.i1; ++i)
      if (G.at(i, j)) { sx[i - T.i0]++; sy[j - T.j0]++; nflag++; }
  if ((double)nflag >= eff * (double)w * (double)h && w <= max_len && h <= max_len) {
    out.push_back(T);
    return;
  }
  const int order[2] = {w >= h ? 0 : 1, w >= h ? 1 : 0};
  const std::vector<long long>* sig[2] = {&sx, &sy};
  const int lo_of[2] = {T.i0, T.j0}, hi_of[2] = {T.i1, T.j1};
  int sd = -1, sp = 0;
  // (a) first hole
  for (int oi = 0; oi < 2 && sd < 0; ++oi) {
    const int d = order[oi];
    const int lo = lo_of[d], hi = hi_of[d];
    for (int p = lo + min_len; p <= hi - min_len; ++p)
      if ((*sig[d])[p - lo] == 0) { sd = d; sp = p; break; }
  }
  // (b) strongest sign change of the second difference
  if (sd < 0) {
    long long best_str = -1;
    int best_rank = 0, best_p = 0, best_d = -1;
    for (int oi = 0; oi < 2; ++oi) {
      const int d = order[oi];
      const std::vector<long long>& S = *sig[d];
      const int lo = lo_of[d], hi = hi_of[d], n = hi - lo;
      if (n < 4) continue;
      for (int k = 1; k <= n - 3; ++k) {
        const long long a = S[k - 1] - 2 * S[k] + S[k + 1];
        const long long c = S[k] - 2 * S[k + 1] + S[k + 2];
        const int p = lo + k + 1;
        if (a * c < 0 && p >= lo + min_len && p <= hi - min_len) {
          const long long str = std::llabs(c - a);
          const bool better = best_d < 0 || str > best_str ||
                              (str == best_str && (oi < best_rank || (oi == best_rank && p < best_p)));
          if (better) { best_str = str; best_rank = oi; best_p = p; best_d = d; }
        }
      }
    }
    if (best_d >= 0) { sd = best_d; sp = best_p; }
  }
  // (c) bisect the longer side
  if (sd < 0) {
    for (int oi = 0; oi < 2 && sd < 0; ++oi) {
      const int d = order[oi];
      const int lo = lo_of[d], hi = hi_of[d];
      const int p = lo + (hi - lo) / 2;
      if (p - lo >= min_len && hi - p >= min_len) { sd = d; sp = p; }
    }
  }
  if (sd < 0) { out.push_back(T); return; }
  if (sd == 0) {
    cluster_box(G, Box{T.i0, T.j0, sp, T.j1}, min_len, max_len, eff, out);
    cluster_box(G, Box{sp, T.j0, T.i1, T.j1}, min_len, max_len, eff, out);
  } else {
    cluster_box(G, Box{T.i0, T.j0, T.i1, sp}, min_len, max_len, eff, out);
    cluster_box(G, Box{T.i0, sp, T.i1, T.j1}, min_len, max_len, eff, out);
  }
}

}  // namespace

std::vector<Box> nest_regions(int level, int nx, int ny, const std::vector<Box>& patches, int n_nest) {
  std::vector<Box> out;
  if (level == 0) { out.push_back(Box{0, 0, nx, ny}); return out; }
  for (const Box& p : patches) {
    Box r{p.i0 == 0 ? 0 : p.i0 + n_nest, p.j0 == 0 ? 0 : p.j0 + n_nest,
          p.i1 == nx ? nx : p.i1 - n_nest, p.j1 == ny ? ny : p.j1 - n_nest};
    if (r.i1 > r.i0 && r.j1 > r.j0) out.push_back(r);
  }
  return out;
}

// Boxes of level+1 (fine indices, sorted by (j0, i0)) from the raw flags of `level`.
std::vector<Box> cluster_flags(const uint8_t* flags, int nx, int ny, int level, const std::vector<Box>& patches,
                               int r, int n_buf, double eff, int min_side, int max_side, int n_nest) {
  std::vector<uint8_t> dil;
  dilate_flags(flags, nx, ny, n_buf, dil);
  const int min_len = (min_side + r - 1) / r, max_len = max_side / r;
  std::vector<Box> boxes;
  std::vector<uint8_t> mask((size_t)nx * ny, 0);
  for (const Box& R : nest_regions(level, nx, ny, patches, n_nest)) {
    for (int j = R.j0; j < R.j1; ++j)
      for (int i = R.i0; i < R.i1; ++i) mask[(size_t)j * nx + i] = dil[(size_t)j * nx + i];
    Grid G{mask.data(), nx};
    cluster_box(G, R, min_len, max_len, eff, boxes);
    for (int j = R.j0; j < R.j1; ++j)
      for (int i = R.i0; i < R.i1; ++i) mask[(size_t)j * nx + i] = 0;
  }
  std::stable_sort(boxes.begin(), boxes.end(),
                   [](const Box& a, const Box& b) { return a.j0 != b.j0 ? a.j0 < b.j0 : a.i0 < b.i0; });
  for (Box& b : boxes) { b.i0 *= r; b.j0 *= r; b.i1 *= r; b.j1 *= r; }
  return boxes;
}

// Rectangles of `a` not covered by any box of `sub` (disjoint, deterministic order).
std::vector<Box> box_difference(const Box& a, const std::vector<Box>& sub) {
  std::vector<Box> cur{a};
  std::vector<Box> nxt;
  for (const Box& s : sub) {
    // a box that misses `a` misses every fragment of it (most of them, on a regrid)
    if (s.i1 <= a.i0 || s.i0 >= a.i1 || s.j1 <= a.j0 || s.j0 >= a.j1) continue;
    nxt.clear();
    for (const Box& c : cur) {
      const int i0 = std::max(c.i0, s.i0), j0 = std::max(c.j0, s.j0), i1 = std::min(c.i1, s.i1), j1 = std::min(c.j1, s.j1);
      if (i0 >= i1 || j0 >= j1) { nxt.push_back(c); continue; }
      if (c.j0 < j0) nxt.push_back(Box{c.i0, c.j0, c.i1, j0});
      if (j1 < c.j1) nxt.push_back(Box{c.i0, j1, c.i1, c.j1});
      if (c.i0 < i0) nxt.push_back(Box{c.i0, j0, i0, j1});
      if (i1 < c.i1) nxt.push_back(Box{i1, j0, c.i1, j1});
    }
    cur.swap(nxt);
  }
  return cur;
}

// The cells of `boxes` outside every box of `old`, as boxes: box_difference of each new box
// against the old boxes that can touch it, found through buckets of kBucket x kBucket cells
// (each old box is listed in every bucket it overlaps; candidates keep their order in `old`).
std::vector<Box> fresh_cells(const std::vector<Box>& boxes, const std::vector<Box>& old) {
  constexpr int kBucket = 64;
  int ni = 1, nj = 1;
  for (const Box& b : old) {
    ni = std::max(ni, (b.i1 + kBucket - 1) / kBucket);
    nj = std::max(nj, (b.j1 + kBucket - 1) / kBucket);
  }
  std::vector<std::vector<int>> bucket((size_t)ni * nj);
  for (int k = 0; k < (int)old.size(); ++k) {
    const Box& b = old[k];
    for (int bj = b.j0 / kBucket; bj <= (b.j1 - 1) / kBucket; ++bj)
      for (int bi = b.i0 / kBucket; bi <= (b.i1 - 1) / kBucket; ++bi) bucket[(size_t)bj * ni + bi].push_back(k);
  }
  std::vector<Box> out, cand;
  std::vector<int> idx;
  std::vector<char> seen(old.size(), 0);
  for (const Box& a : boxes) {
    idx.clear();
    const int bj1 = std::min(nj - 1, (a.j1 - 1) / kBucket), bi1 = std::min(ni - 1, (a.i1 - 1) / kBucket);
    for (int bj = a.j0 / kBucket; bj <= bj1; ++bj)
      for (int bi = a.i0 / kBucket; bi <= bi1; ++bi)
        for (int k : bucket[(size_t)bj * ni + bi])
          if (!seen[k]) { seen[k] = 1; idx.push_back(k); }
    std::sort(idx.begin(), idx.end());
    cand.clear();
    for (int k : idx) { cand.push_back(old[k]); seen[k] = 0; }
    const std::vector<Box> d = box_difference(a, cand);
    out.insert(out.end(), d.begin(), d.end());
  }
  return out;
}

}  // namespace mlswe
