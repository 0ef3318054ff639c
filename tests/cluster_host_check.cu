// Host-side wrapper around the library's flag dilation and clustering (compiled as host
// code by the test, no GPU needed) so that they can be compared with the oracle's.
#include <cstdint>
#include <vector>
#include "../paper_1803_01450_gb300/csrc/mlswe_internal.h"

namespace mlswe {
void dilate_flags(const uint8_t* in, int nx, int ny, int n, std::vector<uint8_t>& out);
std::vector<Box> cluster_flags(const uint8_t* flags, int nx, int ny, int level, const std::vector<Box>& patches,
                               int r, int n_buf, double eff, int min_side, int max_side, int n_nest);
std::vector<Box> fresh_cells(const std::vector<Box>& boxes, const std::vector<Box>& old);
}

extern "C" {

void hc_dilate(const uint8_t* in, int nx, int ny, int n, uint8_t* out) {
  std::vector<uint8_t> o;
  mlswe::dilate_flags(in, nx, ny, n, o);
  for (size_t k = 0; k < o.size(); ++k) out[k] = o[k];
}

// Returns the number of boxes; writes at most cap boxes (i0, j0, i1, j1) to out.
int hc_cluster(const uint8_t* flags, int nx, int ny, int level, const int* patches, int npatch, int r, int n_buf,
               double eff, int min_side, int max_side, int n_nest, int* out, int cap) {
  std::vector<mlswe::Box> P;
  for (int k = 0; k < npatch; ++k)
    P.push_back(mlswe::Box{patches[4 * k], patches[4 * k + 1], patches[4 * k + 2], patches[4 * k + 3]});
  std::vector<mlswe::Box> b = mlswe::cluster_flags(flags, nx, ny, level, P, r, n_buf, eff, min_side, max_side, n_nest);
  for (int k = 0; k < (int)b.size() && k < cap; ++k) {
    out[4 * k] = b[k].i0; out[4 * k + 1] = b[k].j0; out[4 * k + 2] = b[k].i1; out[4 * k + 3] = b[k].j1;
  }
  return (int)b.size();
}


// Boxes of the cells of `boxes` outside every box of `old` (the regrid's new cells); returns
// the count, writes at most cap boxes.
int hc_fresh(const int* boxes, int nb, const int* old, int no, int* out, int cap) {
  std::vector<mlswe::Box> B, O;
  for (int k = 0; k < nb; ++k) B.push_back(mlswe::Box{boxes[4 * k], boxes[4 * k + 1], boxes[4 * k + 2], boxes[4 * k + 3]});
  for (int k = 0; k < no; ++k) O.push_back(mlswe::Box{old[4 * k], old[4 * k + 1], old[4 * k + 2], old[4 * k + 3]});
  std::vector<mlswe::Box> f = mlswe::fresh_cells(B, O);
  for (int k = 0; k < (int)f.size() && k < cap; ++k) {
    out[4 * k] = f[k].i0; out[4 * k + 1] = f[k].j0; out[4 * k + 2] = f[k].i1; out[4 * k + 3] = f[k].j1;
  }
  return (int)f.size();
}

}
