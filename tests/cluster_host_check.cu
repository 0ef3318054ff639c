// Host-side wrapper around the library's flag dilation and clustering (compiled as host
// code by the test, no GPU needed) so that they can be compared with the oracle's.
#include <cstdint>
#include <vector>
#include "../paper_1803_01450_gb300/csrc/mlswe_internal.h"

namespace mlswe {
void dilate_flags(const uint8_t* in, int nx, int ny, int n, std::vector<uint8_t>& out);
std::vector<Box> cluster_flags(const uint8_t* flags, int nx, int ny, int level, const std::vector<Box>& patches,
                               int r, int n_buf, double eff, int min_side, int max_side, int n_nest);
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

}
