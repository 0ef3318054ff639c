// Level-transfer kernels: bathymetry per level, refinement (Sec. 2.1),
// coarsening (Sec. 2.2), refinement flags, flag dilation, ghost fill,
// mass reflux and gauges. All of them are memory-bound, one thread per
// output cell, coalesced along x.
#include <cuda_runtime.h>
#include "mlswe_internal.h"

namespace mlswe {

// r x r mean of fine cells into coarse cells: row-major sum, then times 1/(r r)
// (the operator of Eq. (11), used for bathymetry of coarser levels and for the
// conserved fields of covered coarse cells). nf planes of [ny][pitch].
__global__ void average_kernel(int nf, int r, const double* __restrict__ fine, int fP, size_t fplane,
                               double* __restrict__ coarse, int cP, size_t cplane, int ci0, int cj0, int ci1,
                               int cj1, const uint8_t* __restrict__ mask, int maskNX) {
  const int nxb = ci1 - ci0, nyb = cj1 - cj0;
  const long long total = (long long)nxb * nyb;
  const double inv = 1.0 / (double)(r * r);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int j = cj0 + (int)(t / nxb), i = ci0 + (int)(t % nxb);
    if (mask && !mask[(size_t)j * maskNX + i]) continue;
    for (int f = 0; f < nf; ++f) {
      double s = 0.0;
      for (int b = 0; b < r; ++b)
        for (int a = 0; a < r; ++a) s += fine[f * fplane + (size_t)(j * r + b) * fP + (i * r + a)];
      coarse[f * cplane + (size_t)j * cP + i] = s * inv;
    }
  }
}

cudaError_t launch_average(int nf, int r, const double* fine, int fP, size_t fplane, double* coarse, int cP,
                           size_t cplane, int ci0, int cj0, int ci1, int cj1, const uint8_t* mask, int maskNX,
                           cudaStream_t st) {
  const long long total = (long long)(ci1 - ci0) * (cj1 - cj0);
  if (total <= 0) return cudaSuccess;
  const int grid = (int)std::min<long long>((total + 255) / 256, 65536);
  average_kernel<<<grid, 256, 0, st>>>(nf, r, fine, fP, fplane, coarse, cP, cplane, ci0, cj0, ci1, cj1, mask, maskNX);
  return cudaGetLastError();
}

}  // namespace mlswe

namespace mlswe {

// Gauges: surface elevations eta_m = B + h_M + ... + h_m (Eq. (4)) of given cells.
// cell[k] = (desc, i, j); out[k * M + m].
__global__ void gauge_kernel(int M, const LevelDesc* __restrict__ descs, const int* __restrict__ parity_of_desc,
                             const int* __restrict__ cells, int n, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const LevelDesc& D = descs[cells[3 * k]];
  const int i = cells[3 * k + 1], j = cells[3 * k + 2];
  const size_t o = (size_t)j * D.P + i, plane = (size_t)D.NY * D.P;
  const double* q = D.q[parity_of_desc[cells[3 * k]]];
  double acc = D.B[o];
  for (int m = M - 1; m >= 0; --m) {
    acc = acc + q[(3 * m) * plane + o];
    out[k * M + m] = acc;
  }
}

cudaError_t launch_gauges(int M, const LevelDesc* descs, const int* parity_of_desc, const int* cells, int n,
                          double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  gauge_kernel<<<(n + 127) / 128, 128, 0, st>>>(M, descs, parity_of_desc, cells, n, out);
  return cudaGetLastError();
}

}  // namespace mlswe
