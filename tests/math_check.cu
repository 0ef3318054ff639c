// Device wrapper around the sweep kernel's iterative reciprocal and reciprocal square root
// (compiled by the test for the GPU) so that they can be compared with the library
// functions and with an exact reference.
#include <cuda_runtime.h>
#include "../paper_1803_01450_gb300/csrc/mlswe_device.cuh"

namespace {
__global__ void math_kernel(const double* __restrict__ x, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  out[0 * (size_t)n + i] = mlswe::rcp_fast(v);
  out[1 * (size_t)n + i] = __drcp_rn(v);
  out[2 * (size_t)n + i] = mlswe::rsqrt_fast(v);
  out[3 * (size_t)n + i] = rsqrt(v);
  out[4 * (size_t)n + i] = mlswe::sqrt_fast(v);
  out[5 * (size_t)n + i] = sqrt(v);
}
}  // namespace

extern "C" int mc_run(const double* x_host, int n, double* out_host) {
  if (n <= 0) return 0;
  double *dx = nullptr, *dout = nullptr;
  if (cudaMalloc(&dx, sizeof(double) * n) != cudaSuccess) return 1;
  if (cudaMalloc(&dout, sizeof(double) * 6 * (size_t)n) != cudaSuccess) { cudaFree(dx); return 1; }
  int rc = 0;
  if (cudaMemcpy(dx, x_host, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess) rc = 1;
  if (!rc) {
    math_kernel<<<(n + 255) / 256, 256>>>(dx, n, dout);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = 1;
  }
  if (!rc && cudaMemcpy(out_host, dout, sizeof(double) * 6 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess) rc = 1;
  cudaFree(dx);
  cudaFree(dout);
  return rc;
}
