// Device wrapper around the sweep kernel's iterative reciprocal and reciprocal square root
// and its left share of a limited wave (compiled by the test for the GPU) so that they can
// be compared with the library functions, an exact reference and the textbook formula.
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
__global__ void share_kernel(const double* __restrict__ in, const int* __restrict__ flags, int n,
                             double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int* f = flags + 3 * i;
  out[i] = mlswe::left_share(f[0], f[1], f[2] != 0, in[4 * i], in[4 * i + 1], in[4 * i + 2], in[4 * i + 3]);
}
__global__ void solve_kernel(const double* __restrict__ in, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int N = 6;
  const double* c = in + (size_t)i * (N * N + 2 * N);
  double A1[N][N], A2[N][N], A3[N][N], b1[N], b2[N], bb[2][N], x1[N], x2[N], xx[2][N];
  for (int r = 0; r < N; ++r)
    for (int k = 0; k < N; ++k) A1[r][k] = A2[r][k] = A3[r][k] = c[r * N + k];
  for (int r = 0; r < N; ++r) {
    b1[r] = bb[0][r] = c[N * N + r];
    b2[r] = bb[1][r] = c[N * N + N + r];
  }
  mlswe::gauss_solve<N>(A1, b1, x1);
  mlswe::gauss_solve<N>(A2, b2, x2);
  mlswe::gauss_solve_multi<N, 2>(A3, bb, xx);
  double* o = out + (size_t)i * 4 * N;
  for (int r = 0; r < N; ++r) { o[r] = x1[r]; o[N + r] = x2[r]; o[2 * N + r] = xx[0][r]; o[3 * N + r] = xx[1][r]; }
}
}  // namespace

// Solves of n 6 x 6 systems (per system: A row-major, then two right-hand sides): for each,
// x of both right-hand sides by gauss_solve separately, then by gauss_solve_multi together.
extern "C" int mc_solve(const double* in_host, int n, double* out_host) {
  if (n <= 0) return 0;
  const size_t in_b = sizeof(double) * (size_t)n * 48, out_b = sizeof(double) * (size_t)n * 24;
  double *din = nullptr, *dout = nullptr;
  int rc = 0;
  if (cudaMalloc(&din, in_b) != cudaSuccess) return 1;
  if (cudaMalloc(&dout, out_b) != cudaSuccess) rc = 1;
  if (!rc && cudaMemcpy(din, in_host, in_b, cudaMemcpyHostToDevice) != cudaSuccess) rc = 1;
  if (!rc) {
    solve_kernel<<<(n + 127) / 128, 128>>>(din, n, dout);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = 1;
  }
  if (!rc && cudaMemcpy(out_host, dout, out_b, cudaMemcpyDeviceToHost) != cudaSuccess) rc = 1;
  cudaFree(din);
  cudaFree(dout);
  return rc;
}

// Left share of a wave (the sweep's left_share): in = (num, iden, s, nu) per case, flags =
// (limiter kind, sign class of s, active) per case.
extern "C" int mc_left_share(const double* in_host, const int* flags_host, int n, double* out_host) {
  if (n <= 0) return 0;
  double *din = nullptr, *dout = nullptr;
  int* dfl = nullptr;
  int rc = 0;
  if (cudaMalloc(&din, sizeof(double) * 4 * (size_t)n) != cudaSuccess) return 1;
  if (cudaMalloc(&dout, sizeof(double) * n) != cudaSuccess) rc = 1;
  if (!rc && cudaMalloc(&dfl, sizeof(int) * 3 * (size_t)n) != cudaSuccess) rc = 1;
  if (!rc && cudaMemcpy(din, in_host, sizeof(double) * 4 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess) rc = 1;
  if (!rc && cudaMemcpy(dfl, flags_host, sizeof(int) * 3 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess) rc = 1;
  if (!rc) {
    share_kernel<<<(n + 255) / 256, 256>>>(din, dfl, n, dout);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = 1;
  }
  if (!rc && cudaMemcpy(out_host, dout, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) rc = 1;
  cudaFree(din);
  cudaFree(dout);
  cudaFree(dfl);
  return rc;
}

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
