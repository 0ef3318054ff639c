// One split step of a single walled grid that allocates no memory.
//
// Who needs it: callers that cannot call cudaMalloc or any allocating routine
// while they step the model -- for example a host application that runs the
// solver inside a callback of another framework that owns the device memory
// pool, or a code path that runs under a strict "no allocation after start-up"
// rule (real-time or embedded use, memory-capped services). Such callers own
// their input and output buffers already; what they cannot provide is the
// solver's own working memory. This entry point keeps that working memory (the
// state after the x sweep, the tile list, the level descriptor, the time step
// and the wave-speed slots) in one file-scope device array instead.
//
// The array lives in every GPU that loads the library, for the life of the
// process. All calls share it, so calls that overlap on the GPU (on different
// streams, or from different host threads) race on it and must be serialised
// by the caller. It keeps the last call's contents; the parts that must start
// at zero (the wave-speed slots) are cleared by every call.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>
#include "mlswe_internal.h"

namespace mlswe {

// Largest grid the scratch array holds: the state after the x sweep of M * nx * ny <=
// 2 * 512 * 512 layer cells (12.6 MB: 512 x 512 cells for one or two layers, fewer cells for
// three or four) and up to 65536 tiles per sweep.
constexpr long long kNoAllocMaxLayerCells = 2LL * 512LL * 512LL;
constexpr int kNoAllocMaxItems = 65536;
constexpr size_t kNoAllocQsBytes = (size_t)3 * kNoAllocMaxLayerCells * sizeof(double);
constexpr size_t kNoAllocItemBytes = (size_t)kNoAllocMaxItems * sizeof(SweepItem);
constexpr size_t kNoAllocHeadBytes = 1024;  // descriptor, item counts, dt, wave-speed slots
constexpr size_t kNoAllocBytes = kNoAllocHeadBytes + 2 * kNoAllocItemBytes + kNoAllocQsBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array on each device, looked up once per device with
// that device current (the symbol's host-side name is not a device address).
static std::mutex g_noalloc_mutex;
static std::vector<unsigned char*> g_noalloc_ptr;

static cudaError_t noalloc_scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if ((int)g_noalloc_ptr.size() <= dev) g_noalloc_ptr.resize(dev + 1, nullptr);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = (unsigned char*)p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// Tiles of one sweep over the whole grid (the same tiles the hierarchy uses by default:
// 125 cells x 2 lines in both directions).
static void noalloc_items(int nx, int ny, int dir, std::vector<SweepItem>& out) {
  out.clear();
  const int len = 125, lines = 2;
  if (dir == 0) {
    for (int j = 0; j < ny; j += lines)
      for (int i = 0; i < nx; i += len)
        out.push_back(SweepItem{0, i, j, std::min(len, nx - i), std::min(lines, ny - j), 1});
  } else {
    for (int i = 0; i < nx; i += lines)
      for (int j = 0; j < ny; j += len)
        out.push_back(SweepItem{0, i, j, std::min(len, ny - j), std::min(lines, nx - i), 1});
  }
}

// True when p is memory a kernel can dereference (device or managed). Querying the
// pointer allocates nothing.
static bool noalloc_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error of an unregistered host pointer
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Byte ranges [a, a + na) and [b, b + nb) share at least one byte.
static bool noalloc_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

}  // namespace mlswe

using namespace mlswe;

extern "C" mlswe_status mlswe_step_fixed_noalloc(const mlswe_config* cfg, int nx, int ny, double dx, double dy,
                                                 double dt, const double* q_in, const double* B, double* q_out,
                                                 void* cuda_stream, double* cfl_out) {
  if (!cfg || !q_in || !B || !q_out || cfg->unsplit != 0) return MLSWE_EINVAL;
  if (cfg->M < 1 || cfg->M > 4 || cfg->order < 1 || cfg->order > 2 || cfg->limiter < 0 || cfg->limiter > 2 ||
      cfg->eigen < 0 || cfg->eigen > 1 || !(cfg->g > 0.0) || !(cfg->dry_tol >= 0.0))
    return MLSWE_EINVAL;
  if (cfg->M >= 2 && !(cfg->rho[0] > 0.0)) return MLSWE_EINVAL;
  for (int m = 0; m + 1 < cfg->M; ++m)  // densities increase downwards (stable stratification)
    if (!(cfg->rho[m] < cfg->rho[m + 1])) return MLSWE_EINVAL;
  if (nx < 4 || ny < 4 || !(dx > 0.0) || !(dy > 0.0) || !(dt >= 0.0)) return MLSWE_EINVAL;
  if ((long long)cfg->M * nx * ny > kNoAllocMaxLayerCells) return MLSWE_EINVAL;  // larger than the scratch array
  // The buffers: device memory the kernels can read and write, and an output that shares
  // no byte with either input (the sweeps read q_in and B while they write q_out).
  const size_t state_bytes = (size_t)3 * cfg->M * nx * ny * sizeof(double);
  const size_t bath_bytes = (size_t)nx * ny * sizeof(double);
  if (!noalloc_device_ptr(q_in) || !noalloc_device_ptr(B) || !noalloc_device_ptr(q_out)) return MLSWE_EINVAL;
  if (noalloc_overlap(q_in, state_bytes, q_out, state_bytes) || noalloc_overlap(B, bath_bytes, q_out, state_bytes))
    return MLSWE_EINVAL;
  std::vector<SweepItem> items[2];
  for (int dir = 0; dir < 2; ++dir) {
    noalloc_items(nx, ny, dir, items[dir]);
    if ((int)items[dir].size() > kNoAllocMaxItems) return MLSWE_EINVAL;
  }
  unsigned char* base = nullptr;
  if (noalloc_scratch_address(&base) != cudaSuccess) return MLSWE_ECUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // Layout of the scratch array: [descriptor | counts | dt | speed slots] [x tiles] [y tiles] [Q*].
  LevelDesc* d_desc = (LevelDesc*)base;
  int* d_count = (int*)(base + 512);
  double* d_dt = (double*)(base + 528);
  unsigned long long* d_smax = (unsigned long long*)(base + 544);
  SweepItem* d_items[2] = {(SweepItem*)(base + kNoAllocHeadBytes),
                           (SweepItem*)(base + kNoAllocHeadBytes + kNoAllocItemBytes)};
  double* d_qs = (double*)(base + kNoAllocHeadBytes + 2 * kNoAllocItemBytes);

  LevelDesc D{};
  D.q[0] = const_cast<double*>(q_in);  // parity 0: read q[0], write q[1]
  D.q[1] = q_out;
  D.qs = d_qs;
  D.B = const_cast<double*>(B);
  D.dt = d_dt;
  D.NX = nx; D.NY = ny; D.P = nx;
  D.inv_dx = 1.0 / dx; D.inv_dy = 1.0 / dy;
  D.ue = nullptr; D.uxp = 0; D.uyp = 0;
  const int counts[2] = {(int)items[0].size(), (int)items[1].size()};
  DevParams P;
  fill_dev_params(cfg, &P);  // unsplit is 0 (checked above)

  if (cudaMemcpyAsync(d_desc, &D, sizeof(D), cudaMemcpyHostToDevice, st) != cudaSuccess) return MLSWE_ECUDA;
  if (cudaMemcpyAsync(d_count, counts, sizeof(counts), cudaMemcpyHostToDevice, st) != cudaSuccess) return MLSWE_ECUDA;
  if (cudaMemcpyAsync(d_dt, &dt, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) return MLSWE_ECUDA;
  if (cudaMemsetAsync(d_smax, 0, 2 * sizeof(unsigned long long), st) != cudaSuccess) return MLSWE_ECUDA;
  for (int dir = 0; dir < 2; ++dir)
    if (cudaMemcpyAsync(d_items[dir], items[dir].data(), items[dir].size() * sizeof(SweepItem),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
      return MLSWE_ECUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MLSWE_ECUDA;
  for (int dir = 0; dir < 2; ++dir)
    if (launch_sweep(dir, P, d_desc, d_items[dir], d_count + dir, nullptr, sms, 0, 1, d_smax, nullptr, st) !=
        cudaSuccess)
      return MLSWE_ECUDA;
  if (cfl_out) {
    unsigned long long bits[2];
    if (cudaMemcpyAsync(bits, d_smax, sizeof(bits), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MLSWE_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MLSWE_ECUDA;
    double sx, sy;
    memcpy(&sx, &bits[0], 8);
    memcpy(&sy, &bits[1], 8);
    if (!(sx >= 0.0) || !(sy >= 0.0)) return MLSWE_ENEGDEPTH;
    *cfl_out = dt * std::max(sx / dx, sy / dy);
  }
  return MLSWE_OK;
}
