// Host-side internals of the library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>
#include "../../include/mlswe.h"
#include "mlswe_device.cuh"

namespace mlswe {

struct Box {
  int i0, j0, i1, j1;  // half-open, level cell indices
  int w() const { return i1 - i0; }
  int h() const { return j1 - j0; }
};

// Work item of the level-transfer kernels: a box of cells of one level (the fine level
// for refinement, the coarse level for coarsening and reflux) and the two levels involved.
struct InterpItem {
  int desc_c, desc_f;
  int i0, j0, i1, j1;
};

struct Level {
  int NX = 0, NY = 0, P = 0;
  double dx = 0, dy = 0;
  double* q[2] = {nullptr, nullptr};
  double* qs = nullptr;
  double* B = nullptr;
  uint8_t* in_patch = nullptr;  // level >= 1
  uint8_t* covered = nullptr;   // cells covered by the next finer level (levels < max-1)
  double* fxc = nullptr;
  double* fyc = nullptr;
  double* fxf = nullptr;
  double* fyf = nullptr;
  std::vector<Box> patches;
};

struct Member {
  mlswe_domain dom;
  std::vector<Level> lev;
};

// Tile shape of one sweep direction: `len` cells along the sweep, `lines` lines per tile.
struct TileShape {
  int len = 61;
  int lines = 4;
};

// Kernel classes timed by the optional launch timer.
enum KernelClass { KC_SWEEP_X = 0, KC_SWEEP_Y, KC_GHOST, KC_INTERP, KC_AVERAGE, KC_FLAGS, KC_REFLUX, KC_OTHER, KC_COUNT };

struct LaunchTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Rec { int kc; int e0, e1; };
  std::vector<Rec> recs;
  size_t next = 0;
  double ms[KC_COUNT] = {0};
  long long launches[KC_COUNT] = {0};
};

struct Hier {
  mlswe_config cfg;
  DevParams dp;
  int n_members = 0;
  int L = 1;                  // number of levels
  std::vector<Member> mem;
  std::vector<int> parity;    // per level: which q buffer is current
  mlswe_allocator alloc{};
  bool own_alloc = true;
  cudaStream_t st = nullptr;
  std::string err;
  std::vector<void*> allocations;

  // Device tables.
  LevelDesc* d_desc = nullptr;        // [n_members * L]
  double* d_dt = nullptr;             // [n_members * L]
  unsigned long long* d_smax = nullptr;  // [n_members * L * 2]
  unsigned int* d_lost = nullptr;     // [1]
  std::vector<double> h_dt;           // host copy of dt per (member, level)
  // Sweep work lists per level and direction.
  struct WorkList {
    SweepItem* d_items = nullptr;
    int* d_count = nullptr;
    int capacity = 0;
    int count = 0;
    bool dirty = true;
  };
  std::vector<WorkList> wl;  // [L * 2]
  TileShape shape[2];
  int blocks_per_sm = 1;
  int num_sms = 0;
  double t = 0.0;
  long long coarse_steps = 0;
  LaunchTimer timer;
  long long kernel_launches = 0;   // every kernel this hierarchy launched
  void* scratch = nullptr;         // small per-call device scratch (gauges)
  size_t scratch_bytes = 0;
  void* stage = nullptr;           // staging of per-launch item tables (AMR kernels)
  size_t stage_bytes = 0;
  bool have_rates = false;         // wave-speed rates of the last coarse step are known
  std::vector<double> last_rates;  // [member * L + level]: max(sx/dx, sy/dy)
  std::vector<double> last_dt0;    // [member]: last level-0 step

  int desc_index(int member, int level) const { return member * L + level; }
};

// Optional per-kernel-class timing with CUDA events on the hierarchy's stream.
void timer_begin(Hier* H, int kc, int* token);
void timer_end(Hier* H, int token);

// Memory helpers (implemented in mlswe_host.cu).
void* dev_alloc(Hier* H, size_t bytes);
void dev_free(Hier* H, void* p);

// Kernel launchers.
size_t sweep_smem_bytes(int M);
cudaError_t launch_average(int nf, int r, const double* fine, int fP, size_t fplane, double* coarse, int cP,
                           size_t cplane, int ci0, int cj0, int ci1, int cj1, const uint8_t* mask, int maskNX,
                           cudaStream_t st);
cudaError_t launch_gauges(int M, const LevelDesc* descs, const int* parity_of_desc, const int* cells, int n,
                          double* out, cudaStream_t st);
cudaError_t launch_sweep(int dir, const DevParams& P, const LevelDesc* descs, const SweepItem* items,
                         const int* n_items_dev, int grid, int parity, unsigned long long* smax_bits,
                         unsigned int* lost_count, cudaStream_t st);

}  // namespace mlswe

struct mlswe_hier : public mlswe::Hier {};
