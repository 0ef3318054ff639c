// Host-side internals of the library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
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

// Work entry of the ghost fill: one coarse cell (ic, jc) of level l-1 under a ghost strip
// (fine cells [i0, i1) x [j0, j1) of level l, in the domain) of a level-l patch.
struct GhostCell {
  int desc_c, desc_f;
  int ic, jc;
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
  double* ue = nullptr;         // unsplit step: per-edge arrays (see LevelDesc::ue)
  long long uxp = 0, uyp = 0;
  double* snap = nullptr;       // level >= 1: patch cells before a coarse-step attempt
  std::vector<Box> patches;
};

struct Member {
  mlswe_domain dom;
  std::vector<Level> lev;
};

// Work entry of the partition exchange: one patch (box of level cells of desc) and where its
// values start in its owner's packed buffer (see mlswe_partition.cu for the layout).
struct PackItem {
  int desc;
  int i0, j0, i1, j1;
  int parts;  // bit 0: state fields, 1: boundary mass-flux accumulators, 2: interface fluxes
  long long off;
};
constexpr int kPackState = 1, kPackAccum = 2, kPackIface = 4;

// Tile shape of one sweep direction: `len` cells along the sweep, `lines` lines per tile.
struct TileShape {
  int len = 61;
  int lines = 4;
  int ctas = 1;  // resident CTAs per SM of the persistent grid (kernel variant)
};

// Kernel classes timed by the optional launch timer.
enum KernelClass {
  KC_SWEEP_X = 0, KC_SWEEP_Y, KC_GHOST, KC_INTERP, KC_AVERAGE, KC_FLAGS, KC_REFLUX, KC_OTHER, KC_ADJOINT, KC_UPDATE,
  KC_COUNT
};

struct LaunchTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Rec { int kc; int e0, e1; };
  std::vector<Rec> recs;
  size_t next = 0;
  double ms[KC_COUNT] = {0};
  long long launches[KC_COUNT] = {0};
};

// Device-resident table of work items with a device-resident count (a captured graph
// reads both at replay time, so tables can be rewritten without recapture).
template <class T>
struct DevTable {
  T* d = nullptr;
  int* d_count = nullptr;
  int cap = 0;
  int count = 0;
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
  bool own_stream = false;
  std::string err;
  std::vector<void*> allocations;

  // Device tables.
  LevelDesc* d_desc = nullptr;        // [n_members * L]
  double* d_dt = nullptr;             // [n_members * L]
  unsigned long long* d_smax = nullptr;  // [n_members * L * 2]
  unsigned long long* d_init = nullptr;  // [n_members * L] initial wave speeds
  unsigned int* d_lost = nullptr;     // [1]
  unsigned int* d_status = nullptr;   // [1] bit 0: Courant above cfl_max, bit 1: non-finite speed
  double* d_t = nullptr;              // [n_members] simulated time
  double* d_cfl = nullptr;            // [n_members] Courant number of the last coarse step
  int* d_has = nullptr;               // [n_members * L] level has patches
  double* d_invdx = nullptr;          // [n_members * L]
  double* d_invdy = nullptr;
  int* d_par = nullptr;               // [n_members * L] parity of the desc's level (speed kernel)
  int* d_init_flag = nullptr;         // [1] 1: the next step's dt comes from d_init
  std::vector<double> h_dt;           // host copy of dt per (member, level)
  // Sweep work lists per level and direction, with per-patch ranges for the
  // one-launch-per-patch form.
  struct WorkList {
    SweepItem* d_items = nullptr;
    int* d_count = nullptr;
    int capacity = 0;
    int count = 0;
    bool dirty = true;
    std::vector<int> patch_off;     // item offset of every (member, patch)
    int* d_patch_count = nullptr;   // item count of every (member, patch)
    int patch_cap = 0;
    // Batched form (not per-patch launches): the items are groups of lines packed into tiles
    // of at most kMaxEdges edges, tile t = items [tile_off[t], tile_off[t + 1]).
    bool packed = false;
    int* d_tile_off = nullptr;
    int tile_cap = 0;
    int ntiles = 0;
  };
  std::vector<WorkList> wl;  // [L * 2]
  std::vector<WorkList> wu;  // [L] cell tiles of the unsplit step's update
  std::vector<TileShape> shape;  // [L * 2]
  int blocks_per_sm = 1;
  int num_sms = 0;
  bool per_patch_launch = false;
  bool use_graphs = true;
  // Level-transfer tables per level (ghost strips of level l, coarsening of l onto l-1,
  // reflux scan of l, wave-speed boxes of all levels).
  std::vector<DevTable<InterpItem>> t_avg, t_reflux;  // reflux: single interface cells
  std::vector<DevTable<GhostCell>> t_gcell;                     // ghost fill: coarse cells of the rings
  DevTable<InterpItem> t_speed;
  bool tables_dirty = true;
  bool dt_ready = false;           // device dt holds the next coarse step
  // Graphs of one coarse step, per level-0 parity.
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graph_valid[2] = {false, false};
  long long graph_launches[2] = {0, 0};  // kernels inside each graph
  long long coarse_steps = 0;
  long long regrids = 0;                 // regrids run (automatic and mlswe_regrid)
  std::vector<long long> level_steps;    // [L] steps taken per level
  std::vector<long long> cell_updates;   // [L] patch cells x steps per level, all members
  unsigned long long* d_cfl_count = nullptr;  // [1] member coarse steps above cfl_max
  int* d_rt = nullptr;                 // [n_members * L] time ratio of each level (this step)
  int* d_active = nullptr;             // [n_members * L] the level's current substep is taken
  int* d_fresh = nullptr;              // [1] the next coarse step follows a regrid
  int* d_redo = nullptr;               // [n_members] the last attempt was rejected (Courant > cfl_max)
  long long* d_done = nullptr;         // [n_members] coarse steps kept by mlswe_advance
  bool snaps_ready = false;            // every level >= 1 has its snapshot buffer
  long long* d_cells = nullptr;        // [n_members * L] cells inside the patches
  long long* d_steps_acc = nullptr;    // [n_members * L] level steps of mlswe_advance
  long long* d_cells_acc = nullptr;    // [n_members * L] cell updates of mlswe_advance
  LaunchTimer timer;
  long long kernel_launches = 0;   // every kernel this hierarchy launched
  void* scratch = nullptr;         // small per-call device scratch (gauges, flags)
  // mlswe_set_state_async: copy stream, two staging buffers, events of their copies and of
  // the state copies that read them
  cudaStream_t copy_st = nullptr;
  double* stage[2] = {nullptr, nullptr};
  size_t stage_bytes = 0;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
  int stage_next = 0;
  size_t scratch_bytes = 0;
  void* adj = nullptr;             // buffers of the fixed-grid adjoint (mlswe_adjoint.cu)
  // Patch partition across ranks (mlswe_partition.cu): this rank sweeps only the patches of
  // levels >= 1 it owns; everything else runs on every rank.
  int part_rank = 0, part_size = 1;
  mlswe_exchange_hook part_hook = nullptr;
  void* part_ctx = nullptr;
  bool part_dirty = true;
  std::vector<std::vector<std::vector<int>>> owner;  // [member][level][patch] rank
  struct PartTable {
    DevTable<PackItem> items;      // grouped by owner
    std::vector<int> first;        // [part_size + 1] item range of each owner
    std::vector<long long> size;   // [part_size] doubles in each owner's packed buffer
  };
  struct PartLevel {
    PartTable kind[4];             // exchange tables by MLSWE_XCHG_ kind (full, halo, last,
                                   // averaged: parent cells under the finest level's patches)
  };
  std::vector<PartLevel> part;     // [L]

  int desc_index(int member, int level) const { return member * L + level; }
};

// Arguments of the device-side time-step kernels.
struct DtArgs {
  int L;
  int n_members;
  int ratio[4];
  int dynamic_rt;           // 1: time ratio per level and step from the wave speeds
  double cfl, cfl_max;
  const int* has_patches;   // [member * L + l]
  const double* inv_dx;     // [member * L + l]
  const double* inv_dy;
  int* rt;                  // [member * L + l] time steps of level l per parent step (written)
  int* active;              // [member * L + l] substep activity, reset to 1 at the step end
  int* fresh;               // [1] 1 on the first coarse step after a regrid: fixed ratios (the
                            // last speeds were measured on the old patches); cleared at the end
  const long long* cells;   // [member * L + l] cells inside the level's patches
  long long* steps_acc;     // [member * L + l] level steps taken (accumulated)
  long long* cells_acc;     // [member * L + l] cell updates taken (accumulated)
  int* redo;                // [member] 1: the attempt just taken was rejected
  long long* done;          // [member] coarse steps kept
};
cudaError_t launch_dt_begin(const DtArgs& A, unsigned long long* smax_bits, const unsigned long long* init_bits,
                            int* init_flag, double* dt, cudaStream_t st);
cudaError_t launch_set_active(int L, int n_members, int level, int k, const int* rt, int* active,
                              cudaStream_t st);
cudaError_t launch_step_end(const DtArgs& A, const unsigned long long* smax_bits, const double* dt, double* t_member,
                            double* cfl_reached, unsigned int* status, unsigned long long* cfl_count,
                            cudaStream_t st);

// Parities of every level at the start of a coarse step and after it.
struct ParSet {
  int start[4];
  int next[4];
};
// Courant control of mlswe_advance over the patch boxes of every level (the wave-speed work
// list): mode 0 copies the patch cells of levels >= 1 into their snapshots; mode 1, for the
// members whose attempt was rejected, copies level 0's state before the step into its new
// buffer and the snapshots into the new buffers of levels >= 1.
cudaError_t launch_snapshot(int F, int L, const LevelDesc* descs, const InterpItem* items, const int* n_items_dev,
                            int grid, int mode, const ParSet& par, const int* redo, cudaStream_t st);

// Cells inside the patches of `level`, summed over the members.
long long patch_cells(const Hier* H, int level);

// NVTX range for the duration of a scope (shows host phases in a timeline profiler; costs
// nothing measurable when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Optional per-kernel-class timing with CUDA events on the hierarchy's stream.
void timer_begin(Hier* H, int kc, int* token);
void timer_end(Hier* H, int token);

// Memory helpers (implemented in mlswe_host.cu).
void* dev_alloc(Hier* H, size_t bytes);
void dev_free(Hier* H, void* p);
void* scratch_buffer(Hier* H, size_t bytes);
void invalidate_graphs(Hier* H);
// Solver constants of a configuration, the host-side ones (density ratios, reciprocals,
// reduced gravities) computed here once for every path that launches the sweeps.
void fill_dev_params(const mlswe_config* cfg, DevParams* P);
mlswe_status ensure_snapshots(Hier* H);

// Kernel launchers.
cudaError_t launch_unsplit_update(const DevParams& P, const LevelDesc* descs, const SweepItem* items,
                                  const int* n_items_dev, int grid, int parity, int record, cudaStream_t st);
size_t sweep_smem_bytes(int M);
cudaError_t launch_average(int nf, int r, const double* fine, int fP, size_t fplane, double* coarse, int cP,
                           size_t cplane, int ci0, int cj0, int ci1, int cj1, const uint8_t* mask, int maskNX,
                           cudaStream_t st);
cudaError_t launch_gauges(int M, const LevelDesc* descs, const int* parity_of_desc, const int* cells, int n,
                          double* out, cudaStream_t st);
cudaError_t launch_sweep(int dir, const DevParams& P, const LevelDesc* descs, const SweepItem* items,
                         const int* n_items_dev, const int* tile_off, int grid, int parity, int record,
                         unsigned long long* smax_bits, unsigned int* lost_count, cudaStream_t st, int ctas_per_sm = 1,
                         double* est = nullptr, long long eplane = 0);

mlswe_status enqueue_level_step(Hier* H, int level, int record);

// Patch partition (mlswe_partition.cu): owners and exchange tables rebuilt after a layout
// change; whether this rank sweeps patch p of (member, level) (always on level 0 and when the
// hierarchy is not partitioned); the exchange hook after a level step.
mlswe_status ensure_partition(Hier* H);
// For every patch, the other patches whose box grown by g cells meets it (ascending).
std::vector<std::vector<int>> patches_near(const std::vector<Box>& P, int g);
bool patch_owned(const Hier* H, int member, int level, int p);
mlswe_status run_exchange_hook(Hier* H, int level, int kind);
// This rank coarsens finest-level patch p of member m (the others are coarsened by their
// owners): always when the hierarchy is not partitioned.
bool coarsens_patch(const Hier* H, int member, int level, int p);

// Packed sweep tiles (mlswe_pack.cu). patch_segments appends the runs of lines of patch b
// for a sweep along dir (0: x, lines are rows; 1: y, lines are columns): lines [g0, g1)
// across (the patch's own lines [lo, hi) flagged interior, the others ghost lines), parts of
// at most tile_len cells along. pack_tiles packs runs in order into tiles of at most
// kMaxEdges edges, kMaxCells cells and kMaxGroups groups (runs or their pieces) of one
// desc, cutting a run where it does not fit: tile t is items [toff[t], toff[t + 1]); false
// (nothing usable) when a run's line is longer than a tile holds.
void patch_segments(const Box& b, int dir, int tile_len, int g0, int g1, int desc, std::vector<SweepItem>& out);
bool pack_tiles(const std::vector<SweepItem>& segs, int dir, std::vector<SweepItem>& items, std::vector<int>& toff);
void adjoint_release(Hier* H);
mlswe_status ensure_worklist(Hier* H, int level, int dir);

}  // namespace mlswe

struct mlswe_hier : public mlswe::Hier {};
