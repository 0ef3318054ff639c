// Host side of the AMR: patch layouts and masks, work-item tables of the level
// transfer kernels, the subcycled Berger-Oliger coarse step (captured once per
// level-0 parity as a CUDA graph and replayed), regridding and the tile autotuner.
#include <algorithm>
#include <cmath>
#include <cstring>
#include "mlswe_internal.h"

namespace mlswe {

cudaError_t launch_interp(int M, const DevParams& P, const LevelDesc* descs, const InterpItem* items,
                          const int* n_items_dev, int grid, int r, int par_c, int par_f, double alpha,
                          cudaStream_t st);
cudaError_t launch_average_items(int F, const LevelDesc* descs, const InterpItem* items, const int* n_items_dev,
                                 int grid, int r, int par_c, int par_f, cudaStream_t st);
cudaError_t launch_flags(int M, const LevelDesc* descs, int desc, int par, long long cells, double dry_tol,
                         double inv_dx, double inv_dy, double tol2, uint8_t* flags, cudaStream_t st);
cudaError_t launch_mask_boxes(uint8_t* mask, int NX, const int* boxes, int n, int div, long long max_cells,
                              cudaStream_t st);
cudaError_t launch_reflux(int M, const LevelDesc* descs, const InterpItem* cells, const int* n_dev, int grid,
                          int r, int par_c, cudaStream_t st);
cudaError_t launch_ghost_cells(int M, const DevParams& P, const LevelDesc* descs, const GhostCell* cells,
                               const int* n_dev, int grid, int r, int par_c, int par_f, double alpha, int substep,
                               cudaStream_t st);
cudaError_t launch_speed(int M, const DevParams& P, const LevelDesc* descs, const InterpItem* items,
                         const int* n_items_dev, int grid, const int* par_of_desc, unsigned long long* out,
                         cudaStream_t st);
std::vector<Box> cluster_flags(const uint8_t* flags, int nx, int ny, int level, const std::vector<Box>& patches,
                               int r, int n_buf, double eff, int min_side, int max_side, int n_nest);
std::vector<Box> fresh_cells(const std::vector<Box>& boxes, const std::vector<Box>& old);
void set_level_shape(Hier* H, int level, int dir, int len, int lines, int ctas);

constexpr int kNest = 2;    // nesting margin in coarse cells
constexpr int kChunk = 64;  // largest side of a level-transfer work item

static mlswe_status fail(Hier* H, mlswe_status s, const std::string& msg) {
  if (H) H->err = msg;
  return s;
}

#define CUDA_TRY(H, call)                                                               \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail((H), MLSWE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

static int grid_full(Hier* H) { return 2 * H->num_sms; }
// Flat transfer lists (one thread per entry): enough CTAs to keep the loads of several
// entries in flight per SM.
static int grid_flat(Hier* H) { return 8 * H->num_sms; }

// Appends the chunks (sides <= kChunk) of box b as items.
static void push_chunks(std::vector<InterpItem>& v, int dc, int df, Box b) {
  for (int j = b.j0; j < b.j1; j += kChunk)
    for (int i = b.i0; i < b.i1; i += kChunk)
      v.push_back(InterpItem{dc, df, i, j, std::min(i + kChunk, b.i1), std::min(j + kChunk, b.j1)});
}

template <class T_>
static mlswe_status upload_table(Hier* H, DevTable<T_>& T, const std::vector<T_>& v) {
  if ((int)v.size() > T.cap || !T.d) {
    if (T.d) dev_free(H, T.d);
    T.cap = std::max<int>(256, (int)v.size() * 3 / 2);
    T.d = (T_*)dev_alloc(H, T.cap * sizeof(T_));
    if (!T.d) return fail(H, MLSWE_ENOMEM, "item table allocation failed");
    invalidate_graphs(H);
  }
  if (!T.d_count) {
    T.d_count = (int*)dev_alloc(H, sizeof(int));
    if (!T.d_count) return fail(H, MLSWE_ENOMEM, "item table allocation failed");
  }
  T.count = (int)v.size();
  if (!v.empty())
    CUDA_TRY(H, cudaMemcpyAsync(T.d, v.data(), v.size() * sizeof(T_), cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaMemcpyAsync(T.d_count, &T.count, sizeof(int), cudaMemcpyHostToDevice, H->st));
  return MLSWE_OK;
}

// Rebuilds every level-transfer table from the current patch layouts (host -> device,
// synchronous). Graphs stay valid unless a table had to grow.
static mlswe_status build_tables(Hier* H) {
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  if (H->part_size > 1) {  // the finest level's coarsening takes this rank's patches only
    mlswe_status s = ensure_partition(H);
    if (s != MLSWE_OK) return s;
  }
  std::vector<int> has(H->n_members * H->L, 0);
  std::vector<long long> cells(H->n_members * H->L, 0);
  std::vector<InterpItem> speed;
  for (int l = 0; l < H->L; ++l) {
    std::vector<InterpItem> avg, refl;
    std::vector<GhostCell> gcell;
    for (int m = 0; m < H->n_members; ++m) {
      const Level& V = H->mem[m].lev[l];
      const int d = H->desc_index(m, l);
      has[d] = V.patches.empty() ? 0 : 1;
      for (const Box& b : V.patches) cells[d] += (long long)(b.i1 - b.i0) * (b.j1 - b.j0);
      for (const Box& b : V.patches) push_chunks(speed, d, d, b);
      if (l > 0) {
        const int dc = H->desc_index(m, l - 1);
        const int r = H->cfg.ratio[l - 1];
        for (int p = 0; p < (int)V.patches.size(); ++p) {
          const Box& b = V.patches[p];
          // ghost ring as four strips, clipped to the domain
          const int gi0 = std::max(0, b.i0 - kNG), gi1 = std::min(V.NX, b.i1 + kNG);
          const Box strips[4] = {Box{gi0, std::max(0, b.j0 - kNG), gi1, b.j0},
                                 Box{gi0, b.j1, gi1, std::min(V.NY, b.j1 + kNG)},
                                 Box{gi0, b.j0, b.i0, b.j1},
                                 Box{b.i1, b.j0, gi1, b.j1}};
          // partitioned: only the owner's sweeps read a patch's ring, so the owner fills it
          const bool own = patch_owned(H, m, l, p);
          for (const Box& s : strips)
            if (own && s.i1 > s.i0 && s.j1 > s.j0) {
              for (int jc = s.j0 / r; jc <= (s.j1 - 1) / r; ++jc)
                for (int ic = s.i0 / r; ic <= (s.i1 - 1) / r; ++ic)
                  gcell.push_back(GhostCell{dc, d, ic, jc, s.i0, s.j0, s.i1, s.j1});
            }
          if (coarsens_patch(H, m, l, p)) push_chunks(avg, dc, d, Box{b.i0 / r, b.j0 / r, b.i1 / r, b.j1 / r});
        }
      }
      if (l + 1 < H->L && !H->mem[m].lev[l + 1].patches.empty()) {
        // reflux cells: cells of a patch of this level, not covered by the next level, with a
        // covered face neighbour (found around the coarsened boxes of the finer patches)
        const int r = H->cfg.ratio[l], df = H->desc_index(m, l + 1);
        std::vector<uint8_t> cov((size_t)V.NX * V.NY, 0), inp, seen((size_t)V.NX * V.NY, 0);
        for (const Box& b : H->mem[m].lev[l + 1].patches)
          for (int j = b.j0 / r; j < b.j1 / r; ++j)
            std::memset(&cov[(size_t)j * V.NX + b.i0 / r], 1, b.i1 / r - b.i0 / r);
        if (l > 0) {
          inp.assign((size_t)V.NX * V.NY, 0);
          for (const Box& b : V.patches)
            for (int j = b.j0; j < b.j1; ++j) std::memset(&inp[(size_t)j * V.NX + b.i0], 1, b.i1 - b.i0);
        }
        auto visit = [&](int i, int j) {
          if (i < 0 || j < 0 || i >= V.NX || j >= V.NY) return;
          const size_t c = (size_t)j * V.NX + i;
          if (seen[c] || cov[c] || (l > 0 && !inp[c])) return;
          seen[c] = 1;
          refl.push_back(InterpItem{d, df, i, j, i + 1, j + 1});
        };
        for (const Box& b : H->mem[m].lev[l + 1].patches) {
          const int ci0 = b.i0 / r, cj0 = b.j0 / r, ci1 = b.i1 / r, cj1 = b.j1 / r;
          for (int j = cj0; j < cj1; ++j) { visit(ci0 - 1, j); visit(ci1, j); }
          for (int i = ci0; i < ci1; ++i) { visit(i, cj0 - 1); visit(i, cj1); }
        }
      }
    }
    mlswe_status s = upload_table(H, H->t_gcell[l], gcell);
    if (s == MLSWE_OK) s = upload_table(H, H->t_avg[l], avg);
    if (s == MLSWE_OK) s = upload_table(H, H->t_reflux[l], refl);
    if (s != MLSWE_OK) return s;
  }
  mlswe_status s = upload_table(H, H->t_speed, speed);
  if (s != MLSWE_OK) return s;
  CUDA_TRY(H, cudaMemcpyAsync(H->d_has, has.data(), has.size() * 4, cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaMemcpyAsync(H->d_cells, cells.data(), cells.size() * 8, cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  H->tables_dirty = false;
  return MLSWE_OK;
}

// Rebuilds in_patch of (member, level) and covered of (member, level - 1).
static mlswe_status rebuild_masks(Hier* H, int member, int level) {
  Level& V = H->mem[member].lev[level];
  Level& C = H->mem[member].lev[level - 1];
  std::vector<int> b;
  for (const Box& x : V.patches) { b.push_back(x.i0); b.push_back(x.j0); b.push_back(x.i1); b.push_back(x.j1); }
  CUDA_TRY(H, cudaMemsetAsync(V.in_patch, 0, (size_t)V.NX * V.NY, H->st));
  CUDA_TRY(H, cudaMemsetAsync(C.covered, 0, (size_t)C.NX * C.NY, H->st));
  if (!b.empty()) {
    int* d = (int*)scratch_buffer(H, b.size() * 4);
    if (!d) return fail(H, MLSWE_ENOMEM, "scratch allocation failed");
    CUDA_TRY(H, cudaStreamSynchronize(H->st));
    CUDA_TRY(H, cudaMemcpyAsync(d, b.data(), b.size() * 4, cudaMemcpyHostToDevice, H->st));
    long long mc = 0;
    for (const Box& x : V.patches) mc = std::max<long long>(mc, (long long)x.w() * x.h());
    int tok;
    timer_begin(H, KC_OTHER, &tok);
    CUDA_TRY(H, launch_mask_boxes(V.in_patch, V.NX, d, (int)V.patches.size(), 1, mc, H->st));
    timer_end(H, tok);
    timer_begin(H, KC_OTHER, &tok);
    CUDA_TRY(H, launch_mask_boxes(C.covered, C.NX, d, (int)V.patches.size(), H->cfg.ratio[level - 1], mc, H->st));
    timer_end(H, tok);
  }
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  H->wl[level * 2].dirty = H->wl[level * 2 + 1].dirty = true;
  H->wl[(level - 1) * 2].dirty = H->wl[(level - 1) * 2 + 1].dirty = true;
  H->wu[level].dirty = H->wu[level - 1].dirty = true;
  H->tables_dirty = true;
  H->part_dirty = true;
  return MLSWE_OK;
}

static mlswe_status check_layout(Hier* H, int member, int level, const std::vector<Box>& boxes) {
  const Level& V = H->mem[member].lev[level];
  const Level& C = H->mem[member].lev[level - 1];
  const int r = H->cfg.ratio[level - 1];
  // overlaps: sweep over the boxes in order of i0; only boxes starting before b ends in x
  // can overlap it
  std::vector<int> ord(boxes.size());
  for (size_t a = 0; a < boxes.size(); ++a) ord[a] = (int)a;
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return boxes[x].i0 < boxes[y].i0; });
  for (size_t a = 0; a < ord.size(); ++a) {
    const Box& b = boxes[ord[a]];
    for (size_t c = a + 1; c < ord.size() && boxes[ord[c]].i0 < b.i1; ++c) {
      const Box& o = boxes[ord[c]];
      if (std::max(b.j0, o.j0) < std::min(b.j1, o.j1) && std::max(b.i0, o.i0) < std::min(b.i1, o.i1))
        return fail(H, MLSWE_ENESTING, "patches overlap");
    }
  }
  for (size_t a = 0; a < boxes.size(); ++a) {
    const Box& b = boxes[a];
    if (b.i0 < 0 || b.j0 < 0 || b.i1 > V.NX || b.j1 > V.NY || b.i1 <= b.i0 || b.j1 <= b.j0)
      return fail(H, MLSWE_ENESTING, "patch outside the domain or empty");
    if (b.i0 % r || b.j0 % r || b.i1 % r || b.j1 % r)
      return fail(H, MLSWE_ENESTING, "patch not aligned to coarse cells");
    if (level - 1 > 0) {
      // proper nesting: the patch, grown by kNest coarse cells (not across the domain
      // boundary), lies inside the union of the coarse level's patches.
      const int ci0 = b.i0 / r, cj0 = b.j0 / r, ci1 = b.i1 / r, cj1 = b.j1 / r;
      const int gi0 = std::max(0, ci0 - kNest), gj0 = std::max(0, cj0 - kNest);
      const int gi1 = std::min(C.NX, ci1 + kNest), gj1 = std::min(C.NY, cj1 + kNest);
      long long area = 0;
      for (const Box& p : C.patches) {
        const int i0 = std::max(gi0, p.i0), j0 = std::max(gj0, p.j0), i1 = std::min(gi1, p.i1), j1 = std::min(gj1, p.j1);
        if (i0 < i1 && j0 < j1) area += (long long)(i1 - i0) * (j1 - j0);
      }
      if (area != (long long)(gi1 - gi0) * (gj1 - gj0)) return fail(H, MLSWE_ENESTING, "patch not properly nested");
    }
  }
  return MLSWE_OK;
}

static mlswe_status set_patches_internal(Hier* H, int member, int level, const std::vector<Box>& boxes) {
  mlswe_status s = check_layout(H, member, level, boxes);
  if (s != MLSWE_OK) return s;
  H->mem[member].lev[level].patches = boxes;
  return rebuild_masks(H, member, level);
}

// ---- one-shot (synchronous) level transfers used by the API and by regridding ----
static mlswe_status run_items(Hier* H, int kc, const std::vector<InterpItem>& items, int kind, int r, int par_c,
                              int par_f, double alpha) {
  if (items.empty()) return MLSWE_OK;
  const size_t bytes = items.size() * sizeof(InterpItem) + 64;
  char* base = (char*)scratch_buffer(H, bytes);
  if (!base) return fail(H, MLSWE_ENOMEM, "scratch allocation failed");
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  int* d_count = (int*)base;
  InterpItem* d_items = (InterpItem*)(base + 64);
  const int n = (int)items.size();
  CUDA_TRY(H, cudaMemcpyAsync(d_count, &n, sizeof(int), cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(InterpItem), cudaMemcpyHostToDevice, H->st));
  int tok;
  timer_begin(H, kc, &tok);
  if (kind == 0)
    CUDA_TRY(H, launch_interp(H->cfg.M, H->dp, H->d_desc, d_items, d_count, grid_full(H), r, par_c, par_f, alpha,
                              H->st));
  else
    CUDA_TRY(H, launch_average_items(3 * H->cfg.M, H->d_desc, d_items, d_count, grid_full(H), r, par_c, par_f, H->st));
  timer_end(H, tok);
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  return MLSWE_OK;
}

// Refinement of the cells in `boxes` (fine indices) of (member, coarse_level + 1) from the
// current coarse state.
static mlswe_status interp_boxes(Hier* H, int member, int coarse_level, const std::vector<Box>& boxes) {
  std::vector<InterpItem> items;
  for (const Box& b : boxes)
    push_chunks(items, H->desc_index(member, coarse_level), H->desc_index(member, coarse_level + 1), b);
  return run_items(H, KC_INTERP, items, 0, H->cfg.ratio[coarse_level], H->parity[coarse_level],
                   H->parity[coarse_level + 1], 1.0);
}

// ---- the subcycled coarse step (graph-capturable: no host syncs, tables on device) ----
// Substep `substep` of `level` inside a coarse step (level 0: the coarse step itself): which
// members take it (their time ratio of the level may be below the launch's substep count),
// ghost cells at alpha = substep / rt, the level's sweeps, then the finer levels' substeps,
// coarsening and reflux onto this level.
static mlswe_status enqueue_level_tree(Hier* H, int level, int substep) {
  int tok;
  if (level > 0) {
    timer_begin(H, KC_OTHER, &tok);
    CUDA_TRY(H, launch_set_active(H->L, H->n_members, level, substep, H->d_rt, H->d_active, H->st));
    timer_end(H, tok);
    timer_begin(H, KC_GHOST, &tok);
    CUDA_TRY(H, launch_ghost_cells(H->cfg.M, H->dp, H->d_desc, H->t_gcell[level].d, H->t_gcell[level].d_count,
                                   grid_flat(H), H->cfg.ratio[level - 1], H->parity[level - 1], H->parity[level], 0.0,
                                   substep, H->st));
    timer_end(H, tok);
  }
  mlswe_status s = enqueue_level_step(H, level, 1);
  if (s != MLSWE_OK) return s;
  // Partitioned: the other ranks' patches of this level, all of them for a level with a finer
  // one; for the finest level only their cells within two of this rank's patches (the next
  // substep reads no more), after the last substep with the accumulators the reflux reads.
  int kind = MLSWE_XCHG_FULL;
  if (level == H->L - 1 && level > 0)
    kind = substep < H->cfg.ratio[level - 1] - 1 ? MLSWE_XCHG_HALO : MLSWE_XCHG_LAST;
  s = run_exchange_hook(H, level, kind);
  if (s != MLSWE_OK) return s;
  if (level + 1 < H->L) {
    const int rt = H->cfg.ratio[level];  // the most substeps any member takes
    for (int k = 0; k < rt; ++k) {
      s = enqueue_level_tree(H, level + 1, k);
      if (s != MLSWE_OK) return s;
    }
    timer_begin(H, KC_AVERAGE, &tok);
    CUDA_TRY(H, launch_average_items(3 * H->cfg.M, H->d_desc, H->t_avg[level + 1].d, H->t_avg[level + 1].d_count,
                                     grid_full(H), rt, H->parity[level], H->parity[level + 1], H->st));
    timer_end(H, tok);
    if (level + 1 == H->L - 1) {  // partitioned: each rank coarsened its own finest patches
      s = run_exchange_hook(H, level, MLSWE_XCHG_AVERAGED);
      if (s != MLSWE_OK) return s;
    }
    timer_begin(H, KC_REFLUX, &tok);
    CUDA_TRY(H, launch_reflux(H->cfg.M, H->d_desc, H->t_reflux[level].d, H->t_reflux[level].d_count, grid_flat(H), rt,
                              H->parity[level], H->st));
    timer_end(H, tok);
  }
  return MLSWE_OK;
}

static DtArgs dt_args(Hier* H) {
  DtArgs A;
  A.L = H->L;
  A.n_members = H->n_members;
  for (int k = 0; k < 4; ++k) A.ratio[k] = H->cfg.ratio[k];
  A.dynamic_rt = H->cfg.dynamic_rt;
  A.cfl = H->cfg.cfl_desired;
  A.cfl_max = H->cfg.cfl_max;
  A.has_patches = H->d_has;
  A.inv_dx = H->d_invdx;
  A.inv_dy = H->d_invdy;
  A.rt = H->d_rt;
  A.active = H->d_active;
  A.fresh = H->d_fresh;
  A.cells = H->d_cells;
  A.steps_acc = H->d_steps_acc;
  A.cells_acc = H->d_cells_acc;
  A.redo = H->d_redo;
  A.done = H->d_done;
  return A;
}

// One coarse-step attempt: time step on the device, a snapshot of the refined levels' patch
// cells, the level tree, the Courant check, and the restore of the members whose attempt
// was rejected (their next round retakes the step).
static mlswe_status enqueue_coarse_step(Hier* H) {
  int tok;
  ParSet ps{};
  for (int l = 0; l < H->L; ++l) ps.start[l] = H->parity[l];
  timer_begin(H, KC_OTHER, &tok);
  CUDA_TRY(H, launch_dt_begin(dt_args(H), H->d_smax, H->d_init, H->d_init_flag, H->d_dt, H->st));
  timer_end(H, tok);
  const int F = 3 * H->cfg.M;
  if (H->L > 1) {
    timer_begin(H, KC_OTHER, &tok);
    CUDA_TRY(H, launch_snapshot(F, H->L, H->d_desc, H->t_speed.d, H->t_speed.d_count, grid_full(H), 0, ps,
                                H->d_redo, H->st));
    timer_end(H, tok);
  }
  mlswe_status s = enqueue_level_tree(H, 0, 0);
  if (s != MLSWE_OK) return s;
  for (int l = 0; l < H->L; ++l) ps.next[l] = H->parity[l];
  timer_begin(H, KC_OTHER, &tok);
  CUDA_TRY(H, launch_step_end(dt_args(H), H->d_smax, H->d_dt, H->d_t, H->d_cfl, H->d_status, H->d_cfl_count,
                              H->st));
  timer_end(H, tok);
  timer_begin(H, KC_OTHER, &tok);
  CUDA_TRY(H, launch_snapshot(F, H->L, H->d_desc, H->t_speed.d, H->t_speed.d_count, grid_full(H), 1, ps, H->d_redo,
                              H->st));
  timer_end(H, tok);
  return MLSWE_OK;
}

// Wave speeds of the current state; the next coarse step takes its dt from them.
static mlswe_status initial_dt(Hier* H) {
  const int nd = H->n_members * H->L;
  std::vector<int> par(nd);
  for (int k = 0; k < nd; ++k) par[k] = H->parity[k % H->L];
  CUDA_TRY(H, cudaMemcpyAsync(H->d_par, par.data(), nd * 4, cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaMemsetAsync(H->d_init, 0, nd * 8, H->st));
  int tok;
  timer_begin(H, KC_OTHER, &tok);
  CUDA_TRY(H, launch_speed(H->cfg.M, H->dp, H->d_desc, H->t_speed.d, H->t_speed.d_count, grid_full(H), H->d_par,
                           H->d_init, H->st));
  timer_end(H, tok);
  static const int one = 1;
  CUDA_TRY(H, cudaMemcpyAsync(H->d_init_flag, &one, sizeof(int), cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  H->dt_ready = true;
  return MLSWE_OK;
}

// One coarse step: replay of the captured graph for the current level-0 parity, or
// direct launches (per-patch form, timing on, or graphs disabled).
static mlswe_status coarse_step(Hier* H) {
  const bool graphs = H->use_graphs && !H->per_patch_launch && !H->timer.on && H->part_hook == nullptr;
  if (!graphs) return enqueue_coarse_step(H);
  for (int l = 0; l < H->L; ++l)
    for (int dir = 0; dir < (H->cfg.unsplit ? 3 : 2); ++dir) {  // built before the capture (they sync)
      mlswe_status s = ensure_worklist(H, l, dir);
      if (s != MLSWE_OK) return s;
    }
  const int p = H->parity[0];
  if (!H->graph_valid[p]) {
    const std::vector<int> par0 = H->parity;
    const long long k0 = H->kernel_launches;
    cudaGraph_t g = nullptr;
    CUDA_TRY(H, cudaStreamBeginCapture(H->st, cudaStreamCaptureModeThreadLocal));
    mlswe_status s = enqueue_coarse_step(H);
    cudaError_t e = cudaStreamEndCapture(H->st, &g);
    if (s != MLSWE_OK) {
      if (g) cudaGraphDestroy(g);
      H->parity = par0;  // nothing ran
      return s;
    }
    if (e != cudaSuccess) return fail(H, MLSWE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    if (H->graph[p]) cudaGraphExecDestroy(H->graph[p]);
    e = cudaGraphInstantiate(&H->graph[p], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(H, MLSWE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    H->graph_valid[p] = true;
    H->graph_launches[p] = H->kernel_launches - k0;
    H->kernel_launches = k0;
    H->parity = par0;  // the capture did not run anything
  }
  CUDA_TRY(H, cudaGraphLaunch(H->graph[p], H->st));
  H->kernel_launches += H->graph_launches[p];
  // Parities after one coarse step: level l steps prod_{k<l} r_k times.
  long long steps = 1;
  for (int l = 0; l < H->L; ++l) {
    if (l > 0) steps *= H->cfg.ratio[l - 1];
    if (steps & 1) H->parity[l] ^= 1;
  }
  return MLSWE_OK;
}

static mlswe_status regrid_internal(Hier* H, int base) {
  NvtxRange range("mlswe_regrid");
  if (H->L > 1) {  // partitioned: the flags and the kept patch cells need the whole finest level
    mlswe_status s = run_exchange_hook(H, H->L - 1, MLSWE_XCHG_FULL);
    if (s != MLSWE_OK) return s;
  }
  H->regrids++;
  for (int m = 0; m < H->n_members; ++m) {
    for (int l = base; l + 1 < H->L; ++l) {
      Level& V = H->mem[m].lev[l];
      Level& Fl = H->mem[m].lev[l + 1];
      std::vector<Box> boxes;
      if (l == 0 || !V.patches.empty()) {
        const size_t cells = (size_t)V.NX * V.NY;
        uint8_t* d_flags = (uint8_t*)scratch_buffer(H, cells);
        if (!d_flags) return fail(H, MLSWE_ENOMEM, "scratch allocation failed");
        CUDA_TRY(H, cudaStreamSynchronize(H->st));
        int tok;
        timer_begin(H, KC_FLAGS, &tok);
        CUDA_TRY(H, launch_flags(H->cfg.M, H->d_desc, H->desc_index(m, l), H->parity[l], (long long)cells,
                                 H->cfg.dry_tol, 1.0 / V.dx, 1.0 / V.dy, H->cfg.flag_tol * H->cfg.flag_tol, d_flags,
                                 H->st));
        timer_end(H, tok);
        std::vector<uint8_t> fl(cells);
        CUDA_TRY(H, cudaMemcpyAsync(fl.data(), d_flags, cells, cudaMemcpyDeviceToHost, H->st));
        CUDA_TRY(H, cudaStreamSynchronize(H->st));
        boxes = cluster_flags(fl.data(), V.NX, V.NY, l, V.patches, H->cfg.ratio[l], H->cfg.n_buf, H->cfg.cluster_eff,
                              H->cfg.min_side, H->cfg.max_side, kNest);
      }
      const std::vector<Box> old = Fl.patches;
      mlswe_status s = set_patches_internal(H, m, l + 1, boxes);
      if (s != MLSWE_OK) return s;
      s = interp_boxes(H, m, l, fresh_cells(boxes, old));
      if (s != MLSWE_OK) return s;
    }
  }
  return MLSWE_OK;
}

// Autotuner of the sweep tiles of one level: times every candidate shape on the level's
// current patch layout (CUDA events, sweeps run without recording, the state is not
// advanced) and keeps the fastest per direction.
static mlswe_status autotune_level(Hier* H, int level, int iters, int* chosen) {
  NvtxRange range("mlswe_autotune");
  static const int cand[][2] = {{13, 16}, {29, 8}, {61, 4}, {125, 2}, {253, 1}};
  cudaEvent_t e0, e1;
  CUDA_TRY(H, cudaEventCreate(&e0));
  CUDA_TRY(H, cudaEventCreate(&e1));
  for (int dir = 0; dir < 2; ++dir) {
    float best = 1e30f;
    const TileShape cur = H->shape[level * 2 + dir];
    int bl = cur.len, bn = cur.lines, bc = cur.ctas;
    for (int ctas = 1; ctas <= (H->cfg.M >= 3 ? 1 : 2); ++ctas)
      for (const auto& c : cand) {
        set_level_shape(H, level, dir, c[0], c[1], ctas);
        mlswe_status s = ensure_worklist(H, level, dir);
        if (s != MLSWE_OK) return s;
        Hier::WorkList& W = H->wl[level * 2 + dir];
        if (W.count == 0) continue;
        const int par = H->parity[level];
        const int full = ctas * H->num_sms;
        const int* toff = W.packed ? W.d_tile_off : nullptr;
        CUDA_TRY(H, launch_sweep(dir, H->dp, H->d_desc, W.d_items, W.d_count, toff, full, par, 0, H->d_smax,
                                 nullptr, H->st, ctas));
        CUDA_TRY(H, cudaEventRecord(e0, H->st));
        for (int k = 0; k < iters; ++k)
          CUDA_TRY(H, launch_sweep(dir, H->dp, H->d_desc, W.d_items, W.d_count, toff, full, par, 0, H->d_smax,
                                   nullptr, H->st, ctas));
        CUDA_TRY(H, cudaEventRecord(e1, H->st));
        CUDA_TRY(H, cudaEventSynchronize(e1));
        float ms = 0.f;
        CUDA_TRY(H, cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; bl = c[0]; bn = c[1]; bc = ctas; }
      }
    set_level_shape(H, level, dir, bl, bn, bc);
    mlswe_status s = ensure_worklist(H, level, dir);
    if (s != MLSWE_OK) return s;
    if (chosen) { chosen[3 * dir] = bl; chosen[3 * dir + 1] = bn; chosen[3 * dir + 2] = bc; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  invalidate_graphs(H);
  return MLSWE_OK;
}

}  // namespace mlswe

using namespace mlswe;

extern "C" {

mlswe_status mlswe_set_patches(mlswe_h h, int member, int level, int n, const int32_t* boxes) {
  if (!h || member < 0 || member >= h->n_members || level < 1 || level >= h->L || n < 0 || (n > 0 && !boxes))
    return fail(h, MLSWE_EINVAL, "set_patches: bad argument");
  std::vector<Box> b(n);
  for (int k = 0; k < n; ++k) b[k] = Box{boxes[4 * k], boxes[4 * k + 1], boxes[4 * k + 2], boxes[4 * k + 3]};
  mlswe_status s = set_patches_internal(h, member, level, b);
  if (s == MLSWE_OK) h->dt_ready = false;
  return s;
}

mlswe_status mlswe_get_patches(mlswe_h h, int member, int level, int* n, int32_t* boxes) {
  if (!h || member < 0 || member >= h->n_members || level < 0 || level >= h->L || !n)
    return fail(h, MLSWE_EINVAL, "get_patches: bad argument");
  const std::vector<Box>& P = h->mem[member].lev[level].patches;
  const int cap = *n;
  *n = (int)P.size();
  if (boxes) {
    if (cap < (int)P.size()) return fail(h, MLSWE_EINVAL, "get_patches: capacity too small");
    for (size_t k = 0; k < P.size(); ++k) {
      boxes[4 * k] = P[k].i0; boxes[4 * k + 1] = P[k].j0; boxes[4 * k + 2] = P[k].i1; boxes[4 * k + 3] = P[k].j1;
    }
  }
  return MLSWE_OK;
}

mlswe_status mlswe_fill_ghosts(mlswe_h h, int level, double alpha) {
  if (!h || level < 1 || level >= h->L || !(alpha >= 0.0 && alpha <= 1.0))
    return fail(h, MLSWE_EINVAL, "fill_ghosts: bad argument");
  if (h->tables_dirty) {
    mlswe_status s = build_tables(h);
    if (s != MLSWE_OK) return s;
  }
  int tok;
  timer_begin(h, KC_GHOST, &tok);
  CUDA_TRY(h, launch_ghost_cells(h->cfg.M, h->dp, h->d_desc, h->t_gcell[level].d, h->t_gcell[level].d_count,
                                 grid_flat(h), h->cfg.ratio[level - 1], h->parity[level - 1], h->parity[level], alpha,
                                 -1, h->st));
  timer_end(h, tok);
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return MLSWE_OK;
}

mlswe_status mlswe_interp_fine(mlswe_h h, int coarse_level, int member) {
  if (!h || member < 0 || member >= h->n_members || coarse_level < 0 || coarse_level + 1 >= h->L)
    return fail(h, MLSWE_EINVAL, "interp_fine: bad argument");
  h->dt_ready = false;
  return interp_boxes(h, member, coarse_level, h->mem[member].lev[coarse_level + 1].patches);
}

mlswe_status mlswe_average_coarse(mlswe_h h, int fine_level, int member) {
  if (!h || member < 0 || member >= h->n_members || fine_level < 1 || fine_level >= h->L)
    return fail(h, MLSWE_EINVAL, "average_coarse: bad argument");
  std::vector<InterpItem> items;
  const int r = h->cfg.ratio[fine_level - 1];
  for (const Box& b : h->mem[member].lev[fine_level].patches)
    push_chunks(items, h->desc_index(member, fine_level - 1), h->desc_index(member, fine_level),
                Box{b.i0 / r, b.j0 / r, b.i1 / r, b.j1 / r});
  h->dt_ready = false;
  return run_items(h, KC_AVERAGE, items, 1, r, h->parity[fine_level - 1], h->parity[fine_level], 1.0);
}

mlswe_status mlswe_get_flags(mlswe_h h, int member, int level, uint8_t* flags) {
  if (!h || member < 0 || member >= h->n_members || level < 0 || level >= h->L || !flags)
    return fail(h, MLSWE_EINVAL, "get_flags: bad argument");
  const Level& V = h->mem[member].lev[level];
  const size_t cells = (size_t)V.NX * V.NY;
  uint8_t* d = (uint8_t*)scratch_buffer(h, cells);
  if (!d) return fail(h, MLSWE_ENOMEM, "scratch allocation failed");
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  int tok;
  timer_begin(h, KC_FLAGS, &tok);
  CUDA_TRY(h, launch_flags(h->cfg.M, h->d_desc, h->desc_index(member, level), h->parity[level], (long long)cells,
                           h->cfg.dry_tol, 1.0 / V.dx, 1.0 / V.dy, h->cfg.flag_tol * h->cfg.flag_tol, d, h->st));
  timer_end(h, tok);
  CUDA_TRY(h, cudaMemcpyAsync(flags, d, cells, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return MLSWE_OK;
}

mlswe_status mlswe_regrid(mlswe_h h, int base_level) {
  if (!h || base_level < 0 || base_level >= h->L) return fail(h, MLSWE_EINVAL, "regrid: bad argument");
  mlswe_status s = regrid_internal(h, base_level);
  if (s != MLSWE_OK) return s;
  h->dt_ready = false;
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return MLSWE_OK;
}

// Kept coarse steps of every member (host copy of the device counters).
static mlswe_status read_done(Hier* H, std::vector<long long>& done) {
  done.resize(H->n_members);
  CUDA_TRY(H, cudaMemcpyAsync(done.data(), H->d_done, H->n_members * 8, cudaMemcpyDeviceToHost, H->st));
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  return MLSWE_OK;
}

// Level-0 activity of every member (a member that sits a round out takes no step on any level).
static mlswe_status set_member_active(Hier* H, const std::vector<int>& act) {
  CUDA_TRY(H, cudaMemcpy2DAsync(H->d_active, (size_t)H->L * sizeof(int), act.data(), sizeof(int), sizeof(int),
                                H->n_members, cudaMemcpyHostToDevice, H->st));
  return MLSWE_OK;
}

mlswe_status mlswe_advance(mlswe_h h, int n_coarse_steps) {
  if (!h || n_coarse_steps < 0) return fail(h, MLSWE_EINVAL, "advance: bad argument");
  NvtxRange range("mlswe_advance");
  CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, 4, h->st));
  mlswe_status s = ensure_snapshots(h);
  if (s != MLSWE_OK) return s;
  std::vector<long long> target;
  s = read_done(h, target);
  if (s != MLSWE_OK) return s;
  for (long long& t : target) t += n_coarse_steps;
  for (int k = 0; k < n_coarse_steps; ++k) {
    if (h->cfg.regrid_interval > 0 && h->L > 1 && h->coarse_steps % h->cfg.regrid_interval == 0) {
      s = regrid_internal(h, 0);
      if (s != MLSWE_OK) return s;
      static const int one = 1;  // the next step takes the fixed time ratios
      CUDA_TRY(h, cudaMemcpyAsync(h->d_fresh, &one, sizeof(int), cudaMemcpyHostToDevice, h->st));
    }
    if (h->tables_dirty) {
      s = build_tables(h);
      if (s != MLSWE_OK) return s;
    }
    if (!h->dt_ready) {
      s = initial_dt(h);
      if (s != MLSWE_OK) return s;
    }
    {
      NvtxRange step_range("mlswe_coarse_step");
      s = coarse_step(h);
    }
    if (s != MLSWE_OK) return s;
    h->coarse_steps++;  // level steps and cell updates are counted on the device (dt_begin)
  }
  // Retake rounds (no regrid): members whose rejected attempts left them short of n kept
  // steps step again, the others sit the rounds out.
  bool masked = false;
  bool gave_up = false;
  for (int extra = 0;; ++extra) {
    std::vector<long long> done;
    s = read_done(h, done);
    if (s != MLSWE_OK) return s;
    std::vector<int> act(h->n_members, 0);
    bool any = false;
    for (int m = 0; m < h->n_members; ++m)
      if (done[m] < target[m]) { act[m] = 1; any = true; }
    if (!any) break;
    if (extra >= n_coarse_steps + 8) { gave_up = true; break; }
    s = set_member_active(h, act);
    if (s != MLSWE_OK) return s;
    masked = true;
    NvtxRange step_range("mlswe_coarse_step_retake");
    s = coarse_step(h);
    if (s != MLSWE_OK) return s;
  }
  if (masked) {
    s = set_member_active(h, std::vector<int>(h->n_members, 1));
    if (s != MLSWE_OK) return s;
  }
  if (h->L > 1) {  // partitioned: every rank's finest level whole again for the caller
    s = run_exchange_hook(h, h->L - 1, MLSWE_XCHG_FULL);
    if (s != MLSWE_OK) return s;
  }
  unsigned int status = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&status, h->d_status, 4, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  if (status & 2u) return fail(h, MLSWE_ENEGDEPTH, "non-finite wave speed in a step");
  if (gave_up)
    return fail(h, MLSWE_ECFL, "Courant number above cfl_max in every retake of a step (retake budget spent)");
  return MLSWE_OK;
}

static int clock_doubles(mlswe_h h) { return h->n_members * (1 + 3 * h->L) + 3; }

mlswe_status mlswe_get_clock(mlswe_h h, double* buf, int n_doubles) {
  if (!h || !buf || n_doubles != clock_doubles(h)) return fail(h, MLSWE_EINVAL, "get_clock: bad argument");
  const int n = h->n_members, nd = n * h->L;
  CUDA_TRY(h, cudaMemcpyAsync(buf, h->d_t, n * 8, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(buf + n, h->d_smax, (size_t)2 * nd * 8, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(buf + n + 2 * nd, h->d_init, (size_t)nd * 8, cudaMemcpyDeviceToHost, h->st));
  int flag = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&flag, h->d_init_flag, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  buf[n + 3 * nd] = flag;
  buf[n + 3 * nd + 1] = h->dt_ready ? 1.0 : 0.0;
  buf[n + 3 * nd + 2] = (double)h->coarse_steps;
  return MLSWE_OK;
}

mlswe_status mlswe_set_clock(mlswe_h h, const double* buf, int n_doubles) {
  if (!h || !buf || n_doubles != clock_doubles(h)) return fail(h, MLSWE_EINVAL, "set_clock: bad argument");
  const int n = h->n_members, nd = n * h->L;
  const int flag = buf[n + 3 * nd] != 0.0 ? 1 : 0;
  CUDA_TRY(h, cudaMemcpyAsync(h->d_t, buf, n * 8, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_smax, buf + n, (size_t)2 * nd * 8, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_init, buf + n + 2 * nd, (size_t)nd * 8, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_init_flag, &flag, sizeof(int), cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  h->dt_ready = buf[n + 3 * nd + 1] != 0.0;
  h->coarse_steps = (long long)buf[n + 3 * nd + 2];
  return MLSWE_OK;
}

mlswe_status mlswe_get_time(mlswe_h h, double* t_out, double* dt_out) {
  if (!h) return MLSWE_EINVAL;
  std::vector<double> t(h->n_members), dt(h->n_members * h->L);
  CUDA_TRY(h, cudaMemcpyAsync(t.data(), h->d_t, t.size() * 8, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(dt.data(), h->d_dt, dt.size() * 8, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  if (t_out) for (int m = 0; m < h->n_members; ++m) t_out[m] = t[m];
  if (dt_out) for (int m = 0; m < h->n_members; ++m) dt_out[m] = dt[m * h->L];
  return MLSWE_OK;
}

mlswe_status mlswe_set_execution(mlswe_h h, int use_graphs, int per_patch_launches) {
  if (!h) return MLSWE_EINVAL;
  if (per_patch_launches && h->part_size > 1) return fail(h, MLSWE_EINVAL, "set_execution: partitioned hierarchy");
  h->use_graphs = use_graphs != 0;
  if (h->per_patch_launch != (per_patch_launches != 0))
    for (auto& W : h->wl) W.dirty = true;  // packed tiles (batched) or tiles per patch
  h->per_patch_launch = per_patch_launches != 0;
  invalidate_graphs(h);
  return MLSWE_OK;
}

mlswe_status mlswe_autotune(mlswe_h h, int level, int iters, int* chosen) {
  if (!h || level < 0 || level >= h->L || iters < 1) return fail(h, MLSWE_EINVAL, "autotune: bad argument");
  return autotune_level(h, level, iters, chosen);
}

}  // extern "C"
