// Hierarchy management and the C ABI (see include/mlswe.h).
//
// Every level of every member is one dense device array over the whole
// domain at that level's resolution (GB300's 288 GB of HBM make this cheap
// for the workloads here); patches are index boxes into it. Sibling patches
// therefore share their ghost cells in place, and the solver kernels need no
// patch-to-patch indirection.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include "mlswe_internal.h"

namespace mlswe {

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

void* dev_alloc(Hier* H, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (H->own_alloc) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  } else {
    p = H->alloc.alloc(bytes, (void*)H->st, H->alloc.ctx);
  }
  if (p) H->allocations.push_back(p);
  return p;
}

void dev_free(Hier* H, void* p) {
  if (!p) return;
  auto it = std::find(H->allocations.begin(), H->allocations.end(), p);
  if (it != H->allocations.end()) H->allocations.erase(it);
  if (H->own_alloc) cudaFree(p);
  else H->alloc.free(p, (void*)H->st, H->alloc.ctx);
}

// Per-call device scratch (gauges, flags); the stream is synchronised before reuse.
void* scratch_buffer(Hier* H, size_t bytes) {
  if (bytes > H->scratch_bytes) {
    cudaStreamSynchronize(H->st);
    if (H->scratch) dev_free(H, H->scratch);
    H->scratch_bytes = std::max<size_t>(bytes * 2, 1 << 16);
    H->scratch = dev_alloc(H, H->scratch_bytes);
    if (!H->scratch) H->scratch_bytes = 0;
  }
  return H->scratch;
}

void invalidate_graphs(Hier* H) {
  for (int p = 0; p < 2; ++p) {
    if (H->graph[p]) cudaGraphExecDestroy(H->graph[p]);
    H->graph[p] = nullptr;
    H->graph_valid[p] = false;
  }
}

void timer_begin(Hier* H, int kc, int* token) {
  H->kernel_launches++;
  *token = -1;
  LaunchTimer& T = H->timer;
  if (!T.on) return;
  if (T.next + 2 > T.pool.size()) {
    for (int k = 0; k < 256; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      T.pool.push_back(e);
    }
  }
  const int e0 = (int)T.next++, e1 = (int)T.next++;
  cudaEventRecord(T.pool[e0], H->st);
  T.recs.push_back({kc, e0, e1});
  *token = (int)T.recs.size() - 1;
}

void timer_end(Hier* H, int token) {
  if (token < 0) return;
  LaunchTimer& T = H->timer;
  cudaEventRecord(T.pool[T.recs[token].e1], H->st);
}

// Folds recorded events into the per-class totals (synchronises the stream).
static void timer_collect(Hier* H) {
  LaunchTimer& T = H->timer;
  if (T.recs.empty()) return;
  cudaStreamSynchronize(H->st);
  for (const auto& r : T.recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, T.pool[r.e0], T.pool[r.e1]) == cudaSuccess) {
      T.ms[r.kc] += ms;
      T.launches[r.kc] += 1;
    }
  }
  T.recs.clear();
  T.next = 0;
}

void fill_dev_params(const mlswe_config* cfg, DevParams* P) {
  P->M = cfg->M; P->g = cfg->g; P->r = cfg->M == 2 ? cfg->rho[0] / cfg->rho[1] : 1.0;
  P->omr = 1.0 - P->r; P->four_r = 4.0 * P->r; P->omr_g = (1.0 - P->r) * cfg->g;
  for (int m = 0; m < 4; ++m) P->rho[m] = m < cfg->M ? cfg->rho[m] : 0.0;
  for (int m = 0; m < 4; ++m) {
    P->irho[m] = m < cfg->M ? 1.0 / cfg->rho[m] : 0.0;
    for (int n = 0; n < 4; ++n) P->rr[n][m] = n < cfg->M && m < cfg->M ? cfg->rho[n] / cfg->rho[m] : 0.0;
    P->gap_g[m] = m + 1 < cfg->M ? (1.0 - cfg->rho[m] / cfg->rho[m + 1]) * cfg->g : 0.0;
  }
  P->dry_tol = cfg->dry_tol; P->order = cfg->order; P->limiter = cfg->limiter; P->eigen = cfg->eigen;
  P->unsplit = cfg->unsplit;
}

static mlswe_status upload_desc(Hier* H) {
  const int nd = H->n_members * H->L;
  std::vector<LevelDesc> d(nd);
  std::vector<double> idx(nd), idy(nd);
  for (int m = 0; m < H->n_members; ++m)
    for (int l = 0; l < H->L; ++l) {
      const Level& V = H->mem[m].lev[l];
      const int k = H->desc_index(m, l);
      LevelDesc& D = d[k];
      D.q[0] = V.q[0]; D.q[1] = V.q[1]; D.qs = V.qs; D.B = V.B;
      D.in_patch = V.in_patch; D.covered = V.covered;
      D.fxc = V.fxc; D.fyc = V.fyc; D.fxf = V.fxf; D.fyf = V.fyf;
      D.dt = H->d_dt + k;
      D.rt = H->d_rt + k;
      D.active = H->d_active + k;
      D.NX = V.NX; D.NY = V.NY; D.P = V.P;
      D.inv_dx = 1.0 / V.dx; D.inv_dy = 1.0 / V.dy;
      D.ue = V.ue; D.uxp = V.uxp; D.uyp = V.uyp;
      D.snap = V.snap;
      idx[k] = D.inv_dx; idy[k] = D.inv_dy;
    }
  CUDA_TRY(H, cudaMemcpyAsync(H->d_desc, d.data(), d.size() * sizeof(LevelDesc), cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaMemcpyAsync(H->d_invdx, idx.data(), nd * 8, cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaMemcpyAsync(H->d_invdy, idy.data(), nd * 8, cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  return MLSWE_OK;
}

// Snapshot buffers of levels >= 1 for the Courant control of mlswe_advance (one state array
// per level and member, allocated at the first advance of a multi-level hierarchy).
mlswe_status ensure_snapshots(Hier* H) {
  if (H->snaps_ready || H->L < 2) return MLSWE_OK;
  const int F = 3 * H->cfg.M;
  for (int m = 0; m < H->n_members; ++m)
    for (int l = 1; l < H->L; ++l) {
      Level& V = H->mem[m].lev[l];
      if (V.snap) continue;
      V.snap = (double*)dev_alloc(H, (size_t)V.NY * V.P * F * 8);
      if (!V.snap) return fail(H, MLSWE_ENOMEM, "advance: snapshot allocation failed");
    }
  mlswe_status s = upload_desc(H);
  if (s != MLSWE_OK) return s;
  invalidate_graphs(H);
  H->snaps_ready = true;
  return MLSWE_OK;
}

static bool valid_member_level(Hier* H, int member, int level) {
  return H && member >= 0 && member < H->n_members && level >= 0 && level < H->L;
}

// Tile of a patch for the sweeps: `len` cells along the sweep times as many lines as fill
// kMaxEdges edges (at least ts.lines, at most 32), so narrow patches still give every thread
// an edge. len is ts.len on patches at least twice that long (a shorter last tile), else the
// patch extent split into equal parts of at most ts.len cells.
static void tile_dims(const TileShape& ts, int extent, int* len, int* lines) {
  if (extent >= 2 * ts.len) {
    *len = ts.len;
  } else {
    const int parts = (extent + ts.len - 1) / ts.len;
    *len = (extent + parts - 1) / parts;
  }
  *lines = std::max(ts.lines, std::min(32, kMaxEdges / (*len + 3)));
}

long long patch_cells(const Hier* H, int level) {
  long long c = 0;
  for (int m = 0; m < H->n_members; ++m)
    for (const Box& b : H->mem[m].lev[level].patches) c += (long long)(b.i1 - b.i0) * (b.j1 - b.j0);
  return c;
}

// Sweep work list of one level: tiles over every patch of every member, grouped by patch.
static void build_items(Hier* H, int level, int dir, std::vector<SweepItem>& out, std::vector<int>& patch_off) {
  out.clear();
  patch_off.clear();
  const TileShape ts = H->shape[level * 2 + (dir == 2 ? 0 : dir)];
  for (int m = 0; m < H->n_members; ++m) {
    const Level& V = H->mem[m].lev[level];
    const int desc = H->desc_index(m, level);
    for (const Box& b : V.patches) {
      patch_off.push_back((int)out.size());
      int tl, tn;
      tile_dims(ts, dir != 1 ? b.i1 - b.i0 : b.j1 - b.j0, &tl, &tn);
      if (dir == 2) {
        // update tiles of the unsplit step: up to kUpdRows rows of the patch, the row split
        // into equal parts of at most kUpdLen cells
        const int parts = (b.w() + kUpdLen - 1) / kUpdLen;
        tl = (b.w() + parts - 1) / parts;
        tn = kUpdRows;
        for (int j = b.j0; j < b.j1; j += tn) {
          const int nl = std::min(tn, b.j1 - j);
          for (int i = b.i0; i < b.i1; i += tl) {
            SweepItem it;
            it.desc = desc; it.i0 = i; it.j0 = j; it.len = std::min(tl, b.i1 - i);
            it.nlines = nl; it.flags = 1;
            out.push_back(it);
          }
        }
      } else if (H->cfg.unsplit) {
        // edge passes of the unsplit step: the patch's lines and one ghost line on each side
        // (mirrored where it lies beyond the domain)
        const int lo = dir == 0 ? b.j0 : b.i0, hi = dir == 0 ? b.j1 : b.i1;
        const int a0 = dir == 0 ? b.i0 : b.j0, a1 = dir == 0 ? b.i1 : b.j1;
        for (int seg = 0; seg < 3; ++seg) {
          const int s0 = seg == 0 ? lo - 1 : (seg == 1 ? lo : hi);
          const int s1 = seg == 0 ? lo : (seg == 1 ? hi : hi + 1);
          for (int x = s0; x < s1; x += tn) {
            const int nl = std::min(tn, s1 - x);
            for (int a = a0; a < a1; a += tl) {
              SweepItem it;
              it.desc = desc;
              it.len = std::min(tl, a1 - a);
              if (dir == 0) { it.i0 = a; it.j0 = x; } else { it.i0 = x; it.j0 = a; }
              it.nlines = nl;
              it.flags = (seg == 1 ? 1 : 0) | (a + it.len == a1 ? 2 : 0);
              out.push_back(it);
            }
          }
        }
      } else if (dir == 0) {
        // Rows of the patch, plus (refined levels) the two ghost rows on each side that
        // lie in the domain: the y sweep reads Q* there.
        const int g = level > 0 ? kNG : 0;
        const int jlo = std::max(0, b.j0 - g), jhi = std::min(V.NY, b.j1 + g);
        int j = jlo;
        while (j < jhi) {
          const bool inter = j >= b.j0 && j < b.j1;
          int jend = inter ? b.j1 : (j < b.j0 ? b.j0 : jhi);
          jend = std::min(jend, jhi);
          for (int jj = j; jj < jend; jj += tn) {
            const int nl = std::min(tn, jend - jj);
            for (int i = b.i0; i < b.i1; i += tl) {
              SweepItem it;
              it.desc = desc; it.i0 = i; it.j0 = jj; it.len = std::min(tl, b.i1 - i);
              it.nlines = nl; it.flags = (inter ? 1 : 0) | (i + it.len == b.i1 ? 2 : 0);
              out.push_back(it);
            }
          }
          j = jend;
        }
      } else {
        for (int i = b.i0; i < b.i1; i += tn) {
          const int nl = std::min(tn, b.i1 - i);
          for (int j = b.j0; j < b.j1; j += tl) {
            SweepItem it;
            it.desc = desc; it.i0 = i; it.j0 = j; it.len = std::min(tl, b.j1 - j);
            it.nlines = nl; it.flags = 1 | (j + it.len == b.j1 ? 2 : 0);
            out.push_back(it);
          }
        }
      }
    }
  }
  patch_off.push_back((int)out.size());
}

// Runs of patch lines for the packed (batched) form: for every patch and every part of its
// lines (the tile length of tile_dims), one item holding all consecutive lines of one kind;
// pack_tiles then cuts and packs them into tiles.
// The x sweep of a refined level also sweeps the two rows above and below each patch (the y
// sweep reads its result there). Where such a row runs through another patch swept here, that
// patch's own x sweep already writes the same values (an x-sweep value depends on its row
// only), so those columns are left out: the parts of ghost row r of patch p that no patch q
// (swept by this rank) with q.j0 <= r < q.j1 covers.
static void ghost_row_parts(const std::vector<Box>& P, const std::vector<int>& near, const Box& b, int r,
                            const std::vector<char>& swept, std::vector<std::pair<int, int>>& parts) {
  parts.assign(1, {b.i0, b.i1});
  for (int q : near) {
    const Box& Q = P[q];
    if (!swept[q] || r < Q.j0 || r >= Q.j1) continue;
    std::vector<std::pair<int, int>> next;
    for (const auto& iv : parts) {
      if (Q.i1 <= iv.first || Q.i0 >= iv.second) { next.push_back(iv); continue; }
      if (iv.first < Q.i0) next.push_back({iv.first, Q.i0});
      if (Q.i1 < iv.second) next.push_back({Q.i1, iv.second});
    }
    parts.swap(next);
  }
}

static void build_segments(Hier* H, int level, int dir, std::vector<SweepItem>& out) {
  out.clear();
  const TileShape ts = H->shape[level * 2 + dir];
  const bool ghost_rows = !H->cfg.unsplit && dir == 0 && level > 0;
  for (int m = 0; m < H->n_members; ++m) {
    const Level& V = H->mem[m].lev[level];
    const int desc = H->desc_index(m, level);
    std::vector<std::vector<int>> near;
    std::vector<char> swept(V.patches.size(), 0);
    for (int p = 0; p < (int)V.patches.size(); ++p) swept[p] = patch_owned(H, m, level, p) ? 1 : 0;
    if (ghost_rows) near = patches_near(V.patches, kNG);
    std::vector<std::pair<int, int>> pa, pb;
    for (int p = 0; p < (int)V.patches.size(); ++p) {
      if (!swept[p]) continue;  // another rank sweeps it
      const Box& b = V.patches[p];
      const int lo = dir == 0 ? b.j0 : b.i0, hi = dir == 0 ? b.j1 : b.i1;
      int tl, tn;
      tile_dims(ts, dir == 0 ? b.w() : b.h(), &tl, &tn);
      if (!ghost_rows) {
        int g0 = lo, g1 = hi;  // lines processed: the patch's (unsplit: one ghost line each side)
        if (H->cfg.unsplit) { g0 = lo - 1; g1 = hi + 1; }
        patch_segments(b, dir, tl, g0, g1, desc, out);
        continue;
      }
      // ghost rows below, the patch's rows, ghost rows above; consecutive ghost rows with the
      // same parts form one run
      auto ghost = [&](int r0, int r1) {
        int r = r0;
        while (r < r1) {
          ghost_row_parts(V.patches, near[p], b, r, swept, pa);
          int e = r + 1;
          while (e < r1) {
            ghost_row_parts(V.patches, near[p], b, e, swept, pb);
            if (pb != pa) break;
            ++e;
          }
          for (const auto& iv : pa) patch_segments(Box{iv.first, r, iv.second, r}, dir, tl, r, e, desc, out);
          r = e;
        }
      };
      ghost(std::max(0, lo - kNG), lo);
      patch_segments(b, dir, tl, lo, hi, desc, out);
      ghost(hi, std::min(V.NY, hi + kNG));
    }
  }
}

mlswe_status ensure_worklist(Hier* H, int level, int dir) {
  Hier::WorkList& W = dir == 2 ? H->wu[level] : H->wl[level * 2 + dir];
  if (!W.dirty) return MLSWE_OK;
  if (H->part_size > 1) {
    mlswe_status s = ensure_partition(H);
    if (s != MLSWE_OK) return s;
  }
  std::vector<SweepItem> items;
  build_items(H, level, dir, items, W.patch_off);
  // batched form: groups of lines packed into tiles (the per-patch form keeps a tile per item)
  std::vector<int> toff;
  W.packed = dir != 2 && !H->per_patch_launch;
  if (W.packed) {
    std::vector<SweepItem> segs;
    build_segments(H, level, dir, segs);
    if (!pack_tiles(segs, dir, items, toff)) return fail(H, MLSWE_EINVAL, "sweep tiles: line longer than a tile");
  }
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  if ((int)items.size() > W.capacity) {
    if (W.d_items) dev_free(H, W.d_items);
    const int cap = std::max<int>(1024, (int)items.size() * 3 / 2);
    W.d_items = (SweepItem*)dev_alloc(H, cap * sizeof(SweepItem));
    if (!W.d_items) return fail(H, MLSWE_ENOMEM, "work list allocation failed");
    W.capacity = cap;
    invalidate_graphs(H);
  }
  const int np = (int)W.patch_off.size() - 1;
  if (np + 1 > W.patch_cap) {
    if (W.d_patch_count) dev_free(H, W.d_patch_count);
    W.patch_cap = std::max(64, (np + 1) * 3 / 2);
    W.d_patch_count = (int*)dev_alloc(H, W.patch_cap * sizeof(int));
    if (!W.d_patch_count) return fail(H, MLSWE_ENOMEM, "work list allocation failed");
  }
  if (!W.d_count) {
    W.d_count = (int*)dev_alloc(H, sizeof(int));
    if (!W.d_count) return fail(H, MLSWE_ENOMEM, "work list allocation failed");
  }
  if (W.packed && (int)toff.size() > W.tile_cap) {
    if (W.d_tile_off) dev_free(H, W.d_tile_off);
    W.tile_cap = std::max<int>(1024, (int)toff.size() * 3 / 2);
    W.d_tile_off = (int*)dev_alloc(H, W.tile_cap * sizeof(int));
    if (!W.d_tile_off) return fail(H, MLSWE_ENOMEM, "work list allocation failed");
    invalidate_graphs(H);
  }
  std::vector<int> pc(std::max(np, 1), 0);
  for (int p = 0; p < np; ++p) pc[p] = W.patch_off[p + 1] - W.patch_off[p];
  W.count = (int)items.size();
  W.ntiles = W.packed ? (int)toff.size() - 1 : W.count;
  if (!items.empty())
    CUDA_TRY(H, cudaMemcpyAsync(W.d_items, items.data(), items.size() * sizeof(SweepItem), cudaMemcpyHostToDevice, H->st));
  if (W.packed)
    CUDA_TRY(H, cudaMemcpyAsync(W.d_tile_off, toff.data(), toff.size() * sizeof(int), cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaMemcpyAsync(W.d_count, &W.ntiles, sizeof(int), cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaMemcpyAsync(W.d_patch_count, pc.data(), pc.size() * sizeof(int), cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  W.dirty = false;
  return MLSWE_OK;
}

// Launch the two sweeps of one level step (device work only, no host sync).
// Batched form: one persistent launch per sweep over the tiles of every patch of every
// member. Per-patch form (comparison only): one launch per patch and sweep.
mlswe_status enqueue_level_step(Hier* H, int level, int record) {
  for (int dir = 0; dir < (H->cfg.unsplit ? 3 : 2); ++dir) {
    mlswe_status s = ensure_worklist(H, level, dir);
    if (s != MLSWE_OK) return s;
  }
  const int par = H->parity[level];
  for (int dir = 0; dir < 2; ++dir) {
    Hier::WorkList& W = H->wl[level * 2 + dir];
    const int ctas = H->shape[level * 2 + dir].ctas;
    const int full = ctas * H->num_sms;
    if (!H->per_patch_launch) {
      // Always launched (also with no items): a captured graph must hold the node for
      // when a later regrid fills the work list.
      int tok;
      timer_begin(H, dir == 0 ? KC_SWEEP_X : KC_SWEEP_Y, &tok);
      CUDA_TRY(H, launch_sweep(dir, H->dp, H->d_desc, W.d_items, W.d_count, W.packed ? W.d_tile_off : nullptr,
                               full, par, record, H->d_smax, H->d_lost, H->st, ctas));
      timer_end(H, tok);
    } else {
      const int np = (int)W.patch_off.size() - 1;
      for (int p = 0; p < np; ++p) {
        const int cnt = W.patch_off[p + 1] - W.patch_off[p];
        if (cnt == 0) continue;
        int tok;
        timer_begin(H, dir == 0 ? KC_SWEEP_X : KC_SWEEP_Y, &tok);
        CUDA_TRY(H, launch_sweep(dir, H->dp, H->d_desc, W.d_items + W.patch_off[p], W.d_patch_count + p, nullptr,
                                 std::min(cnt, full), par, record, H->d_smax, H->d_lost, H->st, ctas));
        timer_end(H, tok);
      }
    }
  }
  if (H->cfg.unsplit) {
    // the cell update after both edge passes (4 CTAs of 256 threads per SM)
    Hier::WorkList& W = H->wu[level];
    const int full = 4 * H->num_sms;
    if (!H->per_patch_launch) {
      int tok;
      timer_begin(H, KC_UPDATE, &tok);
      CUDA_TRY(H, launch_unsplit_update(H->dp, H->d_desc, W.d_items, W.d_count, full, par, record, H->st));
      timer_end(H, tok);
    } else {
      const int np = (int)W.patch_off.size() - 1;
      for (int p = 0; p < np; ++p) {
        const int cnt = W.patch_off[p + 1] - W.patch_off[p];
        if (cnt == 0) continue;
        int tok;
        timer_begin(H, KC_UPDATE, &tok);
        CUDA_TRY(H, launch_unsplit_update(H->dp, H->d_desc, W.d_items + W.patch_off[p], W.d_patch_count + p,
                                          std::min(cnt, full), par, record, H->st));
        timer_end(H, tok);
      }
    }
  }
  H->parity[level] ^= 1;
  return MLSWE_OK;
}

static mlswe_status level_cfl(Hier* H, int level, double* cfl_out, bool* nan_seen) {
  std::vector<unsigned long long> bits(H->n_members * H->L * 2);
  CUDA_TRY(H, cudaMemcpyAsync(bits.data(), H->d_smax, bits.size() * 8, cudaMemcpyDeviceToHost, H->st));
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  *nan_seen = false;
  for (int m = 0; m < H->n_members; ++m) {
    const int d = H->desc_index(m, level);
    double sx, sy;
    std::memcpy(&sx, &bits[2 * d], 8);
    std::memcpy(&sy, &bits[2 * d + 1], 8);
    if (std::isnan(sx) || std::isnan(sy)) *nan_seen = true;
    const Level& V = H->mem[m].lev[level];
    const double dt = H->h_dt[d];
    if (cfl_out) cfl_out[m] = dt * std::max(sx / V.dx, sy / V.dy);
  }
  return MLSWE_OK;
}

static bool shape_ok(int len, int lines) {
  return len >= 4 && lines >= 1 && lines <= 32 && lines * (len + 3) <= kMaxEdges && lines * (len + 4) <= kMaxCells;
}

void set_level_shape(Hier* H, int level, int dir, int len, int lines, int ctas) {
  H->shape[level * 2 + dir].len = len;
  H->shape[level * 2 + dir].lines = lines;
  H->shape[level * 2 + dir].ctas = ctas;
  H->wl[level * 2 + dir].dirty = true;
}

}  // namespace mlswe

using namespace mlswe;

extern "C" {

const char* mlswe_last_error(mlswe_h h) { return h ? h->err.c_str() : "null handle"; }

mlswe_status mlswe_create_hierarchy(const mlswe_config* cfg, int n_members, const mlswe_domain* doms,
                                    const mlswe_allocator* alloc, void* cuda_stream, mlswe_h* out) {
  if (!cfg || !doms || !out || n_members <= 0) return MLSWE_EINVAL;
  *out = nullptr;
  if (cfg->M < 1 || cfg->M > 4 || cfg->max_levels < 1 || cfg->max_levels > 4) return MLSWE_EINVAL;
  if (cfg->order < 1 || cfg->order > 2 || cfg->limiter < 0 || cfg->limiter > 2) return MLSWE_EINVAL;
  if (cfg->eigen < 0 || cfg->eigen > 1 || !(cfg->dry_tol >= 0.0) || !(cfg->g > 0.0)) return MLSWE_EINVAL;
  if (cfg->dynamic_rt < 0 || cfg->dynamic_rt > 1) return MLSWE_EINVAL;
  if (cfg->unsplit < 0 || cfg->unsplit > 1) return MLSWE_EINVAL;
  if (cfg->unsplit && cfg->M > 3) return MLSWE_EINVAL;  // the transverse solves take at most three layers
  if (cfg->M >= 2 && !(cfg->rho[0] > 0.0)) return MLSWE_EINVAL;
  for (int m = 0; m + 1 < cfg->M; ++m)  // densities increase downwards (stable stratification)
    if (!(cfg->rho[m] < cfg->rho[m + 1])) return MLSWE_EINVAL;
  for (int l = 0; l + 1 < cfg->max_levels; ++l)
    if (cfg->ratio[l] != 2 && cfg->ratio[l] != 4) return MLSWE_EINVAL;
  if (cfg->max_levels > 1 && (cfg->min_side < 1 || cfg->max_side < 2 * cfg->min_side)) return MLSWE_EINVAL;
  for (int m = 0; m < n_members; ++m)
    if (doms[m].nx0 < 4 || doms[m].ny0 < 4 || !(doms[m].x1 > doms[m].x0) || !(doms[m].y1 > doms[m].y0))
      return MLSWE_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MLSWE_EMISSING;
  mlswe_hier* H = new (std::nothrow) mlswe_hier();
  if (!H) return MLSWE_ENOMEM;
  H->cfg = *cfg;
  H->n_members = n_members;
  H->L = cfg->max_levels;
  H->st = (cudaStream_t)cuda_stream;
  if (!H->st) {
    // The legacy default stream cannot be captured into a graph: own a stream instead.
    if (cudaStreamCreateWithFlags(&H->st, cudaStreamNonBlocking) != cudaSuccess) { delete H; return MLSWE_ECUDA; }
    H->own_stream = true;
  }
  if (alloc && alloc->alloc && alloc->free) { H->alloc = *alloc; H->own_alloc = false; }
  fill_dev_params(cfg, &H->dp);
  cudaDeviceGetAttribute(&H->num_sms, cudaDevAttrMultiProcessorCount, dev);
  H->parity.assign(H->L, 0);
  H->wl.resize(H->L * 2);
  H->wu.resize(H->L);
  H->shape.resize(H->L * 2);
  for (int l = 0; l < H->L; ++l) {
    // Default tiles: 125-cell rows x 2 (x sweep), 125-cell columns x 2 (y sweep); 256 edges;
    // 2 CTAs per SM (the autotuner's choice on every workload measured); one for three layers,
    // whose sweep needs the whole register file and most of the shared memory.
    const int ctas = cfg->M >= 3 ? 1 : 2;
    H->shape[l * 2] = TileShape{125, 2, ctas};
    H->shape[l * 2 + 1] = TileShape{125, 2, ctas};
  }
  H->t_avg.resize(H->L);
  H->t_reflux.resize(H->L);
  H->t_gcell.resize(H->L);
  H->mem.resize(n_members);
  const int F = 3 * cfg->M;
  for (int m = 0; m < n_members; ++m) {
    Member& Mb = H->mem[m];
    Mb.dom = doms[m];
    Mb.lev.resize(H->L);
    int nx = doms[m].nx0, ny = doms[m].ny0;
    for (int l = 0; l < H->L; ++l) {
      Level& V = Mb.lev[l];
      V.NX = nx; V.NY = ny; V.P = (nx + 7) / 8 * 8;
      V.dx = (doms[m].x1 - doms[m].x0) / nx;
      V.dy = (doms[m].y1 - doms[m].y0) / ny;
      const size_t plane = (size_t)V.NY * V.P;
      V.q[0] = (double*)dev_alloc(H, plane * F * 8);
      V.q[1] = (double*)dev_alloc(H, plane * F * 8);
      V.qs = (double*)dev_alloc(H, plane * F * 8);
      V.B = (double*)dev_alloc(H, plane * 8);
      if (!V.q[0] || !V.q[1] || !V.qs || !V.B) { mlswe_destroy(H); return MLSWE_ENOMEM; }
      cudaMemsetAsync(V.q[0], 0, plane * F * 8, H->st);
      cudaMemsetAsync(V.q[1], 0, plane * F * 8, H->st);
      cudaMemsetAsync(V.qs, 0, plane * F * 8, H->st);
      cudaMemsetAsync(V.B, 0, plane * 8, H->st);
      if (cfg->unsplit) {
        V.uxp = (long long)(V.NY + 2) * (V.NX + 1);
        V.uyp = (long long)(V.NY + 1) * (V.NX + 2);
        const size_t ub = (size_t)6 * F * (V.uxp + V.uyp) * 8;
        V.ue = (double*)dev_alloc(H, ub);
        if (!V.ue) { mlswe_destroy(H); return MLSWE_ENOMEM; }
        cudaMemsetAsync(V.ue, 0, ub, H->st);
      }
      if (l == 0) V.patches.push_back(Box{0, 0, nx, ny});
      if (H->L > 1) {
        const int M = cfg->M;
        const size_t ex = (size_t)M * V.NY * (V.NX + 1) * 8, ey = (size_t)M * (V.NY + 1) * V.NX * 8;
        if (l > 0) {
          V.in_patch = (uint8_t*)dev_alloc(H, (size_t)V.NX * V.NY);
          V.fxf = (double*)dev_alloc(H, ex);
          V.fyf = (double*)dev_alloc(H, ey);
          if (!V.in_patch || !V.fxf || !V.fyf) { mlswe_destroy(H); return MLSWE_ENOMEM; }
          cudaMemsetAsync(V.in_patch, 0, (size_t)V.NX * V.NY, H->st);
          cudaMemsetAsync(V.fxf, 0, ex, H->st);
          cudaMemsetAsync(V.fyf, 0, ey, H->st);
        }
        if (l + 1 < H->L) {
          V.covered = (uint8_t*)dev_alloc(H, (size_t)V.NX * V.NY);
          V.fxc = (double*)dev_alloc(H, ex);
          V.fyc = (double*)dev_alloc(H, ey);
          if (!V.covered || !V.fxc || !V.fyc) { mlswe_destroy(H); return MLSWE_ENOMEM; }
          cudaMemsetAsync(V.covered, 0, (size_t)V.NX * V.NY, H->st);
          cudaMemsetAsync(V.fxc, 0, ex, H->st);
          cudaMemsetAsync(V.fyc, 0, ey, H->st);
        }
      }
      if (l + 1 < H->L) { nx *= cfg->ratio[l]; ny *= cfg->ratio[l]; }
    }
  }
  const int nd = n_members * H->L;
  H->d_desc = (LevelDesc*)dev_alloc(H, nd * sizeof(LevelDesc));
  H->d_dt = (double*)dev_alloc(H, nd * sizeof(double));
  H->d_smax = (unsigned long long*)dev_alloc(H, nd * 2 * 8);
  H->d_init = (unsigned long long*)dev_alloc(H, nd * 8);
  H->d_lost = (unsigned int*)dev_alloc(H, 8);
  H->d_status = (unsigned int*)dev_alloc(H, 8);
  H->d_t = (double*)dev_alloc(H, n_members * 8);
  H->d_cfl = (double*)dev_alloc(H, n_members * 8);
  H->d_has = (int*)dev_alloc(H, nd * 4);
  H->d_invdx = (double*)dev_alloc(H, nd * 8);
  H->d_invdy = (double*)dev_alloc(H, nd * 8);
  H->d_par = (int*)dev_alloc(H, nd * 4);
  H->d_init_flag = (int*)dev_alloc(H, 8);
  H->d_cfl_count = (unsigned long long*)dev_alloc(H, 8);
  H->d_rt = (int*)dev_alloc(H, nd * 4);
  H->d_fresh = (int*)dev_alloc(H, 8);
  H->d_active = (int*)dev_alloc(H, nd * 4);
  H->d_cells = (long long*)dev_alloc(H, nd * 8);
  H->d_steps_acc = (long long*)dev_alloc(H, nd * 8);
  H->d_cells_acc = (long long*)dev_alloc(H, nd * 8);
  H->d_redo = (int*)dev_alloc(H, n_members * 4);
  H->d_done = (long long*)dev_alloc(H, n_members * 8);
  if (!H->d_redo || !H->d_done) {
    mlswe_destroy(H);
    return MLSWE_ENOMEM;
  }
  if (!H->d_desc || !H->d_dt || !H->d_smax || !H->d_init || !H->d_lost || !H->d_status || !H->d_t || !H->d_cfl ||
      !H->d_has || !H->d_invdx || !H->d_invdy || !H->d_par || !H->d_init_flag || !H->d_cfl_count || !H->d_rt ||
      !H->d_active || !H->d_cells || !H->d_steps_acc || !H->d_cells_acc || !H->d_fresh) {
    mlswe_destroy(H);
    return MLSWE_ENOMEM;
  }
  H->h_dt.assign(nd, 0.0);
  cudaMemsetAsync(H->d_dt, 0, nd * 8, H->st);
  cudaMemsetAsync(H->d_smax, 0, nd * 16, H->st);
  cudaMemsetAsync(H->d_init, 0, nd * 8, H->st);
  cudaMemsetAsync(H->d_lost, 0, 8, H->st);
  cudaMemsetAsync(H->d_status, 0, 8, H->st);
  cudaMemsetAsync(H->d_t, 0, n_members * 8, H->st);
  cudaMemsetAsync(H->d_cfl, 0, n_members * 8, H->st);
  cudaMemsetAsync(H->d_has, 0, nd * 4, H->st);
  cudaMemsetAsync(H->d_init_flag, 0, 8, H->st);
  cudaMemsetAsync(H->d_cfl_count, 0, 8, H->st);
  {
    // time ratios (the fixed ones until a coarse step chooses), every level active
    std::vector<int> rt(nd), act(nd, 1);
    for (int m = 0; m < n_members; ++m)
      for (int l = 0; l < H->L; ++l) rt[m * H->L + l] = l == 0 ? 1 : cfg->ratio[l - 1];
    cudaMemcpyAsync(H->d_rt, rt.data(), nd * 4, cudaMemcpyHostToDevice, H->st);
    cudaMemcpyAsync(H->d_active, act.data(), nd * 4, cudaMemcpyHostToDevice, H->st);
    cudaMemsetAsync(H->d_cells, 0, nd * 8, H->st);
    cudaMemsetAsync(H->d_fresh, 0, 8, H->st);
    cudaMemsetAsync(H->d_steps_acc, 0, nd * 8, H->st);
    cudaMemsetAsync(H->d_cells_acc, 0, nd * 8, H->st);
    cudaMemsetAsync(H->d_redo, 0, n_members * 4, H->st);
    cudaMemsetAsync(H->d_done, 0, n_members * 8, H->st);
    cudaStreamSynchronize(H->st);
  }
  H->level_steps.assign(H->L, 0);
  H->cell_updates.assign(H->L, 0);
  if (upload_desc(H) != MLSWE_OK) { mlswe_destroy(H); return MLSWE_ECUDA; }
  H->blocks_per_sm = 1;
  *out = H;
  return MLSWE_OK;
}

mlswe_status mlswe_destroy(mlswe_h h) {
  if (!h) return MLSWE_EINVAL;
  cudaStreamSynchronize(h->st);
  invalidate_graphs(h);
  for (cudaEvent_t e : h->timer.pool) cudaEventDestroy(e);
  if (h->copy_st) {
    cudaStreamSynchronize(h->copy_st);
    cudaStreamDestroy(h->copy_st);
    for (int s = 0; s < 2; ++s) {
      if (h->ev_copied[s]) cudaEventDestroy(h->ev_copied[s]);
      if (h->ev_used[s]) cudaEventDestroy(h->ev_used[s]);
    }
  }
  std::vector<void*> all = h->allocations;
  for (void* p : all) dev_free(h, p);
  if (h->own_stream) cudaStreamDestroy(h->st);
  adjoint_release(h);
  delete h;
  return MLSWE_OK;
}

mlswe_status mlswe_level_shape(mlswe_h h, int member, int level, int* nx, int* ny) {
  if (!valid_member_level(h, member, level) || !nx || !ny) return fail(h, MLSWE_EINVAL, "level_shape: bad argument");
  *nx = h->mem[member].lev[level].NX;
  *ny = h->mem[member].lev[level].NY;
  return MLSWE_OK;
}

mlswe_status mlswe_set_state(mlswe_h h, int member, int level, const double* q) {
  if (!valid_member_level(h, member, level) || !q) return fail(h, MLSWE_EINVAL, "set_state: bad argument");
  Level& V = h->mem[member].lev[level];
  const int F = 3 * h->cfg.M;
  double* dst = V.q[h->parity[level]];
  if (V.P == V.NX)  // unpadded rows: one contiguous copy
    CUDA_TRY(h, cudaMemcpyAsync(dst, q, (size_t)F * V.NY * V.NX * 8, cudaMemcpyHostToDevice, h->st));
  else
    CUDA_TRY(h, cudaMemcpy2DAsync(dst, V.P * 8, q, V.NX * 8, V.NX * 8, (size_t)V.NY * F, cudaMemcpyHostToDevice,
                                  h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  h->dt_ready = false;  // the next automatic step starts from this state's wave speeds
  return MLSWE_OK;
}

mlswe_status mlswe_set_state_async(mlswe_h h, int member, int level, const double* q) {
  if (!valid_member_level(h, member, level) || !q) return fail(h, MLSWE_EINVAL, "set_state_async: bad argument");
  Level& V = h->mem[member].lev[level];
  const int F = 3 * h->cfg.M;
  const size_t plane = (size_t)V.NY * V.NX, bytes = plane * F * 8;
  if (!h->copy_st) {
    CUDA_TRY(h, cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking));
    for (int s = 0; s < 2; ++s) {
      CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_copied[s], cudaEventDisableTiming));
      CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_used[s], cudaEventDisableTiming));
    }
  }
  if (bytes > h->stage_bytes) {
    CUDA_TRY(h, cudaStreamSynchronize(h->copy_st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    for (int s = 0; s < 2; ++s) {
      if (h->stage[s]) dev_free(h, h->stage[s]);
      h->stage[s] = (double*)dev_alloc(h, bytes);
      if (!h->stage[s]) { h->stage_bytes = 0; return fail(h, MLSWE_ENOMEM, "staging allocation failed"); }
    }
    h->stage_bytes = bytes;
  }
  const int s = h->stage_next;
  h->stage_next ^= 1;
  // the state copy that last read this staging buffer is done (no-op before its first use)
  CUDA_TRY(h, cudaStreamWaitEvent(h->copy_st, h->ev_used[s], 0));
  CUDA_TRY(h, cudaMemcpyAsync(h->stage[s], q, bytes, cudaMemcpyHostToDevice, h->copy_st));
  CUDA_TRY(h, cudaEventRecord(h->ev_copied[s], h->copy_st));
  CUDA_TRY(h, cudaStreamWaitEvent(h->st, h->ev_copied[s], 0));
  double* dst = V.q[h->parity[level]];
  if (V.P == V.NX)  // unpadded rows: one contiguous copy
    CUDA_TRY(h, cudaMemcpyAsync(dst, h->stage[s], bytes, cudaMemcpyDeviceToDevice, h->st));
  else
    CUDA_TRY(h, cudaMemcpy2DAsync(dst, V.P * 8, h->stage[s], V.NX * 8, V.NX * 8, (size_t)V.NY * F,
                                  cudaMemcpyDeviceToDevice, h->st));
  CUDA_TRY(h, cudaEventRecord(h->ev_used[s], h->st));
  h->dt_ready = false;
  return MLSWE_OK;
}

mlswe_status mlswe_synchronize(mlswe_h h) {
  if (!h) return MLSWE_EINVAL;
  if (h->copy_st) CUDA_TRY(h, cudaStreamSynchronize(h->copy_st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return MLSWE_OK;
}

mlswe_status mlswe_get_state(mlswe_h h, int member, int level, double* q_out) {
  if (!valid_member_level(h, member, level) || !q_out) return fail(h, MLSWE_EINVAL, "get_state: bad argument");
  Level& V = h->mem[member].lev[level];
  const int F = 3 * h->cfg.M;
  const double* src = V.q[h->parity[level]];
  if (V.P == V.NX)
    CUDA_TRY(h, cudaMemcpyAsync(q_out, src, (size_t)F * V.NY * V.NX * 8, cudaMemcpyDeviceToHost, h->st));
  else
    CUDA_TRY(h, cudaMemcpy2DAsync(q_out, V.NX * 8, src, V.P * 8, V.NX * 8, (size_t)V.NY * F, cudaMemcpyDeviceToHost,
                                  h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return MLSWE_OK;
}

// Rows [j0, j0 + n) of every field of the current state, device to device (no host copy,
// no synchronisation: ordered on the hierarchy's stream).
static mlswe_status rows_device(mlswe_h h, int member, int level, int j0, int n, double* other, bool to_other,
                                const char* what) {
  if (!valid_member_level(h, member, level) || !other || n < 0)
    return fail(h, MLSWE_EINVAL, std::string(what) + ": bad argument");
  Level& V = h->mem[member].lev[level];
  if (j0 < 0 || j0 + n > V.NY) return fail(h, MLSWE_EINVAL, std::string(what) + ": rows outside the level");
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, other) != cudaSuccess ||
      (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return fail(h, MLSWE_EINVAL, std::string(what) + ": the buffer must be device memory");
  }
  const int F = 3 * h->cfg.M;
  double* q = V.q[h->parity[level]];
  const size_t plane = (size_t)V.NY * V.P;
  for (int f = 0; f < F; ++f) {
    double* lvl = q + f * plane + (size_t)j0 * V.P;
    double* buf = other + (size_t)f * n * V.NX;
    if (to_other)
      CUDA_TRY(h, cudaMemcpy2DAsync(buf, V.NX * 8, lvl, V.P * 8, V.NX * 8, n, cudaMemcpyDeviceToDevice, h->st));
    else
      CUDA_TRY(h, cudaMemcpy2DAsync(lvl, V.P * 8, buf, V.NX * 8, V.NX * 8, n, cudaMemcpyDeviceToDevice, h->st));
  }
  return MLSWE_OK;
}

mlswe_status mlswe_get_rows_device(mlswe_h h, int member, int level, int j0, int n, double* dst) {
  return rows_device(h, member, level, j0, n, dst, true, "get_rows_device");
}

mlswe_status mlswe_set_rows_device(mlswe_h h, int member, int level, int j0, int n, const double* src) {
  mlswe_status s = rows_device(h, member, level, j0, n, const_cast<double*>(src), false, "set_rows_device");
  if (s == MLSWE_OK) h->dt_ready = false;
  return s;
}

mlswe_status mlswe_set_dt(mlswe_h h, int level, const double* dt) {
  if (!h || level < 0 || level >= h->L || !dt) return fail(h, MLSWE_EINVAL, "set_dt: bad argument");
  for (int m = 0; m < h->n_members; ++m) {
    if (!(dt[m] >= 0.0)) return fail(h, MLSWE_EINVAL, "set_dt: negative or non-finite dt");
    h->h_dt[h->desc_index(m, level)] = dt[m];
  }
  CUDA_TRY(h, cudaMemcpyAsync(h->d_dt, h->h_dt.data(), h->h_dt.size() * 8, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  h->dt_ready = false;
  return MLSWE_OK;
}

mlswe_status mlswe_step_level(mlswe_h h, int level, const double* dt, double* cfl_out) {
  if (!h || level < 0 || level >= h->L) return fail(h, MLSWE_EINVAL, "step_level: bad argument");
  NvtxRange range("mlswe_step_level");
  h->level_steps[level] += 1;
  h->cell_updates[level] += patch_cells(h, level);
  if (dt) {
    mlswe_status s = mlswe_set_dt(h, level, dt);
    if (s != MLSWE_OK) return s;
  }
  CUDA_TRY(h, cudaMemsetAsync(h->d_smax, 0, (size_t)h->n_members * h->L * 16, h->st));
  mlswe_status s = enqueue_level_step(h, level, 1);
  if (s != MLSWE_OK) return s;
  h->dt_ready = false;
  if (cfl_out) {
    bool nan_seen = false;
    s = level_cfl(h, level, cfl_out, &nan_seen);
    if (s != MLSWE_OK) return s;
    if (nan_seen) return fail(h, MLSWE_ENEGDEPTH, "non-finite wave speed in step");
    for (int m = 0; m < h->n_members; ++m)
      if (cfl_out[m] > h->cfg.cfl_max) {
        // Undo the level step for every member (they share its launches): the buffer that
        // held the state before the step becomes current again.
        h->parity[level] ^= 1;
        h->level_steps[level] -= 1;
        h->cell_updates[level] -= patch_cells(h, level);
        return fail(h, MLSWE_ECFL, "Courant number above cfl_max: the level step was undone");
      }
  }
  return MLSWE_OK;
}

mlswe_status mlswe_set_tiles(mlswe_h h, int dir, int len, int lines, int ctas_per_sm) {
  if (!h || dir < 0 || dir > 1 || !shape_ok(len, lines) || ctas_per_sm < 1 || ctas_per_sm > 2)
    return fail(h, MLSWE_EINVAL, "set_tiles: shape out of range");
  for (int l = 0; l < h->L; ++l) set_level_shape(h, l, dir, len, lines, ctas_per_sm);
  invalidate_graphs(h);
  return MLSWE_OK;
}

mlswe_status mlswe_get_stats(mlswe_h h, mlswe_stats* out) {
  if (!h || !out) return fail(h, MLSWE_EINVAL, "get_stats: bad argument");
  std::memset(out, 0, sizeof(*out));
  unsigned long long exceeded = 0;
  std::vector<double> cfl(h->n_members);
  CUDA_TRY(h, cudaMemcpyAsync(&exceeded, h->d_cfl_count, 8, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(cfl.data(), h->d_cfl, cfl.size() * 8, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  const int nd = h->n_members * h->L;
  std::vector<long long> dsteps(nd), dcells(nd);
  CUDA_TRY(h, cudaMemcpyAsync(dsteps.data(), h->d_steps_acc, nd * 8, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(dcells.data(), h->d_cells_acc, nd * 8, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  out->coarse_steps = h->coarse_steps;
  out->regrids = h->regrids;
  for (int l = 0; l < h->L && l < 4; ++l) {
    // steps of mlswe_step_level (host) plus those of mlswe_advance (device: the largest over
    // the members, whose time ratios may differ), cell updates summed over the members
    long long most = 0, cells = 0;
    for (int m = 0; m < h->n_members; ++m) {
      most = std::max(most, dsteps[m * h->L + l]);
      cells += dcells[m * h->L + l];
    }
    out->level_steps[l] = h->level_steps[l] + most;
    out->cell_updates[l] = h->cell_updates[l] + cells;
    int np = 0;
    for (int m = 0; m < h->n_members; ++m) np += (int)h->mem[m].lev[l].patches.size();
    out->patches[l] = np;
  }
  out->cfl_exceeded = (long long)exceeded;
  double mx = 0.0;
  for (double c : cfl) mx = std::max(mx, c);
  out->last_cfl = mx;
  return MLSWE_OK;
}

mlswe_status mlswe_hyperbolicity_losses(mlswe_h h, long long* count, int reset) {
  if (!h || !count) return fail(h, MLSWE_EINVAL, "hyperbolicity_losses: bad argument");
  unsigned int c = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&c, h->d_lost, 4, cudaMemcpyDeviceToHost, h->st));
  if (reset) CUDA_TRY(h, cudaMemsetAsync(h->d_lost, 0, 4, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  *count = (long long)c;
  return MLSWE_OK;
}

mlswe_status mlswe_timing(mlswe_h h, int enable, int n, double* ms_out, long long* launches_out,
                          long long* total_launches) {
  if (!h) return MLSWE_EINVAL;
  timer_collect(h);
  if (ms_out) for (int k = 0; k < n && k < KC_COUNT; ++k) ms_out[k] = h->timer.ms[k];
  if (launches_out) for (int k = 0; k < n && k < KC_COUNT; ++k) launches_out[k] = h->timer.launches[k];
  if (total_launches) *total_launches = h->kernel_launches;
  for (int k = 0; k < KC_COUNT; ++k) { h->timer.ms[k] = 0.0; h->timer.launches[k] = 0; }
  h->kernel_launches = 0;
  h->timer.on = enable != 0;
  return MLSWE_OK;
}

static mlswe_status read_gauges_impl(mlswe_h h, int member, int n, const double* xy, double* eta_out, bool wait) {
  if (!valid_member_level(h, member, 0) || n < 0 || (n > 0 && (!xy || !eta_out)))
    return fail(h, MLSWE_EINVAL, "read_gauges: bad argument");
  if (n == 0) return MLSWE_OK;
  const Member& Mb = h->mem[member];
  const int M = h->cfg.M;
  // Host: finest level whose patch holds each point, and its cell.
  std::vector<int> cells(3 * n), par(h->n_members * h->L);
  for (int k = 0; k < (int)par.size(); ++k) par[k] = h->parity[k % h->L];
  for (int k = 0; k < n; ++k) {
    const double x = xy[2 * k], y = xy[2 * k + 1];
    if (!(x >= Mb.dom.x0 && x <= Mb.dom.x1 && y >= Mb.dom.y0 && y <= Mb.dom.y1))
      return fail(h, MLSWE_EINVAL, "read_gauges: point outside the domain");
    int best = 0, bi = 0, bj = 0;
    for (int l = 0; l < h->L; ++l) {
      const Level& V = Mb.lev[l];
      const int i = std::min(V.NX - 1, (int)std::floor((x - Mb.dom.x0) / V.dx));
      const int j = std::min(V.NY - 1, (int)std::floor((y - Mb.dom.y0) / V.dy));
      bool inside = false;
      for (const Box& b : V.patches)
        if (i >= b.i0 && i < b.i1 && j >= b.j0 && j < b.j1) { inside = true; break; }
      if (inside) { best = l; bi = i; bj = j; }
    }
    cells[3 * k] = h->desc_index(member, best);
    cells[3 * k + 1] = bi;
    cells[3 * k + 2] = bj;
  }
  const size_t need = cells.size() * 4 + par.size() * 4 + (size_t)n * M * 8 + 64;
  // (the scratch is only reused by work later on the same stream: no wait needed)
  char* base = (char*)scratch_buffer(h, need);
  if (!base) return fail(h, MLSWE_ENOMEM, "gauge scratch allocation failed");
  double* d_out = (double*)base;
  int* d_cells = (int*)(base + (size_t)n * M * 8);
  int* d_par = d_cells + cells.size();
  CUDA_TRY(h, cudaMemcpyAsync(d_cells, cells.data(), cells.size() * 4, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(d_par, par.data(), par.size() * 4, cudaMemcpyHostToDevice, h->st));
  int tok;
  timer_begin(h, KC_OTHER, &tok);
  CUDA_TRY(h, launch_gauges(M, h->d_desc, d_par, d_cells, n, d_out, h->st));
  timer_end(h, tok);
  CUDA_TRY(h, cudaMemcpyAsync(eta_out, d_out, (size_t)n * M * 8, cudaMemcpyDeviceToHost, h->st));
  if (wait) CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return MLSWE_OK;
}

mlswe_status mlswe_read_gauges(mlswe_h h, int member, int n, const double* xy, double* eta_out) {
  return read_gauges_impl(h, member, n, xy, eta_out, true);
}

mlswe_status mlswe_read_gauges_async(mlswe_h h, int member, int n, const double* xy, double* eta_out) {
  return read_gauges_impl(h, member, n, xy, eta_out, false);
}

mlswe_status mlswe_set_bathymetry(mlswe_h h, int member, const double* B_finest) {
  if (!valid_member_level(h, member, 0) || !B_finest) return fail(h, MLSWE_EINVAL, "set_bathymetry: bad argument");
  Member& Mb = h->mem[member];
  Level& Fv = Mb.lev[h->L - 1];
  CUDA_TRY(h, cudaMemcpy2DAsync(Fv.B, Fv.P * 8, B_finest, Fv.NX * 8, Fv.NX * 8, Fv.NY, cudaMemcpyHostToDevice, h->st));
  for (int l = h->L - 2; l >= 0; --l) {
    Level& C = Mb.lev[l];
    Level& Fn = Mb.lev[l + 1];
    int tok;
    timer_begin(h, KC_AVERAGE, &tok);
    CUDA_TRY(h, launch_average(1, h->cfg.ratio[l], Fn.B, Fn.P, (size_t)Fn.NY * Fn.P, C.B, C.P, (size_t)C.NY * C.P, 0, 0,
                               C.NX, C.NY, nullptr, 0, h->st));
    timer_end(h, tok);
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return MLSWE_OK;
}

mlswe_status mlswe_get_bathymetry(mlswe_h h, int member, int level, double* B_out) {
  if (!valid_member_level(h, member, level) || !B_out) return fail(h, MLSWE_EINVAL, "get_bathymetry: bad argument");
  Level& V = h->mem[member].lev[level];
  CUDA_TRY(h, cudaMemcpy2DAsync(B_out, V.NX * 8, V.B, V.P * 8, V.NX * 8, V.NY, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return MLSWE_OK;
}

}  // extern "C"
