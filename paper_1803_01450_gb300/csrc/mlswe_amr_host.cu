// Host side of the AMR: patch layouts and masks, ghost fill, refinement,
// coarsening, reflux, regridding and the subcycled Berger-Oliger driver.
#include <algorithm>
#include <cmath>
#include <cstring>
#include "mlswe_internal.h"

namespace mlswe {

cudaError_t launch_interp(int M, const DevParams& P, const LevelDesc* descs, const InterpItem* items, int n_items,
                          long long max_cells, int r, int par_c, int par_f, double alpha, int mode, cudaStream_t st);
cudaError_t launch_average_items(int F, const LevelDesc* descs, const InterpItem* items, int n_items, long long max_cells,
                                 int r, int par_c, int par_f, cudaStream_t st);
cudaError_t launch_flags(int M, const LevelDesc* descs, int desc, int par, long long cells, double dry_tol,
                         double inv_dx, double inv_dy, double tol2, uint8_t* flags, cudaStream_t st);
cudaError_t launch_mask_boxes(uint8_t* mask, int NX, const int* boxes, int n, int div, long long max_cells,
                              cudaStream_t st);
cudaError_t launch_reflux(int M, const LevelDesc* descs, const InterpItem* items, int n_items, long long max_cells,
                          int r, int par_c, cudaStream_t st);
cudaError_t launch_speed(int M, const DevParams& P, const LevelDesc* descs, const InterpItem* items, int n_items,
                         long long max_cells, const int* par_of_desc, unsigned long long* out, cudaStream_t st);
std::vector<Box> cluster_flags(const uint8_t* flags, int nx, int ny, int level, const std::vector<Box>& patches,
                               int r, int n_buf, double eff, int min_side, int max_side, int n_nest);
std::vector<Box> box_difference(const Box& a, const std::vector<Box>& sub);
mlswe_status enqueue_level_step(Hier* H, int level);

constexpr int kNest = 2;  // nesting margin in coarse cells

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

// Device staging buffer for small per-launch tables (items, boxes), grown on demand.
static void* staging(Hier* H, size_t bytes) {
  if (bytes > H->stage_bytes) {
    if (H->stage) dev_free(H, H->stage);
    H->stage_bytes = std::max<size_t>(bytes * 2, 1 << 16);
    H->stage = dev_alloc(H, H->stage_bytes);
    if (!H->stage) H->stage_bytes = 0;
  }
  return H->stage;
}

template <class T>
static mlswe_status upload_items(Hier* H, const std::vector<T>& v, T** dptr) {
  *dptr = nullptr;
  if (v.empty()) return MLSWE_OK;
  // Several tables may be in flight on the stream: copy into a fresh region each time
  // is avoided by synchronising before reuse of the staging buffer.
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  void* p = staging(H, v.size() * sizeof(T));
  if (!p) return fail(H, MLSWE_ENOMEM, "staging allocation failed");
  CUDA_TRY(H, cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, H->st));
  *dptr = (T*)p;
  return MLSWE_OK;
}

static long long max_cells_of(const std::vector<InterpItem>& v) {
  long long m = 0;
  for (const auto& it : v) m = std::max<long long>(m, (long long)(it.i1 - it.i0) * (it.j1 - it.j0));
  return m;
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
    int* d = nullptr;
    mlswe_status s = upload_items(H, b, &d);
    if (s != MLSWE_OK) return s;
    long long mc = 0;
    for (const Box& x : V.patches) mc = std::max<long long>(mc, (long long)x.w() * x.h());
    int tok;
    timer_begin(H, KC_OTHER, &tok);
    CUDA_TRY(H, launch_mask_boxes(V.in_patch, V.NX, d, (int)V.patches.size(), 1, mc, H->st));
    timer_end(H, tok);
    timer_begin(H, KC_OTHER, &tok);
    CUDA_TRY(H, launch_mask_boxes(C.covered, C.NX, d, (int)V.patches.size(), H->cfg.ratio[level - 1], mc, H->st));
    timer_end(H, tok);
    CUDA_TRY(H, cudaStreamSynchronize(H->st));
  }
  H->wl[level * 2].dirty = H->wl[level * 2 + 1].dirty = true;
  H->wl[(level - 1) * 2].dirty = H->wl[(level - 1) * 2 + 1].dirty = true;
  return MLSWE_OK;
}

static mlswe_status check_layout(Hier* H, int member, int level, const std::vector<Box>& boxes) {
  const Level& V = H->mem[member].lev[level];
  const Level& C = H->mem[member].lev[level - 1];
  const int r = H->cfg.ratio[level - 1];
  for (size_t a = 0; a < boxes.size(); ++a) {
    const Box& b = boxes[a];
    if (b.i0 < 0 || b.j0 < 0 || b.i1 > V.NX || b.j1 > V.NY || b.i1 <= b.i0 || b.j1 <= b.j0)
      return fail(H, MLSWE_ENESTING, "patch outside the domain or empty");
    if (b.i0 % r || b.j0 % r || b.i1 % r || b.j1 % r)
      return fail(H, MLSWE_ENESTING, "patch not aligned to coarse cells");
    for (size_t c = a + 1; c < boxes.size(); ++c) {
      const Box& o = boxes[c];
      if (std::max(b.i0, o.i0) < std::min(b.i1, o.i1) && std::max(b.j0, o.j0) < std::min(b.j1, o.j1))
        return fail(H, MLSWE_ENESTING, "patches overlap");
    }
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

mlswe_status set_patches_internal(Hier* H, int member, int level, const std::vector<Box>& boxes) {
  mlswe_status s = check_layout(H, member, level, boxes);
  if (s != MLSWE_OK) return s;
  H->mem[member].lev[level].patches = boxes;
  return rebuild_masks(H, member, level);
}

static int parity_c(Hier* H, int level) { return H->parity[level]; }

// Ghost cells of every patch of `level` (all members) at time fraction alpha.
mlswe_status fill_ghosts_internal(Hier* H, int level, double alpha) {
  std::vector<InterpItem> items;
  for (int m = 0; m < H->n_members; ++m) {
    const Level& V = H->mem[m].lev[level];
    for (const Box& b : V.patches) {
      InterpItem it;
      it.desc_c = H->desc_index(m, level - 1);
      it.desc_f = H->desc_index(m, level);
      it.i0 = std::max(0, b.i0 - kNG); it.j0 = std::max(0, b.j0 - kNG);
      it.i1 = std::min(V.NX, b.i1 + kNG); it.j1 = std::min(V.NY, b.j1 + kNG);
      items.push_back(it);
    }
  }
  if (items.empty()) return MLSWE_OK;
  InterpItem* d;
  mlswe_status s = upload_items(H, items, &d);
  if (s != MLSWE_OK) return s;
  int tok;
  timer_begin(H, KC_GHOST, &tok);
  CUDA_TRY(H, launch_interp(H->cfg.M, H->dp, H->d_desc, d, (int)items.size(), max_cells_of(items),
                            H->cfg.ratio[level - 1], parity_c(H, level - 1), H->parity[level], alpha, 1, H->st));
  timer_end(H, tok);
  return MLSWE_OK;
}

// Refinement of the cells in `boxes` (fine indices) of (member, coarse_level + 1) from the
// current coarse state.
static mlswe_status interp_boxes(Hier* H, int member, int coarse_level, const std::vector<Box>& boxes) {
  std::vector<InterpItem> items;
  for (const Box& b : boxes)
    items.push_back(InterpItem{H->desc_index(member, coarse_level), H->desc_index(member, coarse_level + 1), b.i0, b.j0,
                               b.i1, b.j1});
  if (items.empty()) return MLSWE_OK;
  InterpItem* d;
  mlswe_status s = upload_items(H, items, &d);
  if (s != MLSWE_OK) return s;
  int tok;
  timer_begin(H, KC_INTERP, &tok);
  CUDA_TRY(H, launch_interp(H->cfg.M, H->dp, H->d_desc, d, (int)items.size(), max_cells_of(items),
                            H->cfg.ratio[coarse_level], parity_c(H, coarse_level), H->parity[coarse_level + 1], 1.0, 0,
                            H->st));
  timer_end(H, tok);
  return MLSWE_OK;
}

// Coarsening of every member's level `fine_level` onto fine_level - 1 (members: -1 = all).
mlswe_status average_internal(Hier* H, int fine_level, int member) {
  std::vector<InterpItem> items;
  const int r = H->cfg.ratio[fine_level - 1];
  for (int m = 0; m < H->n_members; ++m) {
    if (member >= 0 && m != member) continue;
    for (const Box& b : H->mem[m].lev[fine_level].patches)
      items.push_back(InterpItem{H->desc_index(m, fine_level - 1), H->desc_index(m, fine_level), b.i0 / r, b.j0 / r,
                                 b.i1 / r, b.j1 / r});
  }
  if (items.empty()) return MLSWE_OK;
  InterpItem* d;
  mlswe_status s = upload_items(H, items, &d);
  if (s != MLSWE_OK) return s;
  int tok;
  timer_begin(H, KC_AVERAGE, &tok);
  CUDA_TRY(H, launch_average_items(3 * H->cfg.M, H->d_desc, d, (int)items.size(), max_cells_of(items), r,
                                   H->parity[fine_level - 1], H->parity[fine_level], H->st));
  timer_end(H, tok);
  return MLSWE_OK;
}

static mlswe_status reflux_internal(Hier* H, int level) {
  std::vector<InterpItem> items;
  for (int m = 0; m < H->n_members; ++m) {
    if (H->mem[m].lev[level + 1].patches.empty()) continue;
    for (const Box& b : H->mem[m].lev[level].patches)
      items.push_back(InterpItem{H->desc_index(m, level), H->desc_index(m, level + 1), b.i0, b.j0, b.i1, b.j1});
  }
  if (items.empty()) return MLSWE_OK;
  InterpItem* d;
  mlswe_status s = upload_items(H, items, &d);
  if (s != MLSWE_OK) return s;
  int tok;
  timer_begin(H, KC_REFLUX, &tok);
  CUDA_TRY(H, launch_reflux(H->cfg.M, H->d_desc, d, (int)items.size(), max_cells_of(items), H->cfg.ratio[level],
                            H->parity[level], H->st));
  timer_end(H, tok);
  return MLSWE_OK;
}

static bool level_has_patches(Hier* H, int level) {
  for (int m = 0; m < H->n_members; ++m)
    if (!H->mem[m].lev[level].patches.empty()) return true;
  return false;
}

static mlswe_status advance_level(Hier* H, int level, double alpha) {
  mlswe_status s;
  if (level > 0) {
    s = fill_ghosts_internal(H, level, alpha);
    if (s != MLSWE_OK) return s;
  }
  s = enqueue_level_step(H, level);
  if (s != MLSWE_OK) return s;
  if (level + 1 < H->L && level_has_patches(H, level + 1)) {
    const int rt = H->cfg.ratio[level];
    for (int k = 0; k < rt; ++k) {
      s = advance_level(H, level + 1, (double)k / rt);
      if (s != MLSWE_OK) return s;
    }
    s = average_internal(H, level + 1, -1);
    if (s != MLSWE_OK) return s;
    s = reflux_internal(H, level);
    if (s != MLSWE_OK) return s;
  }
  return MLSWE_OK;
}

// Per-member level-0 step from wave speeds: dt_0 = cfl * min_l (prod_{k<l} r_k) / rate_l.
static void dt_from_rates(Hier* H, const std::vector<double>& rate /*[member*L + l]*/, std::vector<double>& dt0) {
  dt0.assign(H->n_members, 0.0);
  for (int m = 0; m < H->n_members; ++m) {
    double best = INFINITY, fac = 1.0;
    for (int l = 0; l < H->L; ++l) {
      if (l > 0) fac *= H->cfg.ratio[l - 1];
      if (H->mem[m].lev[l].patches.empty()) continue;
      const double rt = rate[H->desc_index(m, l)];
      if (rt > 0.0) best = std::min(best, fac / rt);
    }
    dt0[m] = std::isfinite(best) ? H->cfg.cfl_desired * best : 0.0;
  }
}

static mlswe_status initial_rates(Hier* H, std::vector<double>& rate) {
  std::vector<InterpItem> items;
  for (int m = 0; m < H->n_members; ++m)
    for (int l = 0; l < H->L; ++l)
      for (const Box& b : H->mem[m].lev[l].patches)
        items.push_back(InterpItem{H->desc_index(m, l), 0, b.i0, b.j0, b.i1, b.j1});
  const int nd = H->n_members * H->L;
  std::vector<int> par(nd);
  for (int k = 0; k < nd; ++k) par[k] = H->parity[k % H->L];
  // layout in staging: items | parity | speeds
  const size_t ib = items.size() * sizeof(InterpItem), pb = nd * sizeof(int);
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  char* base = (char*)staging(H, ib + pb + nd * 8 + 64);
  if (!base) return fail(H, MLSWE_ENOMEM, "staging allocation failed");
  InterpItem* d_items = (InterpItem*)base;
  int* d_par = (int*)(base + ib);
  unsigned long long* d_sp = (unsigned long long*)(base + ((ib + pb + 7) / 8) * 8);
  CUDA_TRY(H, cudaMemcpyAsync(d_items, items.data(), ib, cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaMemcpyAsync(d_par, par.data(), pb, cudaMemcpyHostToDevice, H->st));
  CUDA_TRY(H, cudaMemsetAsync(d_sp, 0, nd * 8, H->st));
  int tok;
  timer_begin(H, KC_OTHER, &tok);
  CUDA_TRY(H, launch_speed(H->cfg.M, H->dp, H->d_desc, d_items, (int)items.size(), max_cells_of(items), d_par, d_sp,
                           H->st));
  timer_end(H, tok);
  std::vector<unsigned long long> bits(nd);
  CUDA_TRY(H, cudaMemcpyAsync(bits.data(), d_sp, nd * 8, cudaMemcpyDeviceToHost, H->st));
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  rate.assign(nd, 0.0);
  for (int k = 0; k < nd; ++k) {
    double s;
    std::memcpy(&s, &bits[k], 8);
    const Level& V = H->mem[k / H->L].lev[k % H->L];
    rate[k] = s / std::min(V.dx, V.dy);
  }
  return MLSWE_OK;
}

static mlswe_status step_rates(Hier* H, std::vector<double>& rate, bool* nan_seen) {
  const int nd = H->n_members * H->L;
  std::vector<unsigned long long> bits(nd * 2);
  CUDA_TRY(H, cudaMemcpyAsync(bits.data(), H->d_smax, nd * 16, cudaMemcpyDeviceToHost, H->st));
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  rate.assign(nd, 0.0);
  *nan_seen = false;
  for (int k = 0; k < nd; ++k) {
    double sx, sy;
    std::memcpy(&sx, &bits[2 * k], 8);
    std::memcpy(&sy, &bits[2 * k + 1], 8);
    if (std::isnan(sx) || std::isnan(sy)) *nan_seen = true;
    const Level& V = H->mem[k / H->L].lev[k % H->L];
    rate[k] = std::max(sx / V.dx, sy / V.dy);
  }
  return MLSWE_OK;
}

static mlswe_status set_level_dts(Hier* H, const std::vector<double>& dt0) {
  for (int m = 0; m < H->n_members; ++m) {
    double dt = dt0[m];
    for (int l = 0; l < H->L; ++l) {
      if (l > 0) dt /= H->cfg.ratio[l - 1];
      H->h_dt[H->desc_index(m, l)] = dt;
    }
  }
  CUDA_TRY(H, cudaMemcpyAsync(H->d_dt, H->h_dt.data(), H->h_dt.size() * 8, cudaMemcpyHostToDevice, H->st));
  return MLSWE_OK;
}

mlswe_status regrid_internal(Hier* H, int base) {
  for (int m = 0; m < H->n_members; ++m) {
    for (int l = base; l + 1 < H->L; ++l) {
      Level& V = H->mem[m].lev[l];
      Level& Fl = H->mem[m].lev[l + 1];
      std::vector<Box> boxes;
      if (l == 0 || !V.patches.empty()) {
        const size_t cells = (size_t)V.NX * V.NY;
        CUDA_TRY(H, cudaStreamSynchronize(H->st));
        uint8_t* d_flags = (uint8_t*)staging(H, cells);
        if (!d_flags) return fail(H, MLSWE_ENOMEM, "staging allocation failed");
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
      std::vector<Box> fresh;
      for (const Box& b : boxes) {
        std::vector<Box> d = box_difference(b, old);
        fresh.insert(fresh.end(), d.begin(), d.end());
      }
      s = interp_boxes(H, m, l, fresh);
      if (s != MLSWE_OK) return s;
    }
  }
  return MLSWE_OK;
}

}  // namespace mlswe

using namespace mlswe;

extern "C" {

mlswe_status mlswe_set_patches(mlswe_h h, int member, int level, int n, const int32_t* boxes) {
  Hier* H = h;
  if (!H || member < 0 || member >= H->n_members || level < 1 || level >= H->L || n < 0 || (n > 0 && !boxes))
    return fail(H, MLSWE_EINVAL, "set_patches: bad argument");
  std::vector<Box> b(n);
  for (int k = 0; k < n; ++k) b[k] = Box{boxes[4 * k], boxes[4 * k + 1], boxes[4 * k + 2], boxes[4 * k + 3]};
  return set_patches_internal(H, member, level, b);
}

mlswe_status mlswe_get_patches(mlswe_h h, int member, int level, int* n, int32_t* boxes) {
  Hier* H = h;
  if (!H || member < 0 || member >= H->n_members || level < 0 || level >= H->L || !n)
    return fail(H, MLSWE_EINVAL, "get_patches: bad argument");
  const std::vector<Box>& P = H->mem[member].lev[level].patches;
  const int cap = *n;
  *n = (int)P.size();
  if (boxes) {
    if (cap < (int)P.size()) return fail(H, MLSWE_EINVAL, "get_patches: capacity too small");
    for (size_t k = 0; k < P.size(); ++k) {
      boxes[4 * k] = P[k].i0; boxes[4 * k + 1] = P[k].j0; boxes[4 * k + 2] = P[k].i1; boxes[4 * k + 3] = P[k].j1;
    }
  }
  return MLSWE_OK;
}

mlswe_status mlswe_fill_ghosts(mlswe_h h, int level, double alpha) {
  Hier* H = h;
  if (!H || level < 1 || level >= H->L || !(alpha >= 0.0 && alpha <= 1.0))
    return fail(H, MLSWE_EINVAL, "fill_ghosts: bad argument");
  mlswe_status s = fill_ghosts_internal(H, level, alpha);
  if (s != MLSWE_OK) return s;
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  return MLSWE_OK;
}

mlswe_status mlswe_interp_fine(mlswe_h h, int coarse_level, int member) {
  Hier* H = h;
  if (!H || member < 0 || member >= H->n_members || coarse_level < 0 || coarse_level + 1 >= H->L)
    return fail(H, MLSWE_EINVAL, "interp_fine: bad argument");
  mlswe_status s = interp_boxes(H, member, coarse_level, H->mem[member].lev[coarse_level + 1].patches);
  if (s != MLSWE_OK) return s;
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  return MLSWE_OK;
}

mlswe_status mlswe_average_coarse(mlswe_h h, int fine_level, int member) {
  Hier* H = h;
  if (!H || member < 0 || member >= H->n_members || fine_level < 1 || fine_level >= H->L)
    return fail(H, MLSWE_EINVAL, "average_coarse: bad argument");
  mlswe_status s = average_internal(H, fine_level, member);
  if (s != MLSWE_OK) return s;
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  return MLSWE_OK;
}

mlswe_status mlswe_get_flags(mlswe_h h, int member, int level, uint8_t* flags) {
  Hier* H = h;
  if (!H || member < 0 || member >= H->n_members || level < 0 || level >= H->L || !flags)
    return fail(H, MLSWE_EINVAL, "get_flags: bad argument");
  const Level& V = H->mem[member].lev[level];
  const size_t cells = (size_t)V.NX * V.NY;
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  uint8_t* d = (uint8_t*)staging(H, cells);
  if (!d) return fail(H, MLSWE_ENOMEM, "staging allocation failed");
  int tok;
  timer_begin(H, KC_FLAGS, &tok);
  CUDA_TRY(H, launch_flags(H->cfg.M, H->d_desc, H->desc_index(member, level), H->parity[level], (long long)cells,
                           H->cfg.dry_tol, 1.0 / V.dx, 1.0 / V.dy, H->cfg.flag_tol * H->cfg.flag_tol, d, H->st));
  timer_end(H, tok);
  CUDA_TRY(H, cudaMemcpyAsync(flags, d, cells, cudaMemcpyDeviceToHost, H->st));
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  return MLSWE_OK;
}

mlswe_status mlswe_regrid(mlswe_h h, int base_level) {
  Hier* H = h;
  if (!H || base_level < 0 || base_level >= H->L) return fail(H, MLSWE_EINVAL, "regrid: bad argument");
  mlswe_status s = regrid_internal(H, base_level);
  if (s != MLSWE_OK) return s;
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  return MLSWE_OK;
}

mlswe_status mlswe_advance(mlswe_h h, int n_coarse_steps) {
  Hier* H = h;
  if (!H || n_coarse_steps < 0) return fail(H, MLSWE_EINVAL, "advance: bad argument");
  mlswe_status warn = MLSWE_OK;
  for (int k = 0; k < n_coarse_steps; ++k) {
    mlswe_status s;
    if (H->cfg.regrid_interval > 0 && H->L > 1 && H->coarse_steps % H->cfg.regrid_interval == 0) {
      s = regrid_internal(H, 0);
      if (s != MLSWE_OK) return s;
    }
    std::vector<double> rate, dt0;
    if (!H->have_rates) {
      s = initial_rates(H, rate);
      if (s != MLSWE_OK) return s;
    } else {
      rate = H->last_rates;
    }
    dt_from_rates(H, rate, dt0);
    s = set_level_dts(H, dt0);
    if (s != MLSWE_OK) return s;
    CUDA_TRY(H, cudaMemsetAsync(H->d_smax, 0, (size_t)H->n_members * H->L * 16, H->st));
    s = advance_level(H, 0, 0.0);
    if (s != MLSWE_OK) return s;
    bool nan_seen = false;
    s = step_rates(H, H->last_rates, &nan_seen);
    if (s != MLSWE_OK) return s;
    if (nan_seen) return fail(H, MLSWE_ENEGDEPTH, "non-finite wave speed in step");
    H->have_rates = true;
    for (int m = 0; m < H->n_members; ++m) {
      double dt = dt0[m];
      for (int l = 0; l < H->L; ++l) {
        if (l > 0) dt /= H->cfg.ratio[l - 1];
        if (dt * H->last_rates[H->desc_index(m, l)] > H->cfg.cfl_max) warn = MLSWE_ECFL;
      }
    }
    H->t += dt0[0];
    H->last_dt0 = dt0;
    H->coarse_steps++;
  }
  if (warn != MLSWE_OK) return fail(H, warn, "Courant number above cfl_max in a step");
  return MLSWE_OK;
}

mlswe_status mlswe_get_time(mlswe_h h, double* t_out, double* dt_out) {
  Hier* H = h;
  if (!H) return MLSWE_EINVAL;
  if (t_out) *t_out = H->t;
  if (dt_out)
    for (int m = 0; m < H->n_members; ++m) dt_out[m] = H->last_dt0.empty() ? 0.0 : H->last_dt0[m];
  return MLSWE_OK;
}

}  // extern "C"
