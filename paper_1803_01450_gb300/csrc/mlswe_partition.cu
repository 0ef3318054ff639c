// Patch partition across ranks: the owner of every patch of the refined levels (a
// space-filling-curve split with balanced cells), the packed exchange buffers of a level
// (state of the owned patch cells and the mass fluxes the reflux reads) and their pack and
// unpack kernels, and the exchange hook that mlswe_advance calls after each refined level
// step. No collective is called here: the caller's hook moves the buffers (for example an
// NCCL all-gather through torch.distributed).
#include <algorithm>
#include <cstring>
#include <numeric>
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

static bool partitioned(const Hier* H) { return H->part_size > 1; }

// Morton (Z-order) key of a cell index pair: bit b of i at bit 2b, bit b of j at bit 2b + 1,
// for the low 21 bits of each.
static unsigned long long morton(int i, int j) {
  unsigned long long key = 0;
  for (int b = 0; b < 21; ++b) {
    key |= (unsigned long long)((i >> b) & 1) << (2 * b);
    key |= (unsigned long long)((j >> b) & 1) << (2 * b + 1);
  }
  return key;
}

// Doubles of one box in a packed buffer with the given parts (layout in
// mlswe_partition_sizes' description; the interface fluxes only on levels with a finer level).
static long long pack_doubles(int M, const Box& b, int parts, bool fine_level_below) {
  const long long w = b.w(), h = b.h();
  long long n = 0;
  if (parts & kPackState) n += 3LL * M * w * h;
  if (parts & kPackAccum) n += 2LL * M * h + 2LL * M * w;
  if ((parts & kPackIface) && fine_level_below) n += (long long)M * h * (w + 1) + (long long)M * (h + 1) * w;
  return n;
}

bool coarsens_patch(const Hier* H, int member, int level, int p) {
  if (!partitioned(H) || level != H->L - 1 || level == 0) return true;
  return H->owner[member][level][p] == H->part_rank;
}

bool patch_owned(const Hier* H, int member, int level, int p) {
  if (!partitioned(H) || level == 0) return true;
  return H->owner[member][level][p] == H->part_rank;
}

static mlswe_status upload_items(Hier* H, DevTable<PackItem>& T, const std::vector<PackItem>& v) {
  if ((int)v.size() > T.cap || !T.d) {
    if (T.d) dev_free(H, T.d);
    T.cap = std::max<int>(64, (int)v.size() * 3 / 2);
    T.d = (PackItem*)dev_alloc(H, T.cap * sizeof(PackItem));
    if (!T.d) return fail(H, MLSWE_ENOMEM, "partition table allocation failed");
  }
  T.count = (int)v.size();
  if (!v.empty())
    CUDA_TRY(H, cudaMemcpyAsync(T.d, v.data(), v.size() * sizeof(PackItem), cudaMemcpyHostToDevice, H->st));
  return MLSWE_OK;
}

// For every patch, the indices of the other patches whose box grown by g cells meets it
// (in increasing order), found through buckets of 64 x 64 cells.
std::vector<std::vector<int>> patches_near(const std::vector<Box>& P, int g) {
  constexpr int kBucket = 64;
  std::vector<std::vector<int>> out(P.size());
  if (P.empty()) return out;
  int ni = 1, nj = 1;
  for (const Box& b : P) {
    ni = std::max(ni, (b.i1 + g + kBucket - 1) / kBucket);
    nj = std::max(nj, (b.j1 + g + kBucket - 1) / kBucket);
  }
  std::vector<std::vector<int>> bucket((size_t)ni * nj);
  for (int k = 0; k < (int)P.size(); ++k) {
    const Box& b = P[k];
    for (int bj = std::max(0, b.j0 - g) / kBucket; bj <= (b.j1 + g - 1) / kBucket; ++bj)
      for (int bi = std::max(0, b.i0 - g) / kBucket; bi <= (b.i1 + g - 1) / kBucket; ++bi)
        bucket[(size_t)bj * ni + bi].push_back(k);
  }
  std::vector<char> seen(P.size(), 0);
  for (int p = 0; p < (int)P.size(); ++p) {
    const Box& a = P[p];
    std::vector<int>& v = out[p];
    for (int bj = a.j0 / kBucket; bj <= std::min(nj - 1, (a.j1 - 1) / kBucket); ++bj)
      for (int bi = a.i0 / kBucket; bi <= std::min(ni - 1, (a.i1 - 1) / kBucket); ++bi)
        for (int q : bucket[(size_t)bj * ni + bi]) {
          if (q == p || seen[q]) continue;
          const Box& b = P[q];
          if (b.i0 - g < a.i1 && a.i0 < b.i1 + g && b.j0 - g < a.j1 && a.j0 < b.j1 + g) {
            seen[q] = 1;
            v.push_back(q);
          }
        }
    for (int q : v) seen[q] = 0;
    std::sort(v.begin(), v.end());
  }
  return out;
}

mlswe_status ensure_partition(Hier* H) {
  if (!H->part_dirty) return MLSWE_OK;
  CUDA_TRY(H, cudaStreamSynchronize(H->st));  // no pack or unpack still reads the old table
  const int n = std::max(1, H->part_size);
  H->owner.assign(H->n_members, std::vector<std::vector<int>>(H->L));
  H->part.resize(H->L);
  struct Entry { int m, p; unsigned long long key; long long cells; };
  for (int l = 0; l < H->L; ++l) {
    std::vector<Entry> e;
    long long total = 0;
    for (int m = 0; m < H->n_members; ++m) {
      const std::vector<Box>& P = H->mem[m].lev[l].patches;
      H->owner[m][l].assign(P.size(), 0);
      for (int p = 0; p < (int)P.size(); ++p) {
        const Box& b = P[p];
        const long long c = (long long)b.w() * b.h();
        e.push_back(Entry{m, p, morton((b.i0 + b.i1) / 2, (b.j0 + b.j1) / 2), c});
        total += c;
      }
    }
    std::stable_sort(e.begin(), e.end(), [](const Entry& a, const Entry& b) {
      if (a.m != b.m) return a.m < b.m;
      if (a.key != b.key) return a.key < b.key;
      return a.p < b.p;
    });
    // owner: the rank whose share of the cells holds the patch's middle cell
    long long before = 0;
    for (const Entry& x : e) {
      int r = 0;
      if (l > 0 && total > 0) r = (int)std::min<long long>(n - 1, (2 * before + x.cells) * n / (2 * total));
      before += x.cells;
      H->owner[x.m][l][x.p] = r;
    }
  }
  // exchange tables per level and kind, each grouped by the rank that packs it
  const int M = H->cfg.M, fin = H->L - 1;
  for (int l = 0; l < H->L; ++l) {
    std::vector<std::vector<PackItem>> per[4];
    long long* sz[4];
    for (int k = 0; k < 4; ++k) {
      per[k].assign(n, {});
      H->part[l].kind[k].size.assign(n, 0);
      sz[k] = H->part[l].kind[k].size.data();
    }
    auto add = [&](int k, int r, int desc, const Box& b, int parts, bool below) {
      per[k][r].push_back(PackItem{desc, b.i0, b.j0, b.i1, b.j1, parts, sz[k][r]});
      sz[k][r] += pack_doubles(M, b, parts, below);
    };
    if (l > 0) {
      std::vector<Entry> order;  // the split's order, for the full buffers
      for (int m = 0; m < H->n_members; ++m)
        for (int p = 0; p < (int)H->mem[m].lev[l].patches.size(); ++p) {
          const Box& b = H->mem[m].lev[l].patches[p];
          order.push_back(Entry{m, p, morton((b.i0 + b.i1) / 2, (b.j0 + b.j1) / 2), 0});
        }
      std::stable_sort(order.begin(), order.end(), [](const Entry& a, const Entry& b) {
        if (a.m != b.m) return a.m < b.m;
        if (a.key != b.key) return a.key < b.key;
        return a.p < b.p;
      });
      const bool below = l + 1 < H->L;
      for (const Entry& x : order) {
        const int r = H->owner[x.m][l][x.p];
        add(MLSWE_XCHG_FULL, r, H->desc_index(x.m, l), H->mem[x.m].lev[l].patches[x.p],
            kPackState | kPackAccum | kPackIface, below);
      }
      // halo boxes: where another rank's patch of the member, grown by two cells, meets an
      // own patch (in the order of the own patches, then of the others); LAST adds every
      // owned patch's accumulators after them
      for (int m = 0; m < H->n_members && n > 1; ++m) {
        const std::vector<Box>& P = H->mem[m].lev[l].patches;
        const std::vector<std::vector<int>> near = patches_near(P, kNG);
        for (int p = 0; p < (int)P.size(); ++p) {
          const int r = H->owner[m][l][p];
          for (int q : near[p]) {
            if (H->owner[m][l][q] == r) continue;
            const Box& Q = P[q];
            const Box c{std::max(P[p].i0, Q.i0 - kNG), std::max(P[p].j0, Q.j0 - kNG), std::min(P[p].i1, Q.i1 + kNG),
                        std::min(P[p].j1, Q.j1 + kNG)};
            if (c.i0 >= c.i1 || c.j0 >= c.j1) continue;
            add(MLSWE_XCHG_HALO, r, H->desc_index(m, l), c, kPackState, below);
            add(MLSWE_XCHG_LAST, r, H->desc_index(m, l), c, kPackState, below);
          }
        }
      }
      for (const Entry& x : order)
        add(MLSWE_XCHG_LAST, H->owner[x.m][l][x.p], H->desc_index(x.m, l), H->mem[x.m].lev[l].patches[x.p],
            kPackAccum, below);
    }
    if (l + 1 == fin) {
      // the parent cells under every finest-level patch, packed by that patch's owner
      const int r_f = H->cfg.ratio[l];
      for (int m = 0; m < H->n_members; ++m) {
        const std::vector<Box>& P = H->mem[m].lev[fin].patches;
        for (int p = 0; p < (int)P.size(); ++p)
          add(MLSWE_XCHG_AVERAGED, H->owner[m][fin][p], H->desc_index(m, l),
              Box{P[p].i0 / r_f, P[p].j0 / r_f, P[p].i1 / r_f, P[p].j1 / r_f}, kPackState, false);
      }
    }
    for (int k = 0; k < 4; ++k) {
      Hier::PartTable& T = H->part[l].kind[k];
      std::vector<PackItem> all;
      T.first.assign(n + 1, 0);
      for (int r = 0; r < n; ++r) {
        T.first[r] = (int)all.size();
        all.insert(all.end(), per[k][r].begin(), per[k][r].end());
      }
      T.first[n] = (int)all.size();
      mlswe_status st = upload_items(H, T.items, all);
      if (st != MLSWE_OK) return st;
    }
  }
  CUDA_TRY(H, cudaStreamSynchronize(H->st));
  H->part_dirty = false;
  return MLSWE_OK;
}

// Copies between the level arrays and a packed buffer, one block per patch: unpack = 1 writes
// the level arrays from buf, 0 writes buf. items [first, last) all belong to one owner.
template <int M>
__global__ void __launch_bounds__(256)
part_copy_kernel(const LevelDesc* __restrict__ descs, const PackItem* __restrict__ items, int first, int last,
                 int par, double* buf, int unpack) {
  for (int k = first + blockIdx.x; k < last; k += gridDim.x) {
    const PackItem it = items[k];
    const LevelDesc& D = descs[it.desc];
    const int w = it.i1 - it.i0, h = it.j1 - it.j0;
    const int NX = D.NX, NY = D.NY;
    double* b = buf + it.off;
    auto mv = [&](double* level_value, long long t) {
      if (unpack) *level_value = b[t];
      else b[t] = *level_value;
    };
    // state of the patch cells, field by field: a warp per row (3M h rows), its lanes along
    // the row (coalesced, no division per value)
    const long long ncell = (long long)w * h;
    const size_t plane = (size_t)NY * D.P;
    const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int nrow = (it.parts & kPackState) ? 3 * M * h : 0;
    for (int row0 = (threadIdx.x >> 5) * 4; row0 < nrow; row0 += nwarp * 4) {
      // four rows per warp at a time: their loads are issued before their stores
      for (int i = lane; i < w; i += 32) {
        double v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int row = row0 + k;
          if (row < nrow) {
            const int f = row / h, j = it.j0 + (row - f * h);
            double* lv = D.q[par] + f * plane + (size_t)j * D.P + it.i0 + i;
            v[k] = unpack ? b[(long long)row * w + i] : *lv;
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int row = row0 + k;
          if (row < nrow) {
            const int f = row / h, j = it.j0 + (row - f * h);
            double* lv = D.q[par] + f * plane + (size_t)j * D.P + it.i0 + i;
            if (unpack) *lv = v[k];
            else b[(long long)row * w + i] = v[k];
          }
        }
      }
    }
    if (it.parts & kPackState) b += 3LL * M * ncell;
    if (it.parts & kPackAccum) {
      // boundary accumulators: x edges at i0 and i1 of every row, y edges at j0 and j1 of
      // every column
      for (int t = threadIdx.x; t < 2 * M * h; t += blockDim.x) {
        const int m = t / (2 * h), rr = t - m * 2 * h, j = it.j0 + (rr >> 1), a = (rr & 1) ? it.i1 : it.i0;
        mv(D.fxf + ((size_t)m * NY + j) * (NX + 1) + a, t);
      }
      b += 2LL * M * h;
      for (int t = threadIdx.x; t < 2 * M * w; t += blockDim.x) {
        const int m = t / (2 * w), rr = t - m * 2 * w, i = it.i0 + (rr >> 1), a = (rr & 1) ? it.j1 : it.j0;
        mv(D.fyf + ((size_t)m * (NY + 1) + a) * NX + i, t);
      }
      b += 2LL * M * w;
    }
    if ((it.parts & kPackIface) && D.fxc != nullptr) {
      // interface fluxes of every edge of the box, sides included
      const int wx = w + 1;
      for (int t = threadIdx.x; t < M * h * wx; t += blockDim.x) {
        const int m = t / (h * wx), rr = t - m * h * wx, j = it.j0 + rr / wx, a = it.i0 + rr % wx;
        mv(D.fxc + ((size_t)m * NY + j) * (NX + 1) + a, t);
      }
      b += (long long)M * h * wx;
      const int hy = h + 1;
      for (int t = threadIdx.x; t < M * hy * w; t += blockDim.x) {
        const int m = t / (hy * w), rr = t - m * hy * w, a = it.j0 + rr / w, i = it.i0 + rr % w;
        mv(D.fyc + ((size_t)m * (NY + 1) + a) * NX + i, t);
      }
    }
  }
}

static cudaError_t launch_part_copy(int M, const LevelDesc* descs, const PackItem* items, int first, int last,
                                    int par, double* buf, int unpack, int grid, cudaStream_t st) {
  if (last <= first) return cudaSuccess;
  const int g = std::min(grid, last - first);
  if (M == 1) part_copy_kernel<1><<<g, 256, 0, st>>>(descs, items, first, last, par, buf, unpack);
  else if (M == 3) part_copy_kernel<3><<<g, 256, 0, st>>>(descs, items, first, last, par, buf, unpack);
  else if (M == 4) part_copy_kernel<4><<<g, 256, 0, st>>>(descs, items, first, last, par, buf, unpack);
  else part_copy_kernel<2><<<g, 256, 0, st>>>(descs, items, first, last, par, buf, unpack);
  return cudaGetLastError();
}

mlswe_status run_exchange_hook(Hier* H, int level, int kind) {
  if (!partitioned(H) || !H->part_hook) return MLSWE_OK;
  if (kind != MLSWE_XCHG_AVERAGED && level == 0) return MLSWE_OK;
  mlswe_status s = ensure_partition(H);
  if (s != MLSWE_OK) return s;
  if (H->part_hook(H->part_ctx, level, kind) != 0) return fail(H, MLSWE_EINVAL, "partition exchange hook failed");
  return MLSWE_OK;
}

// Argument checks shared by the exchange calls; builds the tables when a layout changed.
static mlswe_status part_level_ready(Hier* H, int level, int kind) {
  if (kind < MLSWE_XCHG_FULL || kind > MLSWE_XCHG_AVERAGED) return fail(H, MLSWE_EINVAL, "partition: bad kind");
  if (kind == MLSWE_XCHG_AVERAGED ? (level != H->L - 2) : (level < 1 || level >= H->L))
    return fail(H, MLSWE_EINVAL, "partition: no exchange of this kind on this level");
  return ensure_partition(H);
}

static bool device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace mlswe

using namespace mlswe;

extern "C" {

mlswe_status mlswe_set_partition(mlswe_h h, int rank, int world_size, mlswe_exchange_hook hook, void* ctx) {
  if (!h || world_size < 1 || rank < 0 || rank >= world_size) return fail(h, MLSWE_EINVAL, "partition: bad rank");
  if (world_size > 1 && (h->cfg.unsplit || h->per_patch_launch))
    return fail(h, MLSWE_EINVAL, "partition: split step in the batched form only");
  h->part_rank = world_size > 1 ? rank : 0;
  h->part_size = world_size;
  h->part_hook = world_size > 1 ? hook : nullptr;
  h->part_ctx = ctx;
  h->part_dirty = true;
  h->tables_dirty = true;               // the finest level's coarsening takes this rank's patches
  for (auto& W : h->wl) W.dirty = true;  // the sweeps take this rank's patches
  invalidate_graphs(h);
  return ensure_partition(h);
}

mlswe_status mlswe_partition_owners(mlswe_h h, int member, int level, int* owner_out) {
  if (!h || !owner_out || member < 0 || member >= h->n_members || level < 0 || level >= h->L)
    return fail(h, MLSWE_EINVAL, "partition_owners: bad argument");
  mlswe_status s = ensure_partition(h);
  if (s != MLSWE_OK) return s;
  const std::vector<int>& o = h->owner[member][level];
  std::copy(o.begin(), o.end(), owner_out);
  return MLSWE_OK;
}

mlswe_status mlswe_partition_sizes(mlswe_h h, int level, int kind, long long* doubles_per_rank) {
  if (!h || !doubles_per_rank) return fail(h, MLSWE_EINVAL, "partition_sizes: bad argument");
  mlswe_status s = part_level_ready(h, level, kind);
  if (s != MLSWE_OK) return s;
  const Hier::PartTable& T = h->part[level].kind[kind];
  for (int r = 0; r < h->part_size; ++r) doubles_per_rank[r] = T.size[r];
  return MLSWE_OK;
}

mlswe_status mlswe_partition_pack(mlswe_h h, int level, int kind, double* dst) {
  if (!h || !dst) return fail(h, MLSWE_EINVAL, "partition_pack: bad argument");
  mlswe_status s = part_level_ready(h, level, kind);
  if (s != MLSWE_OK) return s;
  if (!device_pointer(dst)) return fail(h, MLSWE_EINVAL, "partition_pack: dst is not device memory");
  const Hier::PartTable& T = h->part[level].kind[kind];
  const int r = h->part_rank;
  CUDA_TRY(h, launch_part_copy(h->cfg.M, h->d_desc, T.items.d, T.first[r], T.first[r + 1], h->parity[level], dst, 0,
                               8 * h->num_sms, h->st));
  h->kernel_launches += T.first[r + 1] > T.first[r] ? 1 : 0;
  return MLSWE_OK;
}

mlswe_status mlswe_partition_unpack(mlswe_h h, int level, int kind, int from, const double* src) {
  if (!h || !src || from < 0 || from >= h->part_size) return fail(h, MLSWE_EINVAL, "partition_unpack: bad argument");
  mlswe_status s = part_level_ready(h, level, kind);
  if (s != MLSWE_OK) return s;
  if (!device_pointer(src)) return fail(h, MLSWE_EINVAL, "partition_unpack: src is not device memory");
  const Hier::PartTable& T = h->part[level].kind[kind];
  CUDA_TRY(h, launch_part_copy(h->cfg.M, h->d_desc, T.items.d, T.first[from], T.first[from + 1], h->parity[level],
                               const_cast<double*>(src), 1, 8 * h->num_sms, h->st));
  h->kernel_launches += T.first[from + 1] > T.first[from] ? 1 : 0;
  return MLSWE_OK;
}

mlswe_status mlswe_wave_speed_slots(mlswe_h h, double** dev, int* n) {
  if (!h || !dev || !n) return fail(h, MLSWE_EINVAL, "wave_speed_slots: bad argument");
  *dev = reinterpret_cast<double*>(h->d_smax);
  *n = 2 * h->n_members * h->L;
  return MLSWE_OK;
}

}  // extern "C"
