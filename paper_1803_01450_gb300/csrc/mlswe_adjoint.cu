// Discrete adjoint of the fixed-grid, first-order, fixed-dt step on a walled
// single-level grid (wet states only), for gradients of a gauge misfit
//   J = sum_{n=1..N} sum_g (eta_1(cell_g, Q^n) - obs_{n,g})^2,   eta_1 = B + h_2 + h_1 (Eq. (4)),
// with respect to the initial state and the bathymetry. The forward pass keeps a
// checkpoint every `ckpt_every` steps; the backward pass recomputes each segment
// from its checkpoint and applies the transposed step in reverse:
//   lambda_n = (dQ^{n+1}/dQ^n)^T lambda_{n+1} + dJ_n/dQ^n,
//   dJ/dB   += (dQ^{n+1}/dB)^T lambda_{n+1} + dJ_n/dB.
// The transposed split step runs the y sweep's adjoint on the recomputed state
// after the x sweep, then the x sweep's adjoint; each edge's contribution is the
// hand-written vector-Jacobian product of mlswe_adjoint.cuh. Wall ghost cells are
// mirrors of interior cells, so their cotangents fold back into those cells.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstring>
#include "mlswe_adjoint.cuh"
#include "mlswe_internal.h"

namespace mlswe {

template <int DIR>
__device__ __forceinline__ int acslot(int l, int k, int len, int nl) {  // k in [0, len + 2): cells -1 .. len
  return DIR == 0 ? l * (len + 2) + k : k * nl + l;
}
template <int DIR>
__device__ __forceinline__ int aeslot(int l, int e, int len, int nl) {  // e in [0, len + 1): edges -1/2 .. len-1/2
  return DIR == 0 ? l * (len + 1) + e : e * nl + l;
}

// Threads per CTA of the adjoint sweep: two CTAs per SM fit the 255 registers the edge VJP
// takes, so one CTA's load and gather phases overlap the other's FP64 work; tiles have at
// most kAdjThreads edges.
constexpr int kAdjThreads = 128;

// Adjoint of one first-order sweep over the tiles of the level. state: input of the
// forward sweep (pitched like the level); lam_out: cotangent of its output; lam_in:
// cotangent of its input (written); gB: bathymetry cotangent (accumulated).
// LOADED (M = 2): the forward records of the coupled edges (FwdRec, one plane of eplane
// doubles per field, indexed like the sweep kernel's STORE output) are read from est instead
// of being rebuilt.
template <int M, int DIR, bool LOADED>
__global__ void __launch_bounds__(kAdjThreads, 2)
adjoint_sweep_kernel(DevParams P, const LevelDesc* __restrict__ descs, const SweepItem* __restrict__ items,
                     const int* __restrict__ n_items_dev, const double* __restrict__ state,
                     const double* __restrict__ lam_out, double* __restrict__ lam_in, double* __restrict__ gB,
                     unsigned int* __restrict__ status, const double* __restrict__ est, long long eplane) {
  using R = Rec<M>;
  constexpr int RN = ARec<M>::N;
  constexpr int F = 3 * M;
  constexpr int NE = 2 * F + 2;  // edge outputs: qL_b, qR_b, BL_b, BR_b
  extern __shared__ double smem[];
  double* cell = smem;                       // [RN][kMaxCells]
  double* lamo = cell + RN * kMaxCells;      // [F][kMaxCells] (normal frame)
  double* eout = lamo + F * kMaxCells;       // [NE][kMaxEdges]
  unsigned char* wetb = reinterpret_cast<unsigned char*>(eout + NE * kMaxEdges);
  const int n_items = *n_items_dev;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const SweepItem item = items[it];
    const LevelDesc& D = descs[item.desc];
    const int len = item.len, nl = item.nlines;
    const int NX = D.NX, NY = D.NY, Pt = D.P;
    const size_t plane = (size_t)NY * Pt;
    const double nu = (*D.dt) * (DIR == 0 ? D.inv_dx : D.inv_dy);
    // ---- load cells -1 .. len of every line (mirrored at walls), and their output cotangents
    const int ncell = nl * (len + 2);
    for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
      int l, k;
      if (DIR == 0) { l = t / (len + 2); k = t - l * (len + 2); }
      else { k = t / nl; l = t - k * nl; }
      int i, j;
      if (DIR == 0) { i = item.i0 - 1 + k; j = item.j0 + l; }
      else { i = item.i0 + l; j = item.j0 - 1 + k; }
      double sgn = 1.0;
      bool ghost = false;
      if (DIR == 0) {
        if (i < 0) { i = -1 - i; sgn = -1.0; ghost = true; }
        else if (i >= NX) { i = 2 * NX - 1 - i; sgn = -1.0; ghost = true; }
      } else {
        if (j < 0) { j = -1 - j; sgn = -1.0; ghost = true; }
        else if (j >= NY) { j = 2 * NY - 1 - j; sgn = -1.0; ghost = true; }
      }
      const size_t o = (size_t)j * Pt + i;
      const int c = acslot<DIR>(l, k, len, nl);
      double rec[RN];
      rec[R::BB] = D.B[o];
      int wet = 0;
      bool above = true;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const double h = state[(3 * m) * plane + o];
        const double hu = state[(3 * m + 1) * plane + o];
        const double hv = state[(3 * m + 2) * plane + o];
        const double hn = (DIR == 0 ? hu : hv) * sgn;
        const double ht = DIR == 0 ? hv : hu;
        rec[3 * m] = h; rec[3 * m + 1] = hn; rec[3 * m + 2] = ht;
        const bool w = above && (h > P.dry_tol);
        above = w;
        wet |= w ? (1 << m) : 0;
        double un = 0.0, ut = 0.0, is = 0.0, sq;
        if (w) {  // 1/sqrt(h) once; 1/h and sqrt(h) from it
          is = rsqrt(h);
          const double ih = is * is;
          un = hn * ih; ut = ht * ih;
          sq = h * is;
        } else {
          sq = sqrt(fmax(h, 0.0));
        }
        rec[R::UN + 2 * m] = un; rec[R::UN + 2 * m + 1] = ut;
        rec[R::SQ + m] = sq;
        rec[ARec<M>::IS + m] = is;
        // cotangent of the sweep output at this cell (zero for a wall ghost: not an output)
        const double lh = ghost ? 0.0 : lam_out[(3 * m) * plane + o];
        const double lu = ghost ? 0.0 : lam_out[(3 * m + 1) * plane + o];
        const double lv = ghost ? 0.0 : lam_out[(3 * m + 2) * plane + o];
        lamo[(3 * m) * kMaxCells + c] = lh;
        lamo[(3 * m + 1) * kMaxCells + c] = DIR == 0 ? lu : lv;
        lamo[(3 * m + 2) * kMaxCells + c] = DIR == 0 ? lv : lu;
      }
      double acc = rec[R::BB];
#pragma unroll
      for (int m = M - 1; m >= 0; --m) { acc = acc + rec[3 * m]; rec[R::ETA + m] = acc; }
#pragma unroll
      for (int f = 0; f < RN; ++f) cell[f * kMaxCells + c] = rec[f];
      wetb[c] = (unsigned char)wet;
    }
    __syncthreads();
    // ---- edge VJPs: edge e between cells e-1 and e (e = 0 .. len)
    const int nedge = nl * (len + 1);
    for (int t = threadIdx.x; t < nedge; t += blockDim.x) {
      int l, e;
      if (DIR == 0) { l = t / (len + 1); e = t - l * (len + 1); }
      else { e = t / nl; l = t - e * nl; }
      const int cl = acslot<DIR>(l, e, len, nl), cr = acslot<DIR>(l, e + 1, len, nl);
      double cL[RN], cR[RN], amb[6], apb[6];
#pragma unroll
      for (int f = 0; f < RN; ++f) { cL[f] = cell[f * kMaxCells + cl]; cR[f] = cell[f * kMaxCells + cr]; }
#pragma unroll
      for (int f = 0; f < 6; ++f) { amb[f] = 0.0; apb[f] = 0.0; }
      // A-dQ of this edge updates the left cell, A+dQ the right one, both scaled by -nu; the
      // VJP is linear in these cotangents, so the factor -nu is applied per cell in the gather.
#pragma unroll
      for (int f = 0; f < F; ++f) {
        amb[f] = lamo[f * kMaxCells + cl];
        apb[f] = lamo[f * kMaxCells + cr];
      }
      double qLb[6] = {0, 0, 0, 0, 0, 0}, qRb[6] = {0, 0, 0, 0, 0, 0}, BLb = 0.0, BRb = 0.0;
      bool ok;
      if constexpr (LOADED && M == 2) {
        ok = wetb[cl] == 3 && wetb[cr] == 3;
        if (ok) {
          // edge e of the tile lies left of (below) cell i0 + e (j0 + e) of its line
          const size_t gi = DIR == 0 ? (size_t)(item.j0 + l) * (NX + 1) + (item.i0 + e)
                                     : (size_t)(item.j0 + e) * NX + (item.i0 + l);
          double Fr[FwdRec::N];
#pragma unroll
          for (int k = 0; k < FwdRec::N; ++k) Fr[k] = est[(size_t)k * eplane + gi];
          edge_rev_2(P, cL, cR, Fr, amb, apb, qLb, qRb, BLb, BRb);
        }
      } else {
        ok = (M == 2) ? edge_vjp_2(P, cL, cR, wetb[cl], wetb[cr], amb, apb, qLb, qRb, BLb, BRb)
                      : edge_vjp_1(P, cL, cR, wetb[cl], wetb[cr], amb, apb, qLb, qRb, BLb, BRb);
      }
      if (!ok) atomicOr(status, 4u);
      const int es = aeslot<DIR>(l, e, len, nl);
#pragma unroll
      for (int f = 0; f < F; ++f) {
        eout[f * kMaxEdges + es] = qLb[f];
        eout[(F + f) * kMaxEdges + es] = qRb[f];
      }
      eout[(2 * F) * kMaxEdges + es] = BLb;
      eout[(2 * F + 1) * kMaxEdges + es] = BRb;
    }
    __syncthreads();
    // ---- gather per cell: lam_in = lam_out + right side of edge k + left side of edge k+1,
    // plus the ghost cotangents folded back at walls
    const int ncl = nl * len;
    for (int t = threadIdx.x; t < ncl; t += blockDim.x) {
      int l, k;
      if (DIR == 0) { l = t / len; k = t - l * len; }
      else { k = t / nl; l = t - k * nl; }
      const int c = acslot<DIR>(l, k + 1, len, nl);
      const int ew = aeslot<DIR>(l, k, len, nl), ee = aeslot<DIR>(l, k + 1, len, nl);
      int i, j;
      if (DIR == 0) { i = item.i0 + k; j = item.j0 + l; }
      else { i = item.i0 + l; j = item.j0 + k; }
      const int a = DIR == 0 ? i : j, NA = DIR == 0 ? NX : NY;
      double v[F];
#pragma unroll
      for (int f = 0; f < F; ++f) v[f] = eout[(F + f) * kMaxEdges + ew] + eout[f * kMaxEdges + ee];
      double bb = eout[(2 * F + 1) * kMaxEdges + ew] + eout[(2 * F) * kMaxEdges + ee];
      if (a == 0) {  // ghost -1 = mirror of this cell: its cotangent (left side of edge 0)
#pragma unroll
        for (int f = 0; f < F; ++f) v[f] += (f % 3 == 1 ? -1.0 : 1.0) * eout[f * kMaxEdges + ew];
        bb += eout[(2 * F) * kMaxEdges + ew];
      }
      if (a == NA - 1) {  // ghost NA = mirror of this cell (right side of edge NA)
#pragma unroll
        for (int f = 0; f < F; ++f) v[f] += (f % 3 == 1 ? -1.0 : 1.0) * eout[(F + f) * kMaxEdges + ee];
        bb += eout[(2 * F + 1) * kMaxEdges + ee];
      }
      const size_t o = (size_t)j * Pt + i;
#pragma unroll
      for (int f = 0; f < F; ++f) v[f] = lamo[f * kMaxCells + c] - nu * v[f];
      bb = -nu * bb;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        lam_in[(3 * m) * plane + o] = v[3 * m];
        lam_in[(3 * m + 1) * plane + o] = DIR == 0 ? v[3 * m + 1] : v[3 * m + 2];
        lam_in[(3 * m + 2) * plane + o] = DIR == 0 ? v[3 * m + 2] : v[3 * m + 1];
      }
      gB[o] += bb;
    }
    __syncthreads();
  }
}

static size_t adjoint_smem_bytes(int M) {
  const int rn = 8 * M + 1, F = 3 * M, ne = 2 * F + 2;
  return (size_t)rn * kMaxCells * 8 + (size_t)F * kMaxCells * 8 + (size_t)ne * kMaxEdges * 8 + kMaxCells;
}

template <int M, int DIR, bool LOADED>
static cudaError_t launch_adjoint_t(const DevParams& P, const LevelDesc* descs, const SweepItem* items, const int* n,
                                    int grid, const double* state, const double* lam_out, double* lam_in, double* gB,
                                    unsigned int* status, cudaStream_t st, const double* est, long long eplane) {
  const size_t sm = adjoint_smem_bytes(M);
  static std::atomic<unsigned long long> attr_set{0};
  cudaError_t e = set_smem_limit_once(attr_set, adjoint_sweep_kernel<M, DIR, LOADED>, (int)sm);
  if (e != cudaSuccess) return e;
  adjoint_sweep_kernel<M, DIR, LOADED><<<grid, kAdjThreads, sm, st>>>(P, descs, items, n, state, lam_out, lam_in,
                                                                       gB, status, est, eplane);
  return cudaGetLastError();
}

// est: forward records of the swept step (M = 2 only), or null to rebuild them per edge.
static cudaError_t launch_adjoint_sweep(int dir, const DevParams& P, const LevelDesc* descs, const SweepItem* items,
                                        const int* n, int grid, const double* state, const double* lam_out,
                                        double* lam_in, double* gB, unsigned int* status, cudaStream_t st,
                                        const double* est = nullptr, long long eplane = 0) {
  if (P.M == 1)
    return dir == 0 ? launch_adjoint_t<1, 0, false>(P, descs, items, n, grid, state, lam_out, lam_in, gB, status, st,
                                                    nullptr, 0)
                    : launch_adjoint_t<1, 1, false>(P, descs, items, n, grid, state, lam_out, lam_in, gB, status, st,
                                                    nullptr, 0);
  if (est != nullptr)
    return dir == 0 ? launch_adjoint_t<2, 0, true>(P, descs, items, n, grid, state, lam_out, lam_in, gB, status, st,
                                                   est, eplane)
                    : launch_adjoint_t<2, 1, true>(P, descs, items, n, grid, state, lam_out, lam_in, gB, status, st,
                                                   est, eplane);
  return dir == 0 ? launch_adjoint_t<2, 0, false>(P, descs, items, n, grid, state, lam_out, lam_in, gB, status, st,
                                                  nullptr, 0)
                  : launch_adjoint_t<2, 1, false>(P, descs, items, n, grid, state, lam_out, lam_in, gB, status, st,
                                                  nullptr, 0);
}

// Gauge misfit of one state: loss += sum_g (eta_1 - obs_g)^2, summed in gauge order by one
// thread (deterministic); with lam != null also adds its gradient 2 (eta_1 - obs_g) to the
// cotangents of h_1, ..., h_M and of B at the gauge cells.
__global__ void gauge_misfit_kernel(int M, const LevelDesc* __restrict__ descs, const double* __restrict__ q,
                                    const int* __restrict__ gij, int ng, const double* __restrict__ obs,
                                    double* loss, double* lam, double* gB) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const LevelDesc& D = descs[0];
  const size_t plane = (size_t)D.NY * D.P;
  double s = 0.0;
  for (int g = 0; g < ng; ++g) {
    const size_t o = (size_t)gij[2 * g + 1] * D.P + gij[2 * g];
    double eta = D.B[o];
    for (int m = M - 1; m >= 0; --m) eta = eta + q[(3 * m) * plane + o];
    const double r = eta - obs[g];
    s += r * r;
    if (lam) {
      for (int m = 0; m < M; ++m) lam[(3 * m) * plane + o] += 2.0 * r;
      gB[o] += 2.0 * r;
    }
  }
  if (loss) *loss += s;
}

}  // namespace mlswe

using namespace mlswe;

namespace {

struct Adjoint {
  int n_steps = 0, ckpt = 0, ng = 0;
  size_t state_bytes = 0;
  std::vector<double*> ckpts;  // [n_steps / ckpt + 1]
  std::vector<double*> slots;  // [ckpt + 1] recomputed states of a segment
  std::vector<double*> qstar;  // [ckpt] their states after the x sweep
  double* lam = nullptr;
  double* lam2 = nullptr;
  double* gB = nullptr;
  int* gij = nullptr;
  double* obs = nullptr;
  double* loss = nullptr;
  LevelDesc* descs = nullptr;  // [ckpt] level-0 descriptors: step a reads slots[a], writes slots[a+1], qstar[a]
  SweepItem* items[2] = {nullptr, nullptr};  // tiles of the transposed sweeps, per direction
  int* n_items[2] = {nullptr, nullptr};
  int item_cap[2] = {0, 0};
  int tile[2][2] = {{0, 0}, {0, 0}};         // chosen (len, lines) per direction
  bool forward_done = false;
  bool last_kept = false;      // the slots hold the last segment as the forward pass left it
  // Per-edge forward records (FwdRec) of every recomputed step, M = 2: [ckpt][2 sweeps][N]
  // planes of eplane doubles; null when switched off or when the memory was not available.
  bool keep_edges = true;
  double* estore = nullptr;
  long long eplane = 0;
};

}  // namespace

// The adjoint buffers hang off the hierarchy (device memory is in its allocation list
// and is released with it; the host record is deleted by adjoint_release).
static Adjoint* adj_of(mlswe_hier* h, bool create) {
  if (!h->adj && create) h->adj = new Adjoint();
  return (Adjoint*)h->adj;
}

namespace mlswe {
void adjoint_release(Hier* H) {
  delete (Adjoint*)H->adj;
  H->adj = nullptr;
}
}  // namespace mlswe

static mlswe_status afail(mlswe_hier* h, mlswe_status s, const char* msg) {
  h->err = msg;
  return s;
}

#define ACUDA(h, call)                                                                \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
      return MLSWE_ECUDA;                                                             \
    }                                                                                 \
  } while (0)

// Copies a pitched level state.
static cudaError_t copy_state(Hier* H, double* dst, const double* src) {
  const Level& V = H->mem[0].lev[0];
  return cudaMemcpyAsync(dst, src, (size_t)3 * H->cfg.M * V.NY * V.P * 8, cudaMemcpyDeviceToDevice, H->st);
}

// Descriptors of the recomputation slots (built once per setup): step a of a segment reads
// slots[a], keeps its x-sweep result in qstar[a] and writes slots[a + 1].
static mlswe_status adj_build_descs(Hier* H, Adjoint* A) {
  const Level& V = H->mem[0].lev[0];
  std::vector<LevelDesc> d(A->ckpt);
  for (int a = 0; a < A->ckpt; ++a) {
    LevelDesc& D = d[a];
    D = LevelDesc{};
    D.q[0] = A->slots[a];
    D.q[1] = A->slots[a + 1];
    D.qs = A->qstar[a];
    D.B = V.B;
    D.dt = H->d_dt;
    D.NX = V.NX; D.NY = V.NY; D.P = V.P;
    D.inv_dx = 1.0 / V.dx; D.inv_dy = 1.0 / V.dy;
  }
  ACUDA(H, cudaMemcpyAsync(A->descs, d.data(), d.size() * sizeof(LevelDesc), cudaMemcpyHostToDevice, H->st));
  ACUDA(H, cudaStreamSynchronize(H->st));
  return MLSWE_OK;
}

// Tiles of len x lines cells over the whole level for the transposed sweep in direction dir
// (along x: rows j, cells i; along y: columns i, cells j).
static mlswe_status adj_build_items(mlswe_hier* H, Adjoint* A, int dir, int len, int lines) {
  const Level& V = H->mem[0].lev[0];
  const int NA = dir == 0 ? V.NX : V.NY, NL = dir == 0 ? V.NY : V.NX;
  std::vector<SweepItem> it;
  for (int l = 0; l < NL; l += lines)
    for (int a = 0; a < NA; a += len) {
      SweepItem s;
      s.desc = 0;
      s.i0 = dir == 0 ? a : l;
      s.j0 = dir == 0 ? l : a;
      s.len = std::min(len, NA - a);
      s.nlines = std::min(lines, NL - l);
      s.flags = 1;
      it.push_back(s);
    }
  if ((int)it.size() > A->item_cap[dir]) {
    if (A->items[dir]) dev_free(H, A->items[dir]);
    A->items[dir] = (SweepItem*)dev_alloc(H, it.size() * sizeof(SweepItem));
    if (!A->items[dir]) return afail(H, MLSWE_ENOMEM, "adjoint_setup: out of memory");
    A->item_cap[dir] = (int)it.size();
  }
  if (!A->n_items[dir]) {
    A->n_items[dir] = (int*)dev_alloc(H, sizeof(int));
    if (!A->n_items[dir]) return afail(H, MLSWE_ENOMEM, "adjoint_setup: out of memory");
  }
  const int n = (int)it.size();
  ACUDA(H, cudaMemcpyAsync(A->items[dir], it.data(), it.size() * sizeof(SweepItem), cudaMemcpyHostToDevice, H->st));
  ACUDA(H, cudaMemcpyAsync(A->n_items[dir], &n, sizeof(int), cudaMemcpyHostToDevice, H->st));
  ACUDA(H, cudaStreamSynchronize(H->st));
  A->tile[dir][0] = len;
  A->tile[dir][1] = lines;
  return MLSWE_OK;
}

// Picks the tile shape of each transposed sweep by timing it (CUDA events) on the level's
// current state with zero cotangents; candidates have at most kAdjThreads edges per tile.
// Leaves lam, lam2 and gB with scratch values (the backward pass clears them).
static mlswe_status adj_autotune(mlswe_hier* H, Adjoint* A) {
  static const int cand[][2] = {{125, 1}, {61, 2}, {29, 4}};
  const Level& V = H->mem[0].lev[0];
  const double* q = V.q[H->parity[0]];
  ACUDA(H, cudaMemsetAsync(A->lam, 0, A->state_bytes, H->st));
  cudaEvent_t e0, e1;
  ACUDA(H, cudaEventCreate(&e0));
  ACUDA(H, cudaEventCreate(&e1));
  const int grid = 2 * H->num_sms;
  for (int dir = 0; dir < 2; ++dir) {
    float best = 1e30f;
    int bl = cand[0][0], bn = cand[0][1];
    for (const auto& c : cand) {
      mlswe_status s = adj_build_items(H, A, dir, c[0], c[1]);
      if (s != MLSWE_OK) return s;
      ACUDA(H, launch_adjoint_sweep(dir, H->dp, H->d_desc, A->items[dir], A->n_items[dir], grid, q, A->lam, A->lam2,
                                    A->gB, H->d_status, H->st));
      ACUDA(H, cudaEventRecord(e0, H->st));
      for (int k = 0; k < 3; ++k)
        ACUDA(H, launch_adjoint_sweep(dir, H->dp, H->d_desc, A->items[dir], A->n_items[dir], grid, q, A->lam,
                                      A->lam2, A->gB, H->d_status, H->st));
      ACUDA(H, cudaEventRecord(e1, H->st));
      ACUDA(H, cudaEventSynchronize(e1));
      float ms = 0.f;
      ACUDA(H, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; bl = c[0]; bn = c[1]; }
    }
    mlswe_status s = adj_build_items(H, A, dir, bl, bn);
    if (s != MLSWE_OK) return s;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return MLSWE_OK;
}

// Forward records of sweep dir of step a of a segment, or null.
static double* adj_edge_records(Adjoint* A, int a, int dir) {
  if (!A->estore) return nullptr;
  return A->estore + ((size_t)(2 * a + dir) * FwdRec::N) * (size_t)A->eplane;
}

// Step a of the segment being recomputed (both sweeps, no fluxes recorded; the per-edge
// forward records are kept when the store is on).
static mlswe_status adj_forward_step(Hier* H, Adjoint* A, int a) {
  for (int dir = 0; dir < 2; ++dir) {
    Hier::WorkList& W = H->wl[dir];
    const int ctas = H->shape[dir].ctas;
    int tok;
    timer_begin(H, KC_ADJOINT, &tok);
    ACUDA(H, launch_sweep(dir, H->dp, A->descs + a, W.d_items, W.d_count, W.packed ? W.d_tile_off : nullptr,
                          ctas * H->num_sms, 0, 0, H->d_smax, nullptr, H->st, ctas, adj_edge_records(A, a, dir),
                          A->eplane));
    timer_end(H, tok);
  }
  return MLSWE_OK;
}

// Controls of the gauge-misfit problem to its initial state (a fluid at rest, Eqs. (4)-(5)):
// the surface eta_1(0) and the bathymetry B (dense [NY][NX]) give, for two layers with the
// interface at rest at eta_2, h_2 = eta_2 - B and h_1 = eta_1 - eta_2; for one layer
// h_1 = eta_1 - B; momenta 0. B is also written into the level's bathymetry.
__global__ void controls_to_state_kernel(int M, int NX, int NY, int P, const double* __restrict__ eta1,
                                         const double* __restrict__ Bc, double eta2, double* __restrict__ q,
                                         double* __restrict__ B) {
  const size_t plane = (size_t)NY * P;
  const long long n = (long long)NX * NY;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / NX), i = (int)(k - (long long)j * NX);
    const size_t o = (size_t)j * P + i;
    const double b = Bc[k], e1 = eta1[k];
    B[o] = b;
    if (M == 2) {
      q[o] = e1 - eta2;
      q[3 * plane + o] = eta2 - b;
      q[4 * plane + o] = 0.0;
      q[5 * plane + o] = 0.0;
    } else {
      q[o] = e1 - b;
    }
    q[plane + o] = 0.0;
    q[2 * plane + o] = 0.0;
  }
}

// Gradients of J with respect to the state Q^0 (lam, pitched) and to B at fixed Q^0 (gB)
// to the gradients with respect to the controls, by the chain rule of the map above:
// dJ/deta_1 = dJ/dh_1, dJ/dB = gB - dJ/dh_M (h_M = eta_M - B is the only depth B enters).
__global__ void state_grad_to_controls_kernel(int M, int NX, int NY, int P, const double* __restrict__ lam,
                                              const double* __restrict__ gB, double* __restrict__ d_eta1,
                                              double* __restrict__ d_B) {
  const size_t plane = (size_t)NY * P;
  const long long n = (long long)NX * NY;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / NX), i = (int)(k - (long long)j * NX);
    const size_t o = (size_t)j * P + i;
    d_eta1[k] = lam[o];
    d_B[k] = gB[o] - lam[(size_t)3 * (M - 1) * plane + o];
  }
}

// Device (or managed) memory that kernels can dereference.
static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static mlswe_status fixed_backward_core(mlswe_h h);

extern "C" {

mlswe_status mlswe_adjoint_setup(mlswe_h h, int n_steps, int ckpt_every, int n_gauges, const int32_t* gauge_ij,
                                 const double* obs) {
  if (!h || n_steps < 1 || ckpt_every < 1 || n_gauges < 0 || (n_gauges > 0 && (!gauge_ij || !obs)))
    return h ? afail(h, MLSWE_EINVAL, "adjoint_setup: bad argument") : MLSWE_EINVAL;
  if (h->n_members != 1 || h->L != 1 || h->cfg.order != 1 || h->cfg.M > 2 || h->cfg.unsplit)
    return afail(h, MLSWE_EINVAL, "adjoint_setup: needs one member, one level, order 1, M <= 2 and the split step");
  const Level& V = h->mem[0].lev[0];
  for (int g = 0; g < n_gauges; ++g)
    if (gauge_ij[2 * g] < 0 || gauge_ij[2 * g] >= V.NX || gauge_ij[2 * g + 1] < 0 || gauge_ij[2 * g + 1] >= V.NY)
      return afail(h, MLSWE_EINVAL, "adjoint_setup: gauge cell outside the grid");
  Adjoint* A = adj_of(h, true);
  A->n_steps = n_steps;
  A->ckpt = ckpt_every;
  A->ng = n_gauges;
  A->state_bytes = (size_t)3 * h->cfg.M * V.NY * V.P * 8;
  const int nck = n_steps / ckpt_every + 1;
  auto grab = [&](size_t bytes) { return (double*)dev_alloc(h, bytes); };
  while ((int)A->ckpts.size() < nck) A->ckpts.push_back(grab(A->state_bytes));
  while ((int)A->slots.size() < ckpt_every + 1) A->slots.push_back(grab(A->state_bytes));
  while ((int)A->qstar.size() < ckpt_every) A->qstar.push_back(grab(A->state_bytes));
  if (!A->lam) A->lam = grab(A->state_bytes);
  if (!A->lam2) A->lam2 = grab(A->state_bytes);
  if (!A->gB) A->gB = grab((size_t)V.NY * V.P * 8);
  if (!A->loss) A->loss = grab(64);
  if (A->descs) dev_free(h, A->descs);
  A->descs = (LevelDesc*)dev_alloc(h, ckpt_every * sizeof(LevelDesc));
  if (A->gij) dev_free(h, A->gij);
  if (A->obs) dev_free(h, A->obs);
  A->gij = (int*)dev_alloc(h, std::max(1, 2 * n_gauges) * sizeof(int));
  A->obs = grab(std::max<size_t>(1, (size_t)n_steps * n_gauges) * 8);
  // per-edge forward records of a segment (two-layer only); without the memory the
  // transposed sweeps rebuild them
  if (A->estore) dev_free(h, A->estore);
  A->estore = nullptr;
  A->eplane = 0;
  if (A->keep_edges && h->cfg.M == 2) {
    // one spare slot per plane takes the records of tile-halo edges (see sweep_kernel)
    const long long plane = ((long long)(V.NX + 1) * (V.NY + 1) + 1 + 31) / 32 * 32;
    A->estore = grab((size_t)ckpt_every * 2 * FwdRec::N * (size_t)plane * 8);
    if (A->estore) A->eplane = plane;
    cudaGetLastError();  // an allocation failure here is not an error of the call
  }
  for (double* p : A->ckpts) if (!p) return afail(h, MLSWE_ENOMEM, "adjoint_setup: out of memory");
  for (double* p : A->slots) if (!p) return afail(h, MLSWE_ENOMEM, "adjoint_setup: out of memory");
  for (double* p : A->qstar) if (!p) return afail(h, MLSWE_ENOMEM, "adjoint_setup: out of memory");
  if (!A->lam || !A->lam2 || !A->gB || !A->loss || !A->descs || !A->gij || !A->obs)
    return afail(h, MLSWE_ENOMEM, "adjoint_setup: out of memory");
  if (n_gauges > 0) {
    ACUDA(h, cudaMemcpyAsync(A->gij, gauge_ij, 2 * n_gauges * sizeof(int), cudaMemcpyHostToDevice, h->st));
    ACUDA(h, cudaMemcpyAsync(A->obs, obs, (size_t)n_steps * n_gauges * 8, cudaMemcpyHostToDevice, h->st));
  }
  mlswe_status s = adj_build_descs(h, A);
  if (s != MLSWE_OK) return s;
  s = adj_autotune(h, A);
  if (s != MLSWE_OK) return s;
  A->forward_done = false;
  A->last_kept = false;
  return MLSWE_OK;
}

mlswe_status mlswe_adjoint_keep_edge_data(mlswe_h h, int enable) {
  if (!h) return MLSWE_EINVAL;
  Adjoint* A = adj_of(h, true);
  A->keep_edges = enable != 0;
  A->n_steps = 0;  // takes effect at the next mlswe_adjoint_setup
  A->forward_done = false;
  return MLSWE_OK;
}

mlswe_status mlswe_fixed_set_controls(mlswe_h h, const double* eta1_0, const double* B, double eta2) {
  if (!h) return MLSWE_EINVAL;
  if (!eta1_0 || !B) return afail(h, MLSWE_EINVAL, "fixed_set_controls: null pointer");
  if (h->n_members != 1 || h->L != 1 || h->cfg.M > 2)
    return afail(h, MLSWE_EINVAL, "fixed_set_controls: needs one member, one level and M <= 2");
  if (!is_device_ptr(eta1_0) || !is_device_ptr(B))
    return afail(h, MLSWE_EINVAL, "fixed_set_controls: eta1_0 and B must be device pointers");
  Level& V = h->mem[0].lev[0];
  controls_to_state_kernel<<<2 * h->num_sms, 256, 0, h->st>>>(h->cfg.M, V.NX, V.NY, V.P, eta1_0, B, eta2,
                                                               V.q[h->parity[0]], V.B);
  h->kernel_launches++;
  ACUDA(h, cudaGetLastError());
  ACUDA(h, cudaStreamSynchronize(h->st));
  h->dt_ready = false;
  return MLSWE_OK;
}

mlswe_status mlswe_fixed_forward(mlswe_h h, const double* eta1_0, const double* B, double eta2, double* loss) {
  mlswe_status s = mlswe_fixed_set_controls(h, eta1_0, B, eta2);
  if (s != MLSWE_OK) return s;
  return mlswe_fixed_forward_state(h, loss);
}

mlswe_status mlswe_fixed_forward_state(mlswe_h h, double* loss) {
  if (!h) return MLSWE_EINVAL;
  Adjoint* A = adj_of(h, false);
  if (!A || A->n_steps < 1) return afail(h, MLSWE_EINVAL, "fixed_forward: call mlswe_adjoint_setup first");
  NvtxRange range("mlswe_fixed_forward");
  for (int dir = 0; dir < 2; ++dir) {
    mlswe_status s = ensure_worklist(h, 0, dir);
    if (s != MLSWE_OK) return s;
  }
  ACUDA(h, cudaMemsetAsync(A->loss, 0, 8, h->st));
  ACUDA(h, copy_state(h, A->ckpts[0], h->mem[0].lev[0].q[h->parity[0]]));
  // Steps of the last segment run in the recomputation slots (same kernels, same dt), so
  // the backward pass starts from them without recomputing that segment.
  const int C = A->ckpt, N = A->n_steps;
  const int k_last = ((N + C - 1) / C - 1) * C;
  for (int n = 1; n <= N; ++n) {
    const double* qn;
    if (n - 1 >= k_last) {
      const int a = n - 1 - k_last;
      if (a == 0) ACUDA(h, copy_state(h, A->slots[0], h->mem[0].lev[0].q[h->parity[0]]));
      mlswe_status s = adj_forward_step(h, A, a);
      if (s != MLSWE_OK) return s;
      qn = A->slots[a + 1];
    } else {
      mlswe_status s = enqueue_level_step(h, 0, 1);
      if (s != MLSWE_OK) return s;
      qn = h->mem[0].lev[0].q[h->parity[0]];
    }
    int tok;
    timer_begin(h, KC_OTHER, &tok);
    gauge_misfit_kernel<<<1, 32, 0, h->st>>>(h->cfg.M, h->d_desc, qn, A->gij, A->ng,
                                             A->obs + (size_t)(n - 1) * A->ng, A->loss, nullptr, nullptr);
    ACUDA(h, cudaGetLastError());
    timer_end(h, tok);
    if (n % C == 0 && n / C < (int)A->ckpts.size()) ACUDA(h, copy_state(h, A->ckpts[n / C], qn));
  }
  // the hierarchy's state is Q^N, as after N plain steps
  ACUDA(h, copy_state(h, h->mem[0].lev[0].q[h->parity[0]], A->slots[N - k_last]));
  A->last_kept = true;
  double l = 0.0;
  ACUDA(h, cudaMemcpyAsync(&l, A->loss, 8, cudaMemcpyDeviceToHost, h->st));
  ACUDA(h, cudaStreamSynchronize(h->st));
  if (loss) *loss = l;
  A->forward_done = true;
  return MLSWE_OK;
}

mlswe_status mlswe_fixed_backward_state(mlswe_h h, double* dL_dq0, double* dL_dB) {
  if (!h || !dL_dq0 || !dL_dB) return h ? afail(h, MLSWE_EINVAL, "fixed_backward_state: bad argument") : MLSWE_EINVAL;
  if (!is_device_ptr(dL_dq0) || !is_device_ptr(dL_dB))
    return afail(h, MLSWE_EINVAL, "fixed_backward_state: outputs must be device pointers");
  mlswe_status s = fixed_backward_core(h);
  if (s != MLSWE_OK) return s;
  Adjoint* A = adj_of(h, false);
  const Level& V = h->mem[0].lev[0];
  const int F = 3 * h->cfg.M;
  ACUDA(h, cudaMemcpy2DAsync(dL_dq0, V.NX * 8, A->lam, V.P * 8, V.NX * 8, (size_t)F * V.NY, cudaMemcpyDeviceToDevice,
                             h->st));
  ACUDA(h, cudaMemcpy2DAsync(dL_dB, V.NX * 8, A->gB, V.P * 8, V.NX * 8, V.NY, cudaMemcpyDeviceToDevice, h->st));
  ACUDA(h, cudaStreamSynchronize(h->st));
  return MLSWE_OK;
}

mlswe_status mlswe_fixed_backward(mlswe_h h, double* dL_deta1_0, double* dL_dB) {
  if (!h || !dL_deta1_0 || !dL_dB) return h ? afail(h, MLSWE_EINVAL, "fixed_backward: bad argument") : MLSWE_EINVAL;
  if (!is_device_ptr(dL_deta1_0) || !is_device_ptr(dL_dB))
    return afail(h, MLSWE_EINVAL, "fixed_backward: outputs must be device pointers");
  mlswe_status s = fixed_backward_core(h);
  if (s != MLSWE_OK) return s;
  Adjoint* A = adj_of(h, false);
  const Level& V = h->mem[0].lev[0];
  state_grad_to_controls_kernel<<<2 * h->num_sms, 256, 0, h->st>>>(h->cfg.M, V.NX, V.NY, V.P, A->lam, A->gB,
                                                                    dL_deta1_0, dL_dB);
  h->kernel_launches++;
  ACUDA(h, cudaGetLastError());
  ACUDA(h, cudaStreamSynchronize(h->st));
  return MLSWE_OK;
}

}  // extern "C"

// The backward pass: lam = dJ/dQ^0 and gB = dJ/dB at fixed Q^0, in the adjoint's buffers.
static mlswe_status fixed_backward_core(mlswe_h h) {
  Adjoint* A = adj_of(h, false);
  if (!A || !A->forward_done) return afail(h, MLSWE_EINVAL, "fixed_backward: run mlswe_fixed_forward first");
  NvtxRange range("mlswe_fixed_backward");
  const Level& V = h->mem[0].lev[0];
  const int M = h->cfg.M, F = 3 * M;
  const size_t plane = (size_t)V.NY * V.P;
  const int grid = 2 * h->num_sms;
  ACUDA(h, cudaMemsetAsync(A->lam, 0, A->state_bytes, h->st));
  ACUDA(h, cudaMemsetAsync(A->gB, 0, plane * 8, h->st));
  ACUDA(h, cudaMemsetAsync(h->d_status, 0, 4, h->st));
  const int N = A->n_steps, C = A->ckpt;
  const int nseg = (N + C - 1) / C;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int k0 = seg * C, k1 = std::min(N, k0 + C);
    // recompute Q^{k0} .. Q^{k1} into the slots, keeping every step's Q* (the last segment
    // is still there from the forward pass unless an earlier backward pass reused the slots)
    if (!(seg == nseg - 1 && A->last_kept)) {
      ACUDA(h, copy_state(h, A->slots[0], A->ckpts[seg]));
      for (int n = k0; n < k1; ++n) {
        mlswe_status s = adj_forward_step(h, A, n - k0);
        if (s != MLSWE_OK) return s;
      }
    }
    if (seg < nseg - 1) A->last_kept = false;
    for (int n = k1 - 1; n >= k0; --n) {
      const int a = n - k0;
      // gauge term of J at Q^{n+1}
      int tok;
      timer_begin(h, KC_OTHER, &tok);
      gauge_misfit_kernel<<<1, 32, 0, h->st>>>(M, h->d_desc, A->slots[a + 1], A->gij, A->ng,
                                               A->obs + (size_t)n * A->ng, nullptr, A->lam, A->gB);
      ACUDA(h, cudaGetLastError());
      timer_end(h, tok);
      // transposed y sweep (on Q* of step n), then transposed x sweep (on Q^n)
      timer_begin(h, KC_ADJOINT, &tok);
      ACUDA(h, launch_adjoint_sweep(1, h->dp, A->descs + a, A->items[1], A->n_items[1], grid, A->qstar[a], A->lam,
                                    A->lam2, A->gB, h->d_status, h->st, adj_edge_records(A, a, 1), A->eplane));
      timer_end(h, tok);
      timer_begin(h, KC_ADJOINT, &tok);
      ACUDA(h, launch_adjoint_sweep(0, h->dp, A->descs + a, A->items[0], A->n_items[0], grid, A->slots[a], A->lam2,
                                    A->lam, A->gB, h->d_status, h->st, adj_edge_records(A, a, 0), A->eplane));
      timer_end(h, tok);
    }
  }
  unsigned int status = 0;
  ACUDA(h, cudaMemcpyAsync(&status, h->d_status, 4, cudaMemcpyDeviceToHost, h->st));
  ACUDA(h, cudaStreamSynchronize(h->st));
  if (status & 4u) return afail(h, MLSWE_EINVAL, "fixed_backward: a layer was not wet on both sides of an edge");
  return MLSWE_OK;
}
