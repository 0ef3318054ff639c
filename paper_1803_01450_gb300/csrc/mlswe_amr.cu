// AMR transfer kernels: refinement of Sec. 2.1 (new fine cells and fine ghost
// cells), coarsening of Sec. 2.2, refinement flags, patch masks, mass reflux,
// wave speeds and the device-side time step.
//
// All box kernels are persistent: a fixed grid loops over a device-resident
// item table whose length is read from device memory, so a captured CUDA
// graph stays valid when a regrid rewrites the tables. One CTA works on one
// item (a box of at most 64 x 64 cells) at a time, one thread per cell.
#include <cuda_runtime.h>
#include "mlswe_internal.h"

namespace mlswe {

// ---------------------------------------------------------------------------
// Refinement, Sec. 2.1 in 2-D. For a fine cell (I, J) of level l+1 inside
// coarse cell k = (I / r, J / r), for every layer from the bottom up (Sec. 2.1,
// last paragraph):
//   eta_m at k and its 4 face neighbours (Eq. (4), summed from the bottom),
//   slope numerators minmod(eta_k - eta_{k-1}, eta_{k+1} - eta_k) per direction
//   (Eq. (10) times dx; a neighbour dry in layer m gives a zero difference),
//   eta_f = eta_k + sx ((a + 1/2)/r - 1/2) + sy ((b + 1/2)/r - 1/2),
//   Bhat_f = B_f + h_{M,f} + ... + h_{m+1,f} (Eq. (5), fine layers below),
//   h_{m,f} = max(0, eta_f - Bhat_f);
// the momenta take the same limited linear reconstruction of the conserved
// variables and are zero where h_{m,f} <= dry_tol. A layer not wet in k (top-down
// rule) gives zero depth and momentum. The coarse state is (1-alpha) Q^n + alpha Q^{n+1}.
// ---------------------------------------------------------------------------
// minmod on the bit patterns (integer unit): 0 when a and b differ in sign or either is zero,
// else the one of smaller magnitude (a on ties). The same as the product test (a b <= 0 gives
// 0) except where a b underflows to zero for same-signed |a|, |b| below about 1e-154, where
// the product test gives 0.
__device__ __forceinline__ double minmod_bits(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  const unsigned long long ax = (unsigned long long)x & 0x7fffffffffffffffull;
  const unsigned long long ay = (unsigned long long)y & 0x7fffffffffffffffull;
  if ((x ^ y) < 0 || ax == 0 || ay == 0) return 0.0;
  return ax <= ay ? a : b;
}

template <int M>
__device__ void coarse_cell(const LevelDesc& C, const double* qo, const double* qn, double alpha, int i, int j,
                            double* q /*[3M]*/, double& B) {
  // wall mirror: the normal momentum changes sign (on the sign bit)
  long long sx = 0, sy = 0;
  constexpr long long kSign = (long long)0x8000000000000000ull;
  if (i < 0) { i = -1 - i; sx = kSign; } else if (i >= C.NX) { i = 2 * C.NX - 1 - i; sx = kSign; }
  if (j < 0) { j = -1 - j; sy = kSign; } else if (j >= C.NY) { j = 2 * C.NY - 1 - j; sy = kSign; }
  const size_t o = (size_t)j * C.P + i, plane = (size_t)C.NY * C.P;
  if (alpha == 0.0) {  // (1 - 0) q_old + 0 q = q_old
#pragma unroll
    for (int f = 0; f < 3 * M; ++f) q[f] = qo[f * plane + o];
  } else {
    const double a1 = 1.0 - alpha;
#pragma unroll
    for (int f = 0; f < 3 * M; ++f) q[f] = a1 * qo[f * plane + o] + alpha * qn[f * plane + o];
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    q[3 * m + 1] = __longlong_as_double(__double_as_longlong(q[3 * m + 1]) ^ sx);
    q[3 * m + 2] = __longlong_as_double(__double_as_longlong(q[3 * m + 2]) ^ sy);
  }
  B = C.B[o];
}

// k / rt for the substeps of a level (0 <= k < rt <= 4 with the ratios 2 and 4): the quotients
// folded at compile time (correctly rounded, as the division is), so the ghost fill does not
// divide per ring cell; other values divide.
__device__ __forceinline__ double substep_fraction(int k, int rt) {
  if (k < 0 || k >= rt || rt > 4) return (double)k / (double)rt;
  switch (rt * 4 + k) {
    case 4: case 8: case 12: case 16: return 0.0;
    case 9: return 1.0 / 2.0;
    case 13: return 1.0 / 3.0;
    case 14: return 2.0 / 3.0;
    case 17: return 1.0 / 4.0;
    case 18: return 2.0 / 4.0;
    case 19: return 3.0 / 4.0;
    default: return (double)k / (double)rt;
  }
}

// Refinement organised per coarse cell (used by the new-patch fill and the ghost fill): the
// coarse cell's state and its four face neighbours' at alpha are loaded once, the wet flags,
// surfaces and minmod slopes of every layer formed once, and then each of its R x R fine
// cells that is wanted is reconstructed from them (the per-fine-cell form recomputes all of
// that for every fine cell). Wet tests and minmod work on bit patterns: depths are >= 0 and
// dry_tol >= 0, so h > dry_tol exactly when bits(h) > bits(dry_tol) as signed integers.
template <int M>
struct CoarsePrep {
  bool wet0[M];          // layer wet in the coarse cell (top-down rule)
  double eta0[M];        // its surface (Eq. (4))
  double se[M][2];       // limited surface differences in x and y (Eq. (10) times dx)
  double c0[M][2];       // its momenta
  double sm[M][2][2];    // limited momentum differences [component][direction]
};

template <int M>
__device__ __forceinline__ void coarse_prep(const LevelDesc& C, const double* qo, const double* qn, double alpha,
                                            int ic, int jc, long long tol_bits, CoarsePrep<M>& S) {
  constexpr int F = 3 * M;
  // coarse cell k and its face neighbours: 0 = k, 1 = west, 2 = east, 3 = south, 4 = north
  double q[5][F], Bc[5];
  coarse_cell<M>(C, qo, qn, alpha, ic, jc, q[0], Bc[0]);
  coarse_cell<M>(C, qo, qn, alpha, ic - 1, jc, q[1], Bc[1]);
  coarse_cell<M>(C, qo, qn, alpha, ic + 1, jc, q[2], Bc[2]);
  coarse_cell<M>(C, qo, qn, alpha, ic, jc - 1, q[3], Bc[3]);
  coarse_cell<M>(C, qo, qn, alpha, ic, jc + 1, q[4], Bc[4]);
#pragma unroll
  for (int m = M - 1; m >= 0; --m) {
    bool wet[5];
    double eta[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      bool wt = true;
#pragma unroll
      for (int n2 = 0; n2 <= m; ++n2) wt = wt && (__double_as_longlong(q[c][3 * n2]) > tol_bits);
      wet[c] = wt;
      double ev = Bc[c];
#pragma unroll
      for (int n2 = M - 1; n2 >= m; --n2) ev = ev + q[c][3 * n2];
      eta[c] = ev;
    }
    S.wet0[m] = wet[0];
    S.eta0[m] = eta[0];
    S.se[m][0] = minmod_bits(wet[1] ? eta[0] - eta[1] : 0.0, wet[2] ? eta[2] - eta[0] : 0.0);
    S.se[m][1] = minmod_bits(wet[3] ? eta[0] - eta[3] : 0.0, wet[4] ? eta[4] - eta[0] : 0.0);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int f = 3 * m + 1 + k;
      const double cv = q[0][f];
      S.c0[m][k] = cv;
      S.sm[m][k][0] = minmod_bits(wet[1] ? cv - q[1][f] : 0.0, wet[2] ? q[2][f] - cv : 0.0);
      S.sm[m][k][1] = minmod_bits(wet[3] ? cv - q[3][f] : 0.0, wet[4] ? q[4][f] - cv : 0.0);
    }
  }
}

// The x parts of fine column a (offset offx from the coarse centre, in coarse cells): the
// surface eta + sx offx and the momenta c + mx offx, once per column.
template <int M>
__device__ __forceinline__ void fine_column(const CoarsePrep<M>& S, double offx, double (&ex)[M],
                                            double (&mx)[M][2]) {
#pragma unroll
  for (int m = 0; m < M; ++m) {
    ex[m] = fma(S.se[m][0], offx, S.eta0[m]);
    mx[m][0] = fma(S.sm[m][0][0], offx, S.c0[m][0]);
    mx[m][1] = fma(S.sm[m][1][0], offx, S.c0[m][1]);
  }
}

// One fine cell of that column (offset offy), bottom layer first: eta_f, Bhat_f = B_f plus the
// fine layers below (Eq. (5)), h = max(0, eta_f - Bhat_f), momenta where h > dry_tol; written
// to the 3M planes of qf at fo.
template <int M>
__device__ __forceinline__ void fine_cell(const CoarsePrep<M>& S, const double (&ex)[M], const double (&mx)[M][2],
                                          double offy, double Bf, long long tol_bits, double* __restrict__ qf,
                                          size_t fplane, size_t fo) {
  constexpr int F = 3 * M;
  double hf[M], out[F];
#pragma unroll
  for (int m = M - 1; m >= 0; --m) {
    double hv = 0.0, huv = 0.0, hvv = 0.0;
    if (S.wet0[m]) {
      const double ef = fma(S.se[m][1], offy, ex[m]);
      double bh = Bf;
#pragma unroll
      for (int n2 = M - 1; n2 > m; --n2) bh = bh + hf[n2];
      const double d = ef - bh;
      hv = __double_as_longlong(d) < 0 ? 0.0 : d;  // max(0, d); -0 gives +0
      if (__double_as_longlong(hv) > tol_bits) {
        huv = fma(S.sm[m][0][1], offy, mx[m][0]);
        hvv = fma(S.sm[m][1][1], offy, mx[m][1]);
      }
    }
    hf[m] = hv;
    out[3 * m] = hv;
    out[3 * m + 1] = huv;
    out[3 * m + 2] = hvv;
  }
#pragma unroll
  for (int f = 0; f < F; ++f) qf[f * fplane + fo] = out[f];
}

// Every fine cell of the item boxes (new patches: fine-index boxes, clipped to the level) from
// the coarse state at alpha, one thread per coarse cell under the box.
template <int M, int R>
__global__ void __launch_bounds__(256)
interp_kernel(DevParams P, const LevelDesc* __restrict__ descs, const InterpItem* __restrict__ items,
              const int* __restrict__ n_items_dev, int par_c, int par_f, double alpha) {
  constexpr double inv_r = 1.0 / (double)R;
  const int n_items = *n_items_dev;
  const long long tol_bits = __double_as_longlong(P.dry_tol);
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const InterpItem item = items[it];
    const LevelDesc& C = descs[item.desc_c];
    const LevelDesc& Fd = descs[item.desc_f];
    const int i0 = max(item.i0, 0), j0 = max(item.j0, 0);
    const int i1 = min(item.i1, Fd.NX), j1 = min(item.j1, Fd.NY);
    if (i0 >= i1 || j0 >= j1) continue;
    const int ic0 = i0 / R, jc0 = j0 / R;
    const int cw = (i1 + R - 1) / R - ic0, ch = (j1 + R - 1) / R - jc0;
    const double* qo = C.q[par_c ^ 1];
    const double* qn = C.q[par_c];
    double* qf = Fd.q[par_f];
    const size_t fplane = (size_t)Fd.NY * Fd.P;
    for (int t = threadIdx.x; t < cw * ch; t += blockDim.x) {
      const int ic = ic0 + t % cw, jc = jc0 + t / cw;
      CoarsePrep<M> S;
      coarse_prep<M>(C, qo, qn, alpha, ic, jc, tol_bits, S);
#pragma unroll
      for (int a = 0; a < R; ++a) {
        const int I = ic * R + a;
        if (I < i0 || I >= i1) continue;
        double ex[M], mx[M][2];
        fine_column<M>(S, (a + 0.5) * inv_r - 0.5, ex, mx);
        double Bcol[R];
#pragma unroll
        for (int b = 0; b < R; ++b) {
          const int J = jc * R + b;
          Bcol[b] = (J >= j0 && J < j1) ? Fd.B[(size_t)J * Fd.P + I] : 0.0;
        }
#pragma unroll
        for (int b = 0; b < R; ++b) {
          const int J = jc * R + b;
          if (J < j0 || J >= j1) continue;
          fine_cell<M>(S, ex, mx, (b + 0.5) * inv_r - 0.5, Bcol[b], tol_bits, qf, fplane, (size_t)J * Fd.P + I);
        }
      }
    }
  }
}

template <int M>
static void launch_interp_m(const DevParams& P, const LevelDesc* descs, const InterpItem* items,
                            const int* n_items_dev, int grid, int r, int par_c, int par_f, double alpha,
                            cudaStream_t st) {
  if (r == 2) interp_kernel<M, 2><<<grid, 256, 0, st>>>(P, descs, items, n_items_dev, par_c, par_f, alpha);
  else interp_kernel<M, 4><<<grid, 256, 0, st>>>(P, descs, items, n_items_dev, par_c, par_f, alpha);
}

// r: the refinement ratio, 2 or 4 (the only ratios a hierarchy accepts).
cudaError_t launch_interp(int M, const DevParams& P, const LevelDesc* descs, const InterpItem* items,
                          const int* n_items_dev, int grid, int r, int par_c, int par_f, double alpha,
                          cudaStream_t st) {
  if (r != 2 && r != 4) return cudaErrorInvalidValue;
  if (M == 1) launch_interp_m<1>(P, descs, items, n_items_dev, grid, r, par_c, par_f, alpha, st);
  else if (M == 3) launch_interp_m<3>(P, descs, items, n_items_dev, grid, r, par_c, par_f, alpha, st);
  else if (M == 4) launch_interp_m<4>(P, descs, items, n_items_dev, grid, r, par_c, par_f, alpha, st);
  else launch_interp_m<2>(P, descs, items, n_items_dev, grid, r, par_c, par_f, alpha, st);
  return cudaGetLastError();
}

// Ghost fill: the refinement above applied to the ring cells of the patches, one thread per
// coarse cell under a ghost strip; it reconstructs each of its R x R fine cells that lies in
// the strip and in no patch of the fine level. Launched in blocks of 64 threads (four times
// the blocks of the flat grid): a level's list of ring cells often fills only a fraction of
// the GPU, and small blocks spread it over every SM instead of giving some SMs two large
// blocks and others none.
template <int M, int R>
__global__ void __launch_bounds__(256)
ghost_cells_kernel(DevParams P, const LevelDesc* __restrict__ descs, const GhostCell* __restrict__ cells,
                   const int* __restrict__ n_dev, int par_c, int par_f, double alpha_in, int substep) {
  constexpr double inv_r = 1.0 / (double)R;
  const int n = *n_dev;
  const long long tol_bits = __double_as_longlong(P.dry_tol);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const GhostCell g = cells[e];
    const LevelDesc& C = descs[g.desc_c];
    const LevelDesc& Fd = descs[g.desc_f];
    double alpha = alpha_in;
    if (substep >= 0) {
      if (Fd.active != nullptr && *Fd.active == 0) continue;
      alpha = substep_fraction(substep, *Fd.rt);
    }
    const double* qo = C.q[par_c ^ 1];
    const double* qn = C.q[par_c];
    double* qf = Fd.q[par_f];
    const size_t fplane = (size_t)Fd.NY * Fd.P;
    CoarsePrep<M> S;
    coarse_prep<M>(C, qo, qn, alpha, g.ic, g.jc, tol_bits, S);
    // Which of the R x R fine cells take a value: inside the strip and in no patch of the fine
    // level. All R x R mask bytes are loaded before any is used (independent loads in flight
    // together instead of one round trip per fine cell).
    unsigned need = 0;
#pragma unroll
    for (int b = 0; b < R; ++b) {
      const int J = g.jc * R + b;
#pragma unroll
      for (int a = 0; a < R; ++a) {
        const int I = g.ic * R + a;
        const bool strip = I >= g.i0 && I < g.i1 && J >= g.j0 && J < g.j1;
        const uint8_t cov = strip ? Fd.in_patch[(size_t)J * Fd.NX + I] : (uint8_t)1;
        need |= (cov == 0 ? 1u : 0u) << (b * R + a);
      }
    }
    // fine columns a outer: the x parts once per column
#pragma unroll
    for (int a = 0; a < R; ++a) {
      unsigned col = 0;
#pragma unroll
      for (int b = 0; b < R; ++b) col |= ((need >> (b * R + a)) & 1u) << b;
      if (col == 0) continue;
      const int I = g.ic * R + a;
      double ex[M], mx[M][2];
      fine_column<M>(S, (a + 0.5) * inv_r - 0.5, ex, mx);
      // the column's fine bathymetry, all loads issued before the first use
      double Bcol[R];
#pragma unroll
      for (int b = 0; b < R; ++b)
        Bcol[b] = ((col >> b) & 1u) ? Fd.B[(size_t)(g.jc * R + b) * Fd.P + I] : 0.0;
#pragma unroll
      for (int b = 0; b < R; ++b) {
        if (((col >> b) & 1u) == 0) continue;
        fine_cell<M>(S, ex, mx, (b + 0.5) * inv_r - 0.5, Bcol[b], tol_bits, qf, fplane,
                     (size_t)(g.jc * R + b) * Fd.P + I);
      }
    }
  }
}

template <int M>
static void launch_ghost_cells_m(const DevParams& P, const LevelDesc* descs, const GhostCell* cells,
                                 const int* n_dev, int grid, int r, int par_c, int par_f, double alpha,
                                 int substep, cudaStream_t st) {
  if (r == 2)
    ghost_cells_kernel<M, 2><<<4 * grid, 64, 0, st>>>(P, descs, cells, n_dev, par_c, par_f, alpha, substep);
  else
    ghost_cells_kernel<M, 4><<<4 * grid, 64, 0, st>>>(P, descs, cells, n_dev, par_c, par_f, alpha, substep);
}

// r: the level's refinement ratio, 2 or 4 (the only ratios a hierarchy accepts).
cudaError_t launch_ghost_cells(int M, const DevParams& P, const LevelDesc* descs, const GhostCell* cells,
                               const int* n_dev, int grid, int r, int par_c, int par_f, double alpha, int substep,
                               cudaStream_t st) {
  if (r != 2 && r != 4) return cudaErrorInvalidValue;
  if (M == 1) launch_ghost_cells_m<1>(P, descs, cells, n_dev, grid, r, par_c, par_f, alpha, substep, st);
  else if (M == 3) launch_ghost_cells_m<3>(P, descs, cells, n_dev, grid, r, par_c, par_f, alpha, substep, st);
  else if (M == 4) launch_ghost_cells_m<4>(P, descs, cells, n_dev, grid, r, par_c, par_f, alpha, substep, st);
  else launch_ghost_cells_m<2>(P, descs, cells, n_dev, grid, r, par_c, par_f, alpha, substep, st);
  return cudaGetLastError();
}

// Start of substep k of `level` (>= 1) inside a coarse step: a member takes it when its
// parent level's current substep is taken and k < rt of the level.
__global__ void set_active_kernel(int L, int n_members, int level, int k, const int* __restrict__ rt,
                                  int* __restrict__ active) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_members) return;
  const int d = m * L + level;
  active[d] = (active[d - 1] != 0 && k < rt[d]) ? 1 : 0;
}

cudaError_t launch_set_active(int L, int n_members, int level, int k, const int* rt, int* active,
                              cudaStream_t st) {
  set_active_kernel<<<(n_members + 127) / 128, 128, 0, st>>>(L, n_members, level, k, rt, active);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Coarsening, Sec. 2.2, Eq. (11) in 2-D: coarse cells under a fine patch take the
// mean of their r x r fine cells (row-major sum, then times 1/(r r)), every component.
// Items: (desc_c, desc_f, coarse box).
// ---------------------------------------------------------------------------
// RC: the ratio as a compile-time constant (2 or 4; 0: the runtime r), so that the r x r loads
// of a field are unrolled and in flight together; the sum keeps the row-major order.
template <int RC>
__global__ void __launch_bounds__(256)
average_items_kernel(int F, const LevelDesc* __restrict__ descs, const InterpItem* __restrict__ items,
                     const int* __restrict__ n_items_dev, int r_rt, int par_c, int par_f) {
  const int r = RC > 0 ? RC : r_rt;
  const double inv = 1.0 / (double)(r * r);
  const int n_items = *n_items_dev;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const InterpItem item = items[it];
    const LevelDesc& C = descs[item.desc_c];
    const LevelDesc& Fd = descs[item.desc_f];
    if (C.active != nullptr && *C.active == 0) continue;  // the coarse level copied its state through
    const int w = item.i1 - item.i0, h = item.j1 - item.j0;
    const int total = w * h;
    const double* __restrict__ qf = Fd.q[par_f];
    double* __restrict__ qc = C.q[par_c];
    const size_t fplane = (size_t)Fd.NY * Fd.P, cplane = (size_t)C.NY * C.P;
    // one thread per (field, coarse cell): small items still fill the block
    for (int t = threadIdx.x; t < F * total; t += blockDim.x) {
      const int f = t / total, c = t - f * total;
      const int i = item.i0 + c % w, j = item.j0 + c / w;
      {
        const double* __restrict__ src = qf + f * fplane + (size_t)(j * r) * Fd.P + (size_t)i * r;
        double s = 0.0;
        if constexpr (RC > 0) {
          double v[RC * RC];
#pragma unroll
          for (int b = 0; b < RC; ++b)
#pragma unroll
            for (int a = 0; a < RC; ++a) v[b * RC + a] = src[(size_t)b * Fd.P + a];
#pragma unroll
          for (int k = 0; k < RC * RC; ++k) s += v[k];
        } else {
          for (int b = 0; b < r; ++b)
            for (int a = 0; a < r; ++a) s += src[(size_t)b * Fd.P + a];
        }
        qc[f * cplane + (size_t)j * C.P + i] = s * inv;
      }
    }
  }
}

cudaError_t launch_average_items(int F, const LevelDesc* descs, const InterpItem* items, const int* n_items_dev,
                                 int grid, int r, int par_c, int par_f, cudaStream_t st) {
  if (r == 4) average_items_kernel<4><<<grid, 256, 0, st>>>(F, descs, items, n_items_dev, r, par_c, par_f);
  else if (r == 2) average_items_kernel<2><<<grid, 256, 0, st>>>(F, descs, items, n_items_dev, r, par_c, par_f);
  else average_items_kernel<0><<<grid, 256, 0, st>>>(F, descs, items, n_items_dev, r, par_c, par_f);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Refinement flags from the gradient of eta_1 = B + h_M + ... + h_1 (Eq. (4)):
// flag = gx^2 + gy^2 > tol^2, central differences where both neighbours are usable
// (in the domain, in a patch of the level, layer 1 wet), one-sided where only one is.
// Every operation is an explicitly rounded FP64 op (no contraction into FMA), so that
// the flags are bit-identical to a plain sequential evaluation.
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ double eta1_at(const double* q, size_t plane, const double* B, size_t o) {
  double e = B[o];
#pragma unroll
  for (int n = M - 1; n >= 0; --n) e = __dadd_rn(e, q[(3 * n) * plane + o]);
  return e;
}

template <int M>
__global__ void flags_kernel(const LevelDesc* __restrict__ descs, int desc, int par, double dry_tol, double inv_dx,
                             double inv_dy, double tol2, uint8_t* __restrict__ flags) {
  const LevelDesc& D = descs[desc];
  const long long total = (long long)D.NX * D.NY;
  const double* q = D.q[par];
  const size_t plane = (size_t)D.NY * D.P;
  const double hx = __dmul_rn(0.5, inv_dx), hy = __dmul_rn(0.5, inv_dy);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % D.NX), j = (int)(t / D.NX);
    auto usable = [&](int ii, int jj) -> bool {
      if (ii < 0 || jj < 0 || ii >= D.NX || jj >= D.NY) return false;
      if (D.in_patch && !D.in_patch[(size_t)jj * D.NX + ii]) return false;
      return q[(size_t)jj * D.P + ii] > dry_tol;
    };
    uint8_t fl = 0;
    if (usable(i, j)) {
      const size_t o = (size_t)j * D.P + i;
      const double e = eta1_at<M>(q, plane, D.B, o);
      const bool l = usable(i - 1, j), rr = usable(i + 1, j), s = usable(i, j - 1), n = usable(i, j + 1);
      double gx = 0.0, gy = 0.0;
      if (l && rr) gx = __dmul_rn(__dsub_rn(eta1_at<M>(q, plane, D.B, o + 1), eta1_at<M>(q, plane, D.B, o - 1)), hx);
      else if (rr) gx = __dmul_rn(__dsub_rn(eta1_at<M>(q, plane, D.B, o + 1), e), inv_dx);
      else if (l) gx = __dmul_rn(__dsub_rn(e, eta1_at<M>(q, plane, D.B, o - 1)), inv_dx);
      if (s && n) gy = __dmul_rn(__dsub_rn(eta1_at<M>(q, plane, D.B, o + D.P), eta1_at<M>(q, plane, D.B, o - D.P)), hy);
      else if (n) gy = __dmul_rn(__dsub_rn(eta1_at<M>(q, plane, D.B, o + D.P), e), inv_dy);
      else if (s) gy = __dmul_rn(__dsub_rn(e, eta1_at<M>(q, plane, D.B, o - D.P)), inv_dy);
      const double g2 = __dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy));
      fl = g2 > tol2 ? 1 : 0;
    }
    flags[t] = fl;
  }
}

cudaError_t launch_flags(int M, const LevelDesc* descs, int desc, int par, long long cells, double dry_tol,
                         double inv_dx, double inv_dy, double tol2, uint8_t* flags, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((cells + 255) / 256, 4096));
  if (M == 1) flags_kernel<1><<<grid, 256, 0, st>>>(descs, desc, par, dry_tol, inv_dx, inv_dy, tol2, flags);
  else if (M == 3) flags_kernel<3><<<grid, 256, 0, st>>>(descs, desc, par, dry_tol, inv_dx, inv_dy, tol2, flags);
  else if (M == 4) flags_kernel<4><<<grid, 256, 0, st>>>(descs, desc, par, dry_tol, inv_dx, inv_dy, tol2, flags);
  else flags_kernel<2><<<grid, 256, 0, st>>>(descs, desc, par, dry_tol, inv_dx, inv_dy, tol2, flags);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Masks: set mask cells of every box (level indices divided by `div`).
// ---------------------------------------------------------------------------
__global__ void mask_boxes_kernel(uint8_t* __restrict__ mask, int NX, const int* __restrict__ boxes, int n, int div) {
  for (int b = blockIdx.y; b < n; b += gridDim.y) {
    const int i0 = boxes[4 * b] / div, j0 = boxes[4 * b + 1] / div, i1 = boxes[4 * b + 2] / div, j1 = boxes[4 * b + 3] / div;
    const int w = i1 - i0;
    const long long total = (long long)w * (j1 - j0);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
      const int i = i0 + (int)(t % w), j = j0 + (int)(t / w);
      mask[(size_t)j * NX + i] = 1;
    }
  }
}

cudaError_t launch_mask_boxes(uint8_t* mask, int NX, const int* boxes, int n, int div, long long max_cells,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  dim3 grid((unsigned)std::max<long long>(1, std::min<long long>((max_cells + 255) / 256, 256)),
            (unsigned)std::min(n, 65535));
  mask_boxes_kernel<<<grid, 256, 0, st>>>(mask, NX, boxes, n, div);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Mass reflux of a coarse level: for every uncovered cell of the level next to a
// covered one, the coarse mass flux recorded at that edge during the coarse step is
// replaced by the time and space mean of the fine mass fluxes accumulated there:
//   h_C += +-(dt_c F_c - (1/r) sum_k acc_k) / dx_c.
// The consumed fine accumulators are zeroed. Items: (desc_c, desc_f, coarse box to scan).
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(256)
reflux_kernel(const LevelDesc* __restrict__ descs, const InterpItem* __restrict__ cells,
              const int* __restrict__ n_dev, int r, int par_c) {
  // One thread per coarse cell of a patch of the coarse level that is not covered and has a
  // covered face neighbour (the host lists them); it corrects its depths for all such edges.
  // Every read of a thread (coverage of the four neighbours, the coarse fluxes, the r fine
  // fluxes of each covered edge and layer) is issued before any store, so a thread waits for
  // memory about once instead of once per read-then-clear pair; the fine accumulators are
  // cleared afterwards.
  const int n = *n_dev;
  const double inv_r = 1.0 / (double)r;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const InterpItem cell = cells[e];
    const LevelDesc& C = descs[cell.desc_c];
    const LevelDesc& Fd = descs[cell.desc_f];
    if (C.active != nullptr && *C.active == 0) continue;  // no coarse step taken: nothing to correct
    const int i = cell.i0, j = cell.j0;
    const size_t c = (size_t)j * C.NX + i;
    // covered face neighbours: west, east, south, north
    const bool cov[4] = {i > 0 && C.covered[c - 1] != 0, i + 1 < C.NX && C.covered[c + 1] != 0,
                         j > 0 && C.covered[c - C.NX] != 0, j + 1 < C.NY && C.covered[c + C.NX] != 0};
    const double dt_c = *C.dt;
    // first fine flux of each edge (x edges: column I, rows J .. J + r - 1, stride NX_f + 1;
    // y edges: row J, columns I .. I + r - 1, stride 1) and the coarse flux, per layer
    double* fbase[4];
    size_t fstride[4];
    const double* cflux[4];
    size_t cstride[4];
    fbase[0] = Fd.fxf + (size_t)j * r * (Fd.NX + 1) + (size_t)i * r;
    fbase[1] = Fd.fxf + (size_t)j * r * (Fd.NX + 1) + (size_t)(i + 1) * r;
    fbase[2] = Fd.fyf + (size_t)j * r * Fd.NX + (size_t)i * r;
    fbase[3] = Fd.fyf + (size_t)(j + 1) * r * Fd.NX + (size_t)i * r;
    fstride[0] = fstride[1] = (size_t)Fd.NX + 1;
    fstride[2] = fstride[3] = 1;
    const size_t fxplane = (size_t)Fd.NY * (Fd.NX + 1), fyplane = (size_t)(Fd.NY + 1) * Fd.NX;
    cflux[0] = C.fxc + (size_t)j * (C.NX + 1) + i;
    cflux[1] = C.fxc + (size_t)j * (C.NX + 1) + i + 1;
    cflux[2] = C.fyc + (size_t)j * C.NX + i;
    cflux[3] = C.fyc + (size_t)(j + 1) * C.NX + i;
    cstride[0] = cstride[1] = (size_t)C.NY * (C.NX + 1);
    cstride[2] = cstride[3] = (size_t)(C.NY + 1) * C.NX;
    double fine[4][M], coarse[4][M];
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
      for (int m = 0; m < M; ++m) {
        fine[d][m] = 0.0;
        coarse[d][m] = 0.0;
        if (cov[d]) {
          const double* fp = fbase[d] + (size_t)m * (d < 2 ? fxplane : fyplane);
          double sum = 0.0;
#pragma unroll 4
          for (int k = 0; k < r; ++k) sum += fp[k * fstride[d]];
          fine[d][m] = sum;
          coarse[d][m] = cflux[d][m * cstride[d]];
        }
      }
    double dh[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      // west / south: this cell on the right of the edge, h -= corr; east / north: h += corr
      dh[m] = 0.0;
      if (cov[0]) dh[m] -= (dt_c * coarse[0][m] - fine[0][m] * inv_r) * C.inv_dx;
      if (cov[1]) dh[m] += (dt_c * coarse[1][m] - fine[1][m] * inv_r) * C.inv_dx;
      if (cov[2]) dh[m] -= (dt_c * coarse[2][m] - fine[2][m] * inv_r) * C.inv_dy;
      if (cov[3]) dh[m] += (dt_c * coarse[3][m] - fine[3][m] * inv_r) * C.inv_dy;
    }
    double* qc = C.q[par_c];
    const size_t cplane = (size_t)C.NY * C.P;
#pragma unroll
    for (int m = 0; m < M; ++m)
      if (dh[m] != 0.0) qc[(3 * m) * cplane + (size_t)j * C.P + i] += dh[m];
#pragma unroll
    for (int d = 0; d < 4; ++d)
      if (cov[d])
#pragma unroll
        for (int m = 0; m < M; ++m) {
          double* fp = fbase[d] + (size_t)m * (d < 2 ? fxplane : fyplane);
#pragma unroll 4
          for (int k = 0; k < r; ++k) fp[k * fstride[d]] = 0.0;
        }
  }
}

cudaError_t launch_reflux(int M, const LevelDesc* descs, const InterpItem* cells, const int* n_dev, int grid,
                          int r, int par_c, cudaStream_t st) {
  if (M == 1) reflux_kernel<1><<<grid, 256, 0, st>>>(descs, cells, n_dev, r, par_c);
  else if (M == 3) reflux_kernel<3><<<grid, 256, 0, st>>>(descs, cells, n_dev, r, par_c);
  else if (M == 4) reflux_kernel<4><<<grid, 256, 0, st>>>(descs, cells, n_dev, r, par_c);
  else reflux_kernel<2><<<grid, 256, 0, st>>>(descs, cells, n_dev, r, par_c);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Wave speed of the state of every (member, level) before its first step:
// max over patch cells of max_m max(|u_m|, |v_m|) + sqrt(g sum_m h_m).
// Items: (desc, -, box); the level's parity of each desc in par_of_desc.
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(256)
speed_kernel(DevParams P, const LevelDesc* __restrict__ descs, const InterpItem* __restrict__ items,
             const int* __restrict__ n_items_dev, const int* __restrict__ par_of_desc,
             unsigned long long* __restrict__ out) {
  const int n_items = *n_items_dev;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const InterpItem item = items[it];
    const LevelDesc& D = descs[item.desc_c];
    const int w = item.i1 - item.i0, h = item.j1 - item.j0;
    const int total = w * h;
    const double* q = D.q[par_of_desc[item.desc_c]];
    const size_t plane = (size_t)D.NY * D.P;
    double best = 0.0;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int i = item.i0 + t % w, j = item.j0 + t / w;
      const size_t o = (size_t)j * D.P + i;
      double htot = 0.0, umax = 0.0;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const double hm = q[(3 * m) * plane + o];
        htot += hm;
        if (hm > P.dry_tol) {
          const double u = fabs(q[(3 * m + 1) * plane + o]) / hm, v = fabs(q[(3 * m + 2) * plane + o]) / hm;
          umax = fmax(umax, fmax(u, v));
        }
      }
      best = fmax(best, umax + sqrt(P.g * fmax(htot, 0.0)));
    }
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&out[item.desc_c], (unsigned long long)__double_as_longlong(best));
  }
}

cudaError_t launch_speed(int M, const DevParams& P, const LevelDesc* descs, const InterpItem* items,
                         const int* n_items_dev, int grid, const int* par_of_desc, unsigned long long* out,
                         cudaStream_t st) {
  if (M == 1) speed_kernel<1><<<grid, 256, 0, st>>>(P, descs, items, n_items_dev, par_of_desc, out);
  else if (M == 3) speed_kernel<3><<<grid, 256, 0, st>>>(P, descs, items, n_items_dev, par_of_desc, out);
  else if (M == 4) speed_kernel<4><<<grid, 256, 0, st>>>(P, descs, items, n_items_dev, par_of_desc, out);
  else speed_kernel<2><<<grid, 256, 0, st>>>(P, descs, items, n_items_dev, par_of_desc, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Device-side time step, one thread per member, at the start of every coarse step.
// From the largest wave speeds of the previous coarse step (smax bits [desc][x, y])
// or, right after the state was set, from the speeds of the state (init_bits [desc],
// selected by *init_flag, which is then cleared):
//   rate_l = max(sx/dx_l, sy/dy_l)        (state speeds: s * max(1/dx_l, 1/dy_l))
//   dt_0   = cfl * min_l (prod_{k<l} r_k) / rate_l   over levels that have patches now,
//   dt_l   = dt_0 / prod_{k<l} r_k.
// The speed slots are then cleared for the step.
// ---------------------------------------------------------------------------
__global__ void dt_begin_kernel(DtArgs A, unsigned long long* smax_bits, const unsigned long long* init_bits,
                                int* init_flag, double* dt) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const bool initial = *init_flag != 0;
  // A member that sits the round out (its coarse steps are all kept) keeps its time step,
  // wave speeds and counters untouched.
  if (m < A.n_members && A.active[m * A.L] != 0) {
    double best = INFINITY, fac = 1.0;
    double rate[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = 0; l < A.L; ++l) {
      if (l > 0) fac *= A.ratio[l - 1];
      const int d = m * A.L + l;
      if (!A.has_patches[d]) continue;
      if (initial) {
        const double s = __longlong_as_double((long long)init_bits[d]);
        rate[l] = s * fmax(A.inv_dx[d], A.inv_dy[d]);
      } else {
        const double sx = __longlong_as_double((long long)smax_bits[2 * d]);
        const double sy = __longlong_as_double((long long)smax_bits[2 * d + 1]);
        rate[l] = fmax(sx * A.inv_dx[d], sy * A.inv_dy[d]);
      }
      if (rate[l] > 0.0) best = fmin(best, fac / rate[l]);
    }
    const double dt0 = isfinite(best) ? A.cfl * best : 0.0;
    // Time ratio of every level: the fixed r, or (dynamic) the fewest steps of the level per
    // parent step that keep its Courant number at cfl: ceil(dt_parent rate / cfl), in [1, r].
    double dl = dt0;
    long long steps = 1;
    for (int l = 0; l < A.L; ++l) {
      const int d = m * A.L + l;
      int rt = 1;
      if (l > 0) {
        rt = A.ratio[l - 1];
        if (A.dynamic_rt && *A.fresh == 0 && rate[l] > 0.0) {
          const double need = ceil((dl * rate[l]) / A.cfl);
          rt = need < 1.0 ? 1 : (need < (double)rt ? (int)need : rt);
        }
        dl = dl / rt;
      }
      steps *= rt;
      A.rt[d] = rt;
      dt[d] = dl;
      A.steps_acc[d] += steps;
      A.cells_acc[d] += steps * A.cells[d];
      smax_bits[2 * d] = 0ull;
      smax_bits[2 * d + 1] = 0ull;
    }
  }
}

// End of a coarse-step attempt: Courant number reached by every member, the largest over
// its levels of dt_l max(sx/dx_l, sy/dy_l). Above cfl_max the attempt is rejected (Sec. 2:
// the time refinement exists to keep each level's Courant number below one): redo is set,
// the member's time does not advance, and the snapshot kernel that follows restores its
// state; the next round retakes the step with the time step dt_begin derives from the speeds
// this attempt measured. Status bit 1 when a wave speed was not finite.
__global__ void step_end_kernel(DtArgs A, const unsigned long long* smax_bits, const double* dt, double* t_member,
                                double* cfl_reached, unsigned int* status, unsigned long long* cfl_count) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m == 0) *A.fresh = 0;
  if (m >= A.n_members) return;
  const bool took = A.active[m * A.L] != 0;
  for (int l = 1; l < A.L; ++l) A.active[m * A.L + l] = 1;  // steps outside advance take every level
  if (!took) {
    A.redo[m] = 0;
    return;
  }
  double reached = 0.0;
  bool bad = false;
  for (int l = 0; l < A.L; ++l) {
    const int d = m * A.L + l;
    const double sx = __longlong_as_double((long long)smax_bits[2 * d]);
    const double sy = __longlong_as_double((long long)smax_bits[2 * d + 1]);
    if (!(sx >= 0.0) || !(sy >= 0.0)) bad = true;
    reached = fmax(reached, dt[d] * fmax(sx * A.inv_dx[d], sy * A.inv_dy[d]));
  }
  cfl_reached[m] = reached;
  if (bad) atomicOr(status, 2u);
  if (reached > A.cfl_max) {
    A.redo[m] = 1;
    atomicAdd(cfl_count, 1ull);
    return;
  }
  A.redo[m] = 0;
  A.done[m] += 1;
  t_member[m] += dt[m * A.L];
}

// Courant control (see launch_snapshot): one block per patch chunk, F fields of its cells.
__global__ void __launch_bounds__(256)
snapshot_kernel(int F, int L, const LevelDesc* __restrict__ descs, const InterpItem* __restrict__ items,
                const int* __restrict__ n_items_dev, int mode, ParSet par, const int* __restrict__ redo) {
  const int n_items = *n_items_dev;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const InterpItem item = items[it];
    const int d = item.desc_c, l = d % L, m = d / L;
    const LevelDesc& D = descs[d];
    const double* __restrict__ src;
    double* __restrict__ dst;
    if (mode == 0) {
      if (l == 0) continue;  // level 0 keeps its state before the step in its other buffer
      src = D.q[par.start[l]];
      dst = D.snap;
    } else {
      if (redo[m] == 0) continue;
      src = l == 0 ? D.q[par.start[0]] : D.snap;
      dst = D.q[par.next[l]];
    }
    const int w = item.i1 - item.i0, n = w * (item.j1 - item.j0);
    const size_t plane = (size_t)D.NY * D.P;
    for (int t = threadIdx.x; t < n * F; t += blockDim.x) {
      const int f = t / n, c = t - f * n, j = c / w, i = c - j * w;
      const size_t o = (size_t)f * plane + (size_t)(item.j0 + j) * D.P + (item.i0 + i);
      dst[o] = src[o];
    }
  }
}

cudaError_t launch_snapshot(int F, int L, const LevelDesc* descs, const InterpItem* items, const int* n_items_dev,
                            int grid, int mode, const ParSet& par, const int* redo, cudaStream_t st) {
  snapshot_kernel<<<grid, 256, 0, st>>>(F, L, descs, items, n_items_dev, mode, par, redo);
  return cudaGetLastError();
}

cudaError_t launch_dt_begin(const DtArgs& A, unsigned long long* smax_bits, const unsigned long long* init_bits,
                            int* init_flag, double* dt, cudaStream_t st) {
  // one thread per member; the flag is cleared after the kernel, in stream order
  dt_begin_kernel<<<(A.n_members + 255) / 256, 256, 0, st>>>(A, smax_bits, init_bits, init_flag, dt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(init_flag, 0, sizeof(int), st);
}

cudaError_t launch_step_end(const DtArgs& A, const unsigned long long* smax_bits, const double* dt, double* t_member,
                            double* cfl_reached, unsigned int* status, unsigned long long* cfl_count,
                            cudaStream_t st) {
  step_end_kernel<<<(A.n_members + 127) / 128, 128, 0, st>>>(A, smax_bits, dt, t_member, cfl_reached, status,
                                                              cfl_count);
  return cudaGetLastError();
}

}  // namespace mlswe
