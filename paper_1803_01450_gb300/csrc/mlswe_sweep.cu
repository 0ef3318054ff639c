// Dimensionally split finite-volume sweeps over tiles of patches.
//
// One sweep (x or y) of the step: for every edge of a line, the Riemann solve
// of mlswe_device.cuh, then first-order fluctuations plus the second-order
// wave correction (MC-limited, upwind neighbour of each wave family), then the
// update of every cell of the line and the positivity fix
//   Q_i <- Q_i - (dt/dx) (A+dQ_{i-1/2} + A-dQ_{i+1/2}) - (dt/dx)(F_{i+1/2} - F_{i-1/2}).
// The x sweep writes Q* for the patch rows (and, on refined levels, the two
// ghost rows on each side); the y sweep reads Q* and writes Q^{n+1}.
//
// Layout of one work tile in shared memory: a cell record of Rec<M>::N doubles
// per cell (structure of arrays), then the compressed waves of every edge,
// then (reusing the wave space) the left/right cell contributions of every
// edge. Every thread owns one edge; no CTA ever waits on another.
#include <cuda_runtime.h>
#include "mlswe_device.cuh"

namespace mlswe {

template <int DIR>
__device__ __forceinline__ int cslot(int l, int k, int len, int nl) {
  return DIR == 0 ? l * (len + 4) + k : k * nl + l;
}
template <int DIR>
__device__ __forceinline__ int eslot(int l, int e, int len, int nl) {
  return DIR == 0 ? l * (len + 3) + e : e * nl + l;
}
template <int DIR>
__device__ __forceinline__ int gslot(int l, int e, int len, int nl) {
  return DIR == 0 ? l * (len + 1) + e : e * nl + l;
}

// Shared memory of the split layout in doubles: cell records, edge records, wall and wet
// bytes (rounded up to whole doubles).
__host__ __device__ constexpr size_t sweep_smem_doubles(int M) {
  return (size_t)(7 * M + 1) * kMaxCells + (size_t)(2 * M * M + 7 * M) * kMaxEdges +
         ((size_t)kMaxEdges * 4 + kMaxCells + 7) / 8;
}

// Largest |s| of a warp folded into the tile's shared maximum (no barrier of its own: the
// phase barrier that follows orders it before thread 0 reads the tile's maximum). v holds |s|
// as a bit pattern with the sign cleared, so non-negative doubles order like their unsigned
// 64-bit patterns and a NaN (exponent all ones, mantissa not zero) lies above +inf: reducing
// the patterns with an integer max keeps a non-finite speed visible to the host (fmax would
// drop it).
__device__ __forceinline__ void warp_max_to_shared(double v, unsigned long long* tile_max) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  for (int o = 16; o > 0; o >>= 1) b = umax64(b, __shfl_xor_sync(0xffffffffu, b, o));
  if ((threadIdx.x & 31) == 0) atomicMax(tile_max, b);
}

// MINB: CTAs resident per SM the build targets (1: up to 255 registers per thread; 2: at
// most 128, 16 warps per SM to hide FP64 latency). The autotuner picks per level.
// STORE (M = 2, for the adjoint's recomputation): every coupled edge between the cells of a
// tile and their first neighbours also writes its FwdRec record to est, one plane of
// eplane doubles per field, at the edge's index on the level (x edges: j (NX + 1) + i for
// the edge left of cell i; y edges: j NX + i for the edge below cell j); the other coupled
// edges of the tile write to slot eplane - 1, which eplane > (NX + 1) (NY + 1) keeps spare.
// UNSPLIT (M <= 2): the edge pass of the unsplit step. Both directions read Q^n; tiles also
// cover one ghost line on each side of a patch (mirrored beyond the domain); every edge
// between the cells of a tile line writes the fluctuations its two cells receive and their
// transverse splits to the level's edge arrays (LevelDesc::ue) instead of updating cells.
template <int M, int DIR, int MINB, bool STORE, bool UNSPLIT>
__global__ void __launch_bounds__(kThreads, MINB)
sweep_kernel(DevParams P, const LevelDesc* __restrict__ descs, const SweepItem* __restrict__ items,
             const int* __restrict__ n_tiles_dev, const int* __restrict__ tile_off, int parity, int record,
             unsigned long long* smax_bits, unsigned int* lost_count, double* __restrict__ est, long long eplane) {
  using R = Rec<M>;
  using WR = WRec<M>;
  constexpr int F = 3 * M;
  extern __shared__ double smem[];
  double* cell = smem;                                  // [R::N][kMaxCells]
  double* wav = cell + R::N * kMaxCells;                // [WR::N][kMaxEdges], reused for contributions
  int* wallb = reinterpret_cast<int*>(wav + WR::N * kMaxEdges);   // [kMaxEdges]
  unsigned char* wetb = reinterpret_cast<unsigned char*>(wallb + kMaxEdges);  // [kMaxCells]
  // unsplit only: transverse depth of every edge [M][kMaxEdges], after the split layout, and
  // (M >= 3) the eigenvalues of the coupling matrix [M][kMaxEdges]
  double* hbw = reinterpret_cast<double*>(smem) + sweep_smem_doubles(M);
  double* muw = hbw + M * kMaxEdges;
  __shared__ unsigned long long s_smax;  // largest |s| of the tile (bit pattern)
  // The tile's groups (items tile_off[it] .. tile_off[it + 1], or item it alone), all of one
  // (member, level), and their running counts of cells, edges, cell contributions and updates.
  __shared__ SweepItem sg[kMaxGroups];
  __shared__ int sb[4][kMaxGroups + 1];
  __shared__ int sng, s_rec;

  const int n_tiles = *n_tiles_dev;
  for (int it = blockIdx.x; it < n_tiles; it += gridDim.x) {
    if (threadIdx.x == 0) {
      const int g0 = tile_off ? tile_off[it] : it, g1 = tile_off ? tile_off[it + 1] : it + 1;
      int c = 0, e = 0, gc = 0, u = 0, rc = 0;
      for (int g = 0; g < g1 - g0; ++g) {
        const SweepItem x = items[g0 + g];
        sg[g] = x;
        sb[0][g] = c; sb[1][g] = e; sb[2][g] = gc; sb[3][g] = u;
        c += x.nlines * (x.len + 4); e += x.nlines * (x.len + 3); gc += x.nlines * (x.len + 1);
        u += x.nlines * x.len;
        rc |= x.flags & 1;
      }
      sng = g1 - g0;
      sb[0][g1 - g0] = c; sb[1][g1 - g0] = e; sb[2][g1 - g0] = gc; sb[3][g1 - g0] = u;
      s_rec = rc;
      s_smax = 0ull;
    }
    __syncthreads();
    const int ngrp = sng;
    // group of flat index t in the running counts k (0 cells, 1 edges, 2 contributions, 3 updates)
    auto group_of = [&](int k, int t) {
      int g = 0;
#pragma unroll
      for (int h = 1; h < kMaxGroups; ++h) g += (h < ngrp && t >= sb[k][h]) ? 1 : 0;
      return g;
    };
    const LevelDesc& D = descs[sg[0].desc];
    const int NX = D.NX, NY = D.NY, Pt = D.P;
    const size_t plane = (size_t)NY * Pt;
    const double* __restrict__ qin = (DIR == 0 || UNSPLIT) ? D.q[parity] : D.qs;
    double* __restrict__ qout = DIR == 0 ? D.qs : D.q[parity ^ 1];
    if (D.active != nullptr && *D.active == 0) {
      // This member's level takes no step in this substep (its time ratio is smaller than
      // the substep count of the launch): the y sweep copies the tile's cells from the step's
      // input to its output (the x sweep's scratch is skipped), nothing is recorded. (Unsplit:
      // the update kernel copies.)
      if (DIR == 0 || UNSPLIT) {
        __syncthreads();  // the group table is rewritten for the next tile
        continue;
      }
      const double* __restrict__ qsrc = D.q[parity];
      const int ncp = sb[3][ngrp];
      for (int t = threadIdx.x; t < ncp; t += blockDim.x) {
        const int g = group_of(3, t);
        const SweepItem& item = sg[g];
        const int len = item.len, nl = item.nlines, tt = t - sb[3][g];
        int l, k;
        if (DIR == 0) { l = tt / len; k = tt - l * len; }
        else { k = tt / nl; l = tt - k * nl; }
        const size_t o = DIR == 0 ? (size_t)(item.j0 + l) * Pt + (item.i0 + k) : (size_t)(item.j0 + k) * Pt + (item.i0 + l);
#pragma unroll
        for (int f = 0; f < F; ++f) qout[f * plane + o] = qsrc[f * plane + o];
      }
      __syncthreads();
      continue;
    }
    const double dt = *D.dt;
    const double nu = dt * (DIR == 0 ? D.inv_dx : D.inv_dy);
    const long long tol_bits = __double_as_longlong(P.dry_tol);

    // ---- phase 1: load cells (mirror at walls) and compute the per-cell record ----
    const int ncell = sb[0][ngrp];
    for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
      const int g = group_of(0, t);
      const SweepItem& item = sg[g];
      const int len = item.len, nl = item.nlines, tt = t - sb[0][g];
      int l, k;
      if (DIR == 0) { l = tt / (len + 4); k = tt - l * (len + 4); }
      else { k = tt / nl; l = tt - k * nl; }
      int i, j;
      if (DIR == 0) { i = item.i0 - kNG + k; j = item.j0 + l; }
      else { i = item.i0 + l; j = item.j0 - kNG + k; }
      // wall mirror: the momentum normal to the wall changes sign (sign-bit masks, applied on
      // the integer unit)
      long long sgn = 0, sgt = 0;
      constexpr long long kSign = (long long)0x8000000000000000ull;
      if (DIR == 0) {
        if (i < 0) { i = -1 - i; sgn = kSign; }
        else if (i >= NX) { i = 2 * NX - 1 - i; sgn = kSign; }
        if (UNSPLIT) {  // ghost rows beyond the domain: wall mirror
          if (j < 0) { j = -1 - j; sgt = kSign; }
          else if (j >= NY) { j = 2 * NY - 1 - j; sgt = kSign; }
        }
      } else {
        if (j < 0) { j = -1 - j; sgn = kSign; }
        else if (j >= NY) { j = 2 * NY - 1 - j; sgn = kSign; }
        if (UNSPLIT) {
          if (i < 0) { i = -1 - i; sgt = kSign; }
          else if (i >= NX) { i = 2 * NX - 1 - i; sgt = kSign; }
        }
      }
      auto flip = [](double v, long long mask) { return __longlong_as_double(__double_as_longlong(v) ^ mask); };
      const size_t o = (size_t)j * Pt + i;
      const int c = sb[0][g] + cslot<DIR>(l, k, len, nl);
      double rec[R::N];
      const double Bv = D.B[o];
      rec[R::BB] = Bv;
      int wet = 0;
      bool above = true;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const double h = qin[(3 * m) * plane + o];
        const double hu = qin[(3 * m + 1) * plane + o];
        const double hv = qin[(3 * m + 2) * plane + o];
        const double hn = flip(DIR == 0 ? hu : hv, sgn);
        const double ht = UNSPLIT ? flip(DIR == 0 ? hv : hu, sgt) : (DIR == 0 ? hv : hu);
        rec[3 * m] = h; rec[3 * m + 1] = hn; rec[3 * m + 2] = ht;
        // comparisons on bit patterns (integer unit): for a bound b >= +0 and any non-NaN
        // x, x > b exactly when bits(x) > bits(b) as signed 64-bit integers
        const long long hbits = __double_as_longlong(h);
        const bool w = above && (hbits > tol_bits);
        above = w;
        wet |= w ? (1 << m) : 0;
        // one reciprocal square root gives sqrt(h) = h t and sqrt(h) u = hn t, sqrt(h) v = ht t
        const double t = hbits > 0 ? rsqrt_fast(h) : 0.0;
        double un = 0.0, ut = 0.0;
        if (w) { un = hn * t; ut = ht * t; }
        rec[R::UN + 2 * m] = un; rec[R::UN + 2 * m + 1] = ut;
        rec[R::SQ + m] = h * t;
      }
      double acc = Bv;
#pragma unroll
      for (int m = M - 1; m >= 0; --m) { acc = acc + rec[3 * m]; rec[R::ETA + m] = acc; }
#pragma unroll
      for (int f = 0; f < R::N; ++f) cell[f * kMaxCells + c] = rec[f];
      wetb[c] = (unsigned char)wet;
    }
    __syncthreads();

    // ---- phase 2: Riemann solve at every edge of the tile ----
    const int nedge = sb[1][ngrp];
    double smax = 0.0;
    int lost = 0;
    for (int t = threadIdx.x; t < nedge; t += blockDim.x) {
      const int g = group_of(1, t);
      const SweepItem& item = sg[g];
      const int len = item.len, nl = item.nlines, tt = t - sb[1][g];
      // interior lines of a recorded step count toward the CFL reduction and the reflux fluxes
      const bool interior = (item.flags & 1) && record;
      int l, e;
      if (DIR == 0) { l = tt / (len + 3); e = tt - l * (len + 3); }
      else { e = tt / nl; l = tt - e * nl; }
      const int cl = sb[0][g] + cslot<DIR>(l, e, len, nl), cr = sb[0][g] + cslot<DIR>(l, e + 1, len, nl);
      const SmemRec cL{cell + cl}, cR{cell + cr};
      EdgeW<M> W;
      int lst = 0;
      // halo edges write their record to the spare last slot of each plane
      double* st = nullptr;
      if (STORE) {
        st = est + (eplane - 1);
        if (e >= 1 && e <= len + 1)
          st = DIR == 0 ? est + (size_t)(item.j0 + l) * (NX + 1) + (item.i0 - 1 + e)
                        : est + (size_t)(item.j0 - 1 + e) * NX + (item.i0 + l);
      }
      solve_edge<M, STORE, SmemRec>(P, cL, cR, wetb[cl], wetb[cr], W, lst, st, eplane);
      const int es = sb[1][g] + eslot<DIR>(l, e, len, nl);
#pragma unroll
      for (int p = 0; p < 2 * M; ++p) {
#pragma unroll
        for (int m = 0; m < M; ++m) wav[(WR::A + 2 * M * m + p) * kMaxEdges + es] = W.mass[m][p];
        wav[(WR::S + p) * kMaxEdges + es] = W.s[p];
      }
#pragma unroll
      for (int m = 0; m < M; ++m) {
        wav[(WR::Z + m) * kMaxEdges + es] = W.z[m];
        wav[(WR::US + m) * kMaxEdges + es] = W.us[m];
        wav[(WR::VH + m) * kMaxEdges + es] = W.vh[m];
        wav[(WR::T0 + m) * kMaxEdges + es] = W.t0[m];
        wav[(WR::T1 + m) * kMaxEdges + es] = W.t1[m];
      }
      wallb[es] = W.wall;
      if (UNSPLIT) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
          hbw[m * kMaxEdges + es] = W.hbt[m];
          if (M >= 3) muw[m * kMaxEdges + es] = W.muk[m];
        }
      }
      if (interior && e >= 1 && e <= len + 1) {
        // |s| as bit patterns: non-negative doubles order like unsigned integers (NaN above all)
        unsigned long long sm = __double_as_longlong(smax);
#pragma unroll
        for (int p = 0; p < 2 * M; ++p) sm = umax64(sm, abs_bits(W.s[p]));
#pragma unroll
        for (int m = 0; m < M; ++m) sm = umax64(sm, abs_bits(W.us[m]));
        smax = __longlong_as_double((long long)sm);
        // each edge counted once: the edge after the tile's last cell belongs to the next
        // tile unless the tile ends the patch line (flag bit 1)
        if (e <= len || (item.flags & 2)) lost += lst;
      }
    }
    if (record && s_rec) warp_max_to_shared(smax, &s_smax);
    __syncthreads();

    // ---- phase 3: fluctuations + limited correction -> left/right cell contributions ----
    const int ng = sb[2][ngrp];
    double Lc[F], Rc[F];
    int gl = -1, ge = -1, gg = 0;
    if (threadIdx.x < ng) {
      const int t = threadIdx.x;
      const int g = group_of(2, t);
      const SweepItem& item = sg[g];
      const int len = item.len, nl = item.nlines, tt = t - sb[2][g];
      int l, e1;
      if (DIR == 0) { l = tt / (len + 1); e1 = tt - l * (len + 1); }
      else { e1 = tt / nl; l = tt - e1 * nl; }
      gl = l; ge = e1; gg = g;
      const int e = e1 + 1;
      const int es = sb[1][g] + eslot<DIR>(l, e, len, nl);
      const int esl = sb[1][g] + eslot<DIR>(l, e - 1, len, nl), esr = sb[1][g] + eslot<DIR>(l, e + 1, len, nl);
      const int wall = wallb[es];
      double vh[M];
#pragma unroll
      for (int m = 0; m < M; ++m) vh[m] = wav[(WR::VH + m) * kMaxEdges + es];
      // Left-going parts L (A-dQ minus the correction flux); the right-going parts follow as
      // R = T - L, since the waves of a layer sum to its flux jump T (mass, normal momentum)
      // and the transverse row to vh T_mass + z.
      double Lm[M], Lsm[M];
      // Wave limiter: theta_p = zu_p / zz_p for the acoustic waves and zu_m / z_m for the shear
      // waves ((z_up z)/(z z) with z != 0), with one reciprocal for all of them.
      constexpr int NA = 2 * M, NR = 2 * M + M;
      double den[NR], num[NR];
      int sc[NR];
      bool act[NR];
#pragma unroll
      for (int p = 0; p < NA; ++p) {
        double mp[M];
#pragma unroll
        for (int m = 0; m < M; ++m) mp[m] = wav[(WR::A + NA * m + p) * kMaxEdges + es];
        const double s = wav[(WR::S + p) * kMaxEdges + es];
        sc[p] = sign_class(s);
        const int lay = layer_of_slot<M>(p);
        const bool walled = (wall >> (2 * lay)) & 3;
        act[p] = P.order >= 2 && sc[p] != 0 && !walled;
        den[p] = 1.0;
        num[p] = 0.0;
        if (act[p]) {
          const int eu = sc[p] > 0 ? esl : esr;
          const double su = wav[(WR::S + p) * kMaxEdges + eu];
          const double ss = 1.0 + s * s, su1 = 1.0 + s * su;
          // Z_p . Z_p and Z_up . Z_p, layer by layer
          double zz = 0.0, zu = 0.0;
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const double mu_m = wav[(WR::A + NA * m + p) * kMaxEdges + eu];
            const double vu = wav[(WR::VH + m) * kMaxEdges + eu];
            if (m == 0) {
              zz = mp[0] * mp[0] * (ss + vh[0] * vh[0]);
              zu = mp[0] * mu_m * (su1 + vh[0] * vu);
            } else {
              zz += mp[m] * mp[m] * (ss + vh[m] * vh[m]);
              zu += mp[m] * mu_m * (su1 + vh[m] * vu);
            }
          }
          if (__double_as_longlong(zz) > 0) { den[p] = zz; num[p] = zu; }
          else act[p] = false;
        }
      }
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const double z = wav[(WR::Z + m) * kMaxEdges + es];
        const double us = wav[(WR::US + m) * kMaxEdges + es];
        const bool walled = (wall >> (2 * m)) & 3;
        const int q = NA + m;
        sc[q] = sign_class(us);
        act[q] = P.order >= 2 && sc[q] != 0 && !walled && ((__double_as_longlong(z) << 1) != 0);
        den[q] = 1.0;
        num[q] = 0.0;
        if (act[q]) {
          den[q] = z;
          num[q] = wav[(WR::Z + m) * kMaxEdges + (sc[q] > 0 ? esl : esr)];
        }
      }
      double iden[NR];
      reciprocal2_group<NR>(den, iden);  // limiter ratios: second-order reciprocals suffice
#pragma unroll
      for (int p = 0; p < NA; ++p) {
        const double s = wav[(WR::S + p) * kMaxEdges + es];
        const double cl = left_share(P.limiter, sc[p], act[p], num[p], iden[p], s, nu);
        const double cs = cl * s;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const double a = wav[(WR::A + NA * m + p) * kMaxEdges + es];
          if (p == 0) { Lm[m] = cl * a; Lsm[m] = cs * a; }
          else { Lm[m] = fma(cl, a, Lm[m]); Lsm[m] = fma(cs, a, Lsm[m]); }
        }
      }
      double Lz[M], Rz[M];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int q = NA + m;
        const double z = wav[(WR::Z + m) * kMaxEdges + es];
        const double us = wav[(WR::US + m) * kMaxEdges + es];
        const double cl = left_share(P.limiter, sc[q], act[q], num[q], iden[q], us, nu);
        Lz[m] = cl * z;
        Rz[m] = z - Lz[m];
      }
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const double T0 = wav[(WR::T0 + m) * kMaxEdges + es], T1 = wav[(WR::T1 + m) * kMaxEdges + es];
        Lc[3 * m] = Lm[m]; Lc[3 * m + 1] = Lsm[m]; Lc[3 * m + 2] = vh[m] * Lm[m] + Lz[m];
        Rc[3 * m] = T0 - Lm[m]; Rc[3 * m + 1] = T1 - Lsm[m]; Rc[3 * m + 2] = vh[m] * Rc[3 * m] + Rz[m];
      }
#pragma unroll
      for (int m = 0; m < M; ++m) {
        if ((wall >> (2 * m)) & 1) { Lc[3 * m] = 0.0; Lc[3 * m + 1] = 0.0; Lc[3 * m + 2] = 0.0; }
        if ((wall >> (2 * m + 1)) & 1) { Rc[3 * m] = 0.0; Rc[3 * m + 1] = 0.0; Rc[3 * m + 2] = 0.0; }
      }
      if constexpr (UNSPLIT) {
        // transverse split of what each cell receives, at this edge's state
        const int wL = wetb[sb[0][g] + cslot<DIR>(l, e, len, nl)], wR = wetb[sb[0][g] + cslot<DIR>(l, e + 1, len, nl)];
        double hbt[M], un[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          hbt[m] = hbw[m * kMaxEdges + es];
          un[m] = wav[(WR::US + m) * kMaxEdges + es];
        }
        const int full = (1 << M) - 1;
        const long long pl = DIR == 0 ? D.uxp : D.uyp;
        const int line = (DIR == 0 ? item.j0 : item.i0) + l;
        const int a = (DIR == 0 ? item.i0 : item.j0) + e1;
        double* __restrict__ base = D.ue + (DIR == 0 ? 0 : 6LL * F * D.uxp) +
                                    (DIR == 0 ? (long long)(line + 1) * (NX + 1) + a
                                              : (long long)a * (NX + 2) + (line + 1));
        // field f of the normal frame -> plane of the (h, hu, hv) order
        auto put = [&](int grp, const double* v) {
#pragma unroll
          for (int m = 0; m < M; ++m) {
            base[(grp * F + 3 * m) * pl] = v[3 * m];
            base[(grp * F + 3 * m + (DIR == 0 ? 1 : 2)) * pl] = v[3 * m + 1];
            base[(grp * F + 3 * m + (DIR == 0 ? 2 : 1)) * pl] = v[3 * m + 2];
          }
        };
        put(0, Lc);
        put(1, Rc);
        double up[F], dn[F];
        if constexpr (M >= 3) {
          if (wL == full && wR == full) {
            double muk[M], up2[F], dn2[F];
#pragma unroll
            for (int m = 0; m < M; ++m) muk[m] = muw[m * kMaxEdges + es];
            trans_apply_general<M>(P, hbt, un, vh, muk, Lc, Rc, up, dn, up2, dn2);
            put(2, up);
            put(3, dn);
            put(4, up2);
            put(5, dn2);
          }
        }
        if (M == 2 && wL == full && wR == full) {
          TransEig2 E;
          trans_eigen2(P, hbt, vh, E);
          trans_apply2(E, un, vh, Lc, up, dn);
          put(2, up);
          put(3, dn);
          trans_apply2(E, un, vh, Rc, up, dn);
          put(4, up);
          put(5, dn);
        } else if (M == 1 || wL != full || wR != full) {
          const int act = wL | wR;
          trans_apply_layers<M>(P, act, hbt, un, vh, Lc, up, dn);
          put(2, up);
          put(3, dn);
          trans_apply_layers<M>(P, act, hbt, un, vh, Rc, up, dn);
          put(4, up);
          put(5, dn);
        }
      }
    }
    __syncthreads();  // every neighbour read of the waves is done: reuse the space
    if (gl >= 0) {
      const SweepItem& item = sg[gg];
      const int len = item.len, nl = item.nlines;
      const bool interior = (item.flags & 1) && record;
      if (!UNSPLIT) {
        const int g = sb[2][gg] + gslot<DIR>(gl, ge, len, nl);
#pragma unroll
        for (int f = 0; f < F; ++f) {
          wav[f * kMaxEdges + g] = Lc[f];
          wav[(F + f) * kMaxEdges + g] = Rc[f];
        }
      }
      // Mass flux of every layer through this edge, seen from the left cell:
      // hn_L + (A-dQ + F)_h. Recorded at coarse/fine interfaces of this level (for the
      // reflux of the coarser level) and accumulated, times dt, at the patch boundaries of a
      // refined level (for the reflux of its parent level).
      if (interior && (D.covered != nullptr || D.in_patch != nullptr)) {
        const int a = (DIR == 0 ? item.i0 : item.j0) + ge;  // edge a - 1/2 between cells a-1 and a
        const int line = DIR == 0 ? item.j0 + gl : item.i0 + gl;
        const int NA = DIR == 0 ? NX : NY;
        if (a >= 1 && a <= NA - 1) {
          const size_t cA = DIR == 0 ? (size_t)line * NX + (a - 1) : (size_t)(a - 1) * NX + line;
          const size_t cB = DIR == 0 ? cA + 1 : cA + NX;
          const int clft = sb[0][gg] + cslot<DIR>(gl, ge + 1, len, nl);
          const bool iface = D.covered != nullptr && D.covered[cA] != D.covered[cB];
          const bool bnd = D.in_patch != nullptr && D.in_patch[cA] != D.in_patch[cB];
          if (iface || bnd) {
#pragma unroll
            for (int m = 0; m < M; ++m) {
              const double fm = cell[(3 * m + 1) * kMaxCells + clft] + Lc[3 * m];
              const size_t fo = DIR == 0 ? ((size_t)m * NY + line) * (NX + 1) + a
                                         : ((size_t)m * (NY + 1) + a) * NX + line;
              if (iface) (DIR == 0 ? D.fxc : D.fyc)[fo] = fm;
              if (bnd) (DIR == 0 ? D.fxf : D.fyf)[fo] += dt * fm;
            }
          }
        }
      }
    }
    __syncthreads();

    // ---- phase 4: update the cells of the tile (the unsplit step updates in its own kernel) ----
    const int nupd = UNSPLIT ? 0 : sb[3][ngrp];
    for (int t = threadIdx.x; t < nupd; t += blockDim.x) {
      const int g = group_of(3, t);
      const SweepItem& item = sg[g];
      const int len = item.len, nl = item.nlines, tt = t - sb[3][g];
      int l, k;
      if (DIR == 0) { l = tt / len; k = tt - l * len; }
      else { k = tt / nl; l = tt - k * nl; }
      const int c = sb[0][g] + cslot<DIR>(l, k + 2, len, nl);
      const int gL = sb[2][g] + gslot<DIR>(l, k, len, nl), gR = sb[2][g] + gslot<DIR>(l, k + 1, len, nl);
      double qn[F];
#pragma unroll
      for (int f = 0; f < F; ++f)
        qn[f] = cell[f * kMaxCells + c] - nu * (wav[(F + f) * kMaxEdges + gL] + wav[f * kMaxEdges + gR]);
#pragma unroll
      for (int m = 0; m < M; ++m) {
        // h < 0 (or -0) -> +0; h <= dry_tol -> momenta 0 (bit-pattern comparisons as above)
        if (__double_as_longlong(qn[3 * m]) < 0) qn[3 * m] = 0.0;
        if (__double_as_longlong(qn[3 * m]) <= tol_bits) { qn[3 * m + 1] = 0.0; qn[3 * m + 2] = 0.0; }
      }
      int i, j;
      if (DIR == 0) { i = item.i0 + k; j = item.j0 + l; }
      else { i = item.i0 + l; j = item.j0 + k; }
      const size_t o = (size_t)j * Pt + i;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        qout[(3 * m) * plane + o] = qn[3 * m];
        qout[(3 * m + 1) * plane + o] = DIR == 0 ? qn[3 * m + 1] : qn[3 * m + 2];
        qout[(3 * m + 2) * plane + o] = DIR == 0 ? qn[3 * m + 2] : qn[3 * m + 1];
      }
    }
    if (record && s_rec && threadIdx.x == 0) atomicMax(&smax_bits[sg[0].desc * 2 + DIR], s_smax);
    if (lost_count) {
      for (int o = 16; o > 0; o >>= 1) lost += __shfl_xor_sync(0xffffffffu, lost, o);
      if ((threadIdx.x & 31) == 0 && lost) atomicAdd(lost_count, (unsigned)lost);
    }
    __syncthreads();
  }
}

size_t sweep_smem_bytes(int M) { return sweep_smem_doubles(M) * 8; }

template <int M, int DIR, int MINB, bool STORE, bool UNSPLIT>
static cudaError_t launch_sweep_t(const DevParams& P, const LevelDesc* descs, const SweepItem* items,
                                  const int* n_items_dev, const int* tile_off, int grid, int parity, int record,
                                  unsigned long long* smax_bits, unsigned int* lost_count, cudaStream_t st,
                                  double* est, long long eplane) {
  const size_t sm = sweep_smem_bytes(M) + (UNSPLIT ? (size_t)(M >= 3 ? 2 * M : M) * kMaxEdges * 8 : 0);
  static std::atomic<unsigned long long> attr_set{0};
  cudaError_t e = set_smem_limit_once(attr_set, sweep_kernel<M, DIR, MINB, STORE, UNSPLIT>, (int)sm);
  if (e != cudaSuccess) return e;
  sweep_kernel<M, DIR, MINB, STORE, UNSPLIT><<<grid, kThreads, sm, st>>>(P, descs, items, n_items_dev, tile_off,
                                                                         parity, record, smax_bits, lost_count, est,
                                                                         eplane);
  return cudaGetLastError();
}

template <int M, int DIR>
static cudaError_t launch_sweep_m(int ctas, const DevParams& P, const LevelDesc* descs, const SweepItem* items,
                                  const int* n_items_dev, const int* tile_off, int grid, int parity, int record,
                                  unsigned long long* smax_bits, unsigned int* lost_count, cudaStream_t st,
                                  double* est, long long eplane) {
  if constexpr (M == 2) {
    if (est != nullptr)
      return ctas >= 2 ? launch_sweep_t<M, DIR, 2, true, false>(P, descs, items, n_items_dev, tile_off, grid, parity, record,
                                                                 smax_bits, lost_count, st, est, eplane)
                       : launch_sweep_t<M, DIR, 1, true, false>(P, descs, items, n_items_dev, tile_off, grid, parity, record,
                                                                 smax_bits, lost_count, st, est, eplane);
  }
  if constexpr (M >= 3) {  // three layers fill the register file and shared memory: one CTA per SM
    if constexpr (M == 3) {
      if (P.unsplit)
        return launch_sweep_t<M, DIR, 1, false, true>(P, descs, items, n_items_dev, tile_off, grid, parity, record,
                                                      smax_bits, lost_count, st, nullptr, 0);
    }
    return launch_sweep_t<M, DIR, 1, false, false>(P, descs, items, n_items_dev, tile_off, grid, parity, record, smax_bits,
                                                   lost_count, st, nullptr, 0);
  } else {
    if (P.unsplit)
      return ctas >= 2 ? launch_sweep_t<M, DIR, 2, false, true>(P, descs, items, n_items_dev, tile_off, grid, parity, record,
                                                                 smax_bits, lost_count, st, nullptr, 0)
                       : launch_sweep_t<M, DIR, 1, false, true>(P, descs, items, n_items_dev, tile_off, grid, parity, record,
                                                                 smax_bits, lost_count, st, nullptr, 0);
    return ctas >= 2 ? launch_sweep_t<M, DIR, 2, false, false>(P, descs, items, n_items_dev, tile_off, grid, parity, record,
                                                                smax_bits, lost_count, st, nullptr, 0)
                     : launch_sweep_t<M, DIR, 1, false, false>(P, descs, items, n_items_dev, tile_off, grid, parity, record,
                                                                smax_bits, lost_count, st, nullptr, 0);
  }
}

cudaError_t launch_sweep(int dir, const DevParams& P, const LevelDesc* descs, const SweepItem* items,
                         const int* n_items_dev, const int* tile_off, int grid, int parity, int record,
                         unsigned long long* smax_bits, unsigned int* lost_count, cudaStream_t st, int ctas_per_sm,
                         double* est, long long eplane) {
  if (grid <= 0) return cudaSuccess;
  const int c = ctas_per_sm;
  if (P.M == 1)
    return dir == 0 ? launch_sweep_m<1, 0>(c, P, descs, items, n_items_dev, tile_off, grid, parity, record, smax_bits,
                                           lost_count, st, nullptr, 0)
                    : launch_sweep_m<1, 1>(c, P, descs, items, n_items_dev, tile_off, grid, parity, record, smax_bits,
                                           lost_count, st, nullptr, 0);
  if (P.M == 3)
    return dir == 0 ? launch_sweep_m<3, 0>(1, P, descs, items, n_items_dev, tile_off, grid, parity, record, smax_bits,
                                           lost_count, st, nullptr, 0)
                    : launch_sweep_m<3, 1>(1, P, descs, items, n_items_dev, tile_off, grid, parity, record, smax_bits,
                                           lost_count, st, nullptr, 0);
  if (P.M == 4)  // split step only (the host refuses the unsplit step for four layers)
    return dir == 0 ? launch_sweep_m<4, 0>(1, P, descs, items, n_items_dev, tile_off, grid, parity, record, smax_bits,
                                           lost_count, st, nullptr, 0)
                    : launch_sweep_m<4, 1>(1, P, descs, items, n_items_dev, tile_off, grid, parity, record, smax_bits,
                                           lost_count, st, nullptr, 0);
  return dir == 0 ? launch_sweep_m<2, 0>(c, P, descs, items, n_items_dev, tile_off, grid, parity, record, smax_bits,
                                         lost_count, st, est, eplane)
                  : launch_sweep_m<2, 1>(c, P, descs, items, n_items_dev, tile_off, grid, parity, record, smax_bits,
                                         lost_count, st, est, eplane);
}

}  // namespace mlswe
