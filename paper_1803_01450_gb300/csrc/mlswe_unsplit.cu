// Cell update of the unsplit step (wave propagation with transverse Riemann solves, in the
// corner-transport form of the book's Ch. 21), after the two edge passes of the sweep kernel
// (UNSPLIT variant) have written, for every x edge and y edge of the level's patches (and of
// their first ghost lines), the fluctuation each of its two cells receives (correction flux
// included) and the transverse split of each towards +t and -t. For cell (i, j):
//   Q -= dt/dx (R_{i-1/2} + L_{i+1/2}) + dt/dy (R_{j-1/2} + L_{j+1/2})
//        + dt/dx (Gx_{i+1/2} - Gx_{i-1/2}) + dt/dy (Gy_{j+1/2} - Gy_{j-1/2}),
// with the transverse correction fluxes Gx = -(dt / 2 dy) (parts towards +x received by the
// cell left of the x edge + parts towards -x received by the cell right of it), Gy likewise
// with dt / 2 dx; then the positivity fix. At coarse/fine interfaces and refined patch
// boundaries the transverse part of the mass flux is added to the flux records the edge
// passes started (one cell owns each edge).
//
// Each transverse sum belongs to an edge, and two cells use it: tiles of at most
// kUpdLen x kUpdRows cells, one warp per row. Lane k forms the sum of the x edge left of its
// cell (lane len the one right of the last cell) and takes its right one from lane k + 1 by
// a shuffle; each warp forms the sums of the y edges below its row into shared memory (the
// last row's warp also those above it). Every sum is formed once (plus one edge per row and
// one row of edges per tile) instead of twice, with the same operands in the same order, so
// the values are those of forming them per cell. All global reads of a tile are issued
// before its one barrier; the reads of the edge records (36 doubles per edge for two layers)
// set the time.
#include <cuda_runtime.h>
#include "mlswe_device.cuh"

namespace mlswe {

// Resident CTAs: the kernel waits on its reads, so more warps help even at the cost of some
// spilling (M <= 2: 4 CTAs of 64 registers, 0.96 ms against 1.03 ms with 2 CTAs of 128 on the
// 2048^2 two-layer workload); three layers keep 2 CTAs of 128 registers.
template <int M>
__global__ void __launch_bounds__(kThreads, M >= 3 ? 2 : 4)
unsplit_update_kernel(DevParams P, const LevelDesc* __restrict__ descs, const SweepItem* __restrict__ items,
                      const int* __restrict__ n_items_dev, int parity, int record) {
  static_assert(kUpdRows * 32 == kThreads && kUpdLen < 32, "one warp per row, one spare lane");
  constexpr int F = 3 * M;
  __shared__ double gys[3][kUpdRows + 1][32];  // one layer's sums of the y edges below rows 0 .. nl (row nl: above nl - 1)
  const int lane = threadIdx.x & 31, l = threadIdx.x >> 5;
  const int n_items = *n_items_dev;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const SweepItem item = items[it];
    const LevelDesc& D = descs[item.desc];
    const int NX = D.NX, NY = D.NY, Pt = D.P;
    const size_t plane = (size_t)NY * Pt;
    const double* __restrict__ qin = D.q[parity];
    double* __restrict__ qout = D.q[parity ^ 1];
    const int len = item.len, nl = item.nlines;  // len <= kUpdLen, nl <= kUpdRows
    const int i = item.i0 + lane, j = item.j0 + l;
    const bool row = l < nl, cell = row && lane < len;
    if (D.active != nullptr && *D.active == 0) {
      // no step for this member in this substep: copy the state through
      if (cell) {
        const size_t o = (size_t)j * Pt + i;
#pragma unroll
        for (int f = 0; f < F; ++f) qout[f * plane + o] = qin[f * plane + o];
      }
      continue;  // the same for every thread of the block; no shared memory used
    }
    const double dt = *D.dt;
    const double nux = dt * D.inv_dx, nuy = dt * D.inv_dy;
    const double hxy = 0.5 * nux * nuy;
    const double* __restrict__ X = D.ue;
    const double* __restrict__ Y = D.ue + 6LL * F * D.uxp;
    const long long xp = D.uxp, yp = D.uyp;
    const long long xr = NX + 1, yr = NX + 2;  // edges per x-edge row, per y-edge row
    // groups: 0 into the lower-index cell, 1 into the higher-index cell, 2/3 the transverse
    // parts of group 0 towards +t/-t, 4/5 those of group 1
    auto XG = [&](int g, int f, long long e) { return X[(long long)(g * F + f) * xp + e]; };
    auto YG = [&](int g, int f, long long e) { return Y[(long long)(g * F + f) * yp + e]; };
    // transverse sum of the y edge above the cell whose left x edge is x
    auto ysum = [&](int f, long long x) {
      return XG(4, f, x) + XG(2, f, x + 1) + XG(5, f, x + xr) + XG(3, f, x + xr + 1);
    };
    // transverse sum of the x edge right of the cell whose bottom y edge is y
    auto xsum = [&](int f, long long y) {
      return YG(4, f, y) + YG(2, f, y + yr) + YG(5, f, y + 1) + YG(3, f, y + yr + 1);
    };
    const long long xl = (long long)(j + 1) * xr + i;  // x edge left of the cell
    const long long yb = (long long)j * yr + (i + 1);   // y edge below the cell
    const bool edge = row && lane <= len;  // lanes 0 .. len form the x edges of the row
    // One layer at a time (the update and the positivity fix of a layer use only its own
    // three fields): its global reads before the barrier (the y-edge sums into shared memory,
    // the x-edge sums, fluctuations and Q^n in registers), then its update. Three fields at a
    // time keep the two-layer kernel within 64 registers with few spills (the loop is kept a
    // loop there; unrolled, the compiler draws later layers' reads forward and spills more);
    // three layers, at 128 registers, unroll it without spilling.
#pragma unroll(M >= 3 ? M : 1)
    for (int m = 0; m < M; ++m) {
      double sgl[3], dxn[3], dyn[3], q0[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) { sgl[k] = 0.0; dxn[k] = 0.0; dyn[k] = 0.0; q0[k] = 0.0; }
      if (cell) {
#pragma unroll
        for (int k = 0; k < 3; ++k) gys[k][l][lane] = ysum(3 * m + k, xl - xr);
        if (l == nl - 1) {
#pragma unroll
          for (int k = 0; k < 3; ++k) gys[k][nl][lane] = ysum(3 * m + k, xl);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int f = 3 * m + k;
          dxn[k] = XG(1, f, xl) + XG(0, f, xl + 1);
          dyn[k] = YG(1, f, yb) + YG(0, f, yb + yr);
          q0[k] = qin[f * plane + (size_t)j * Pt + i];
        }
      }
      if (edge) {
#pragma unroll
        for (int k = 0; k < 3; ++k) sgl[k] = xsum(3 * m + k, yb - 1);
      }
      __syncthreads();
      if (row) {  // whole warps
        double qn[3], gxl = 0.0, gxr = 0.0, gyb = 0.0, gyt = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double sgr = __shfl_down_sync(0xffffffffu, sgl[k], 1);
          qn[k] = 0.0;
          if (cell) {
            const double sgb = gys[k][l][lane], sgt = gys[k][l + 1][lane];
            qn[k] = q0[k] - nux * dxn[k] - nuy * dyn[k] + hxy * ((sgr - sgl[k]) + (sgt - sgb));
            if (k == 0) { gxl = sgl[0]; gxr = sgr; gyb = sgb; gyt = sgt; }
          }
        }
        if (cell) {
          const long long tol_bits = __double_as_longlong(P.dry_tol);
          if (__double_as_longlong(qn[0]) < 0) qn[0] = 0.0;
          if (__double_as_longlong(qn[0]) <= tol_bits) { qn[1] = 0.0; qn[2] = 0.0; }
          const size_t o = (size_t)j * Pt + i;
#pragma unroll
          for (int k = 0; k < 3; ++k) qout[(3 * m + k) * plane + o] = qn[k];
          if (record && (D.covered != nullptr || D.in_patch != nullptr)) {
            // Transverse part of layer m's mass flux through this cell's left / bottom edge,
            // and through its right / top edge when the neighbour there is in no patch of the
            // level (otherwise that neighbour owns the edge).
            const double hy = -0.5 * nuy, hx = -0.5 * nux;
            auto add = [&](bool xdir, int a, int line, double sv, double h) {
              const size_t cA = xdir ? (size_t)line * NX + (a - 1) : (size_t)(a - 1) * NX + line;
              const size_t cB = xdir ? cA + 1 : cA + NX;
              const bool iface = D.covered != nullptr && D.covered[cA] != D.covered[cB];
              const bool bnd = D.in_patch != nullptr && D.in_patch[cA] != D.in_patch[cB];
              if (!iface && !bnd) return;
              const double gm = h * sv;
              const size_t fo = xdir ? ((size_t)m * NY + line) * (NX + 1) + a : ((size_t)m * (NY + 1) + a) * NX + line;
              if (iface) (xdir ? D.fxc : D.fyc)[fo] += gm;
              if (bnd) (xdir ? D.fxf : D.fyf)[fo] += dt * gm;
            };
            if (i >= 1) add(true, i, j, gxl, hy);
            if (i + 1 <= NX - 1 && D.in_patch != nullptr && D.in_patch[(size_t)j * NX + i + 1] == 0)
              add(true, i + 1, j, gxr, hy);
            if (j >= 1) add(false, j, i, gyb, hx);
            if (j + 1 <= NY - 1 && D.in_patch != nullptr && D.in_patch[(size_t)(j + 1) * NX + i] == 0)
              add(false, j + 1, i, gyt, hx);
          }
        }
      }
      __syncthreads();  // the y-edge sums are rewritten for the next layer or tile
    }
  }
}

cudaError_t launch_unsplit_update(const DevParams& P, const LevelDesc* descs, const SweepItem* items,
                                  const int* n_items_dev, int grid, int parity, int record, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  if (P.M == 1)
    unsplit_update_kernel<1><<<grid, kThreads, 0, st>>>(P, descs, items, n_items_dev, parity, record);
  else if (P.M == 2)
    unsplit_update_kernel<2><<<grid, kThreads, 0, st>>>(P, descs, items, n_items_dev, parity, record);
  else if (P.M == 3)
    unsplit_update_kernel<3><<<grid, kThreads, 0, st>>>(P, descs, items, n_items_dev, parity, record);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace mlswe
