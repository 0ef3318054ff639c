// Device-side data structures and the per-edge multilayer Riemann solver.
//
// Paper: arXiv:1803.01450. The paper cites GeoClaw's multilayer solver (Sec. 1)
// without writing it out; the solver below is this library's reading of it:
//  * surfaces eta_m = B + h_M + ... + h_m (Sec. 2.1, Eq. (4)), effective
//    bathymetry Bhat_m = eta_{m+1} (Eq. (5)), top-down wet rule (Sec. 2.1);
//  * f-waves of the flux jump with the layer coupling folded into the
//    momentum row: d1_m = D(hn un) + g hbar_m (D eta_m + sum_{n<m} r D h_n);
//  * all layers wet on both sides (M = 2): 4 acoustic waves of the coupled
//    normal system, eigenvalues from the closed-form guesses for equal layer
//    velocities refined by 2 Newton steps on the characteristic quartic, wave
//    strengths from R beta = delta with eigenvectors (1, l, a, a l),
//    a = ((l - u1)^2 - g hbar_1) / (g hbar_1), plus one shear wave per layer;
//  * otherwise every layer alone (Roe speeds), a dry layer whose wet
//    neighbour's surface lies below the dry cell's effective bathymetry
//    becomes a reflecting wall for that layer only.
//
// GPU specifics (not in the paper): FP64 is the bound on GB300 (about 1/66 of
// the FP32 rate), so every per-cell quantity (velocities, sqrt(h), surfaces,
// wet bits) is computed once per cell and staged in shared memory, divisions
// are reciprocal-and-multiply, and the 4x4 wave-strength system is solved in
// closed form through its Vandermonde structure instead of by elimination.
#pragma once
#include <atomic>
#include <cstdint>

namespace mlswe {

constexpr int kNG = 2;          // ghost cells per side
constexpr int kMaxEdges = 256;  // edges per tile (one thread each)
constexpr int kMaxCells = 288;  // cells per tile (edges + lines, lines <= 32)
constexpr int kThreads = 256;
constexpr int kMaxGroups = 4;   // groups of lines (runs of patch lines) packed into one sweep tile
constexpr int kUpdLen = 31, kUpdRows = 8;  // cell tiles of the unsplit step's update (one warp per row)

struct DevParams {
  int M;
  double g;
  double r;        // rho_1 / rho_2 (M = 2)
  double omr, four_r, omr_g;  // 1 - r, 4 r, (1 - r) g (M = 2), computed on the host
  double rho[4];   // layer densities, top (lightest) first
  double rr[4][4];  // rho_n / rho_m at [n][m], computed on the host
  double irho[4];   // 1 / rho_m
  double gap_g[4];  // (1 - rho_m / rho_{m+1}) g: reduced gravity between layers m and m + 1
  double dry_tol;
  int order;
  int limiter;
  int eigen;
  int unsplit;     // 1: unsplit step with transverse Riemann solves (M <= 2)
};

// One (member, level) of the hierarchy: dense arrays over the whole level.
struct LevelDesc {
  double* q[2];        // state double buffer [3M][NY][P]
  double* qs;          // state after the x sweep [3M][NY][P]
  double* B;           // bathymetry [NY][P]
  const uint8_t* in_patch;   // [NY][NX] 1 inside a patch of this level (null on level 0)
  const uint8_t* covered;    // [NY][NX] 1 where a finer patch covers the cell (null if none)
  double* fxc;         // interface mass flux of this (coarse) level, x edges [M][NY][NX+1]
  double* fyc;         // y edges [M][NY+1][NX]
  double* fxf;         // boundary mass flux accumulators of this (fine) level, x edges
  double* fyf;         // y edges
  const double* dt;    // device scalar: time step of this member on this level
  const int* rt;       // device scalar: time steps of this level per step of its parent
  const int* active;   // device scalar: 0 while a substep beyond this member's rt runs for
                       // others (the step then copies the state through and records nothing);
                       // null: always active
  int NX, NY, P;
  double inv_dx, inv_dy;
  // Unsplit step: per-edge arrays of the level, 6 groups of 3M planes for the x edges (plane
  // size uxp, edge left of cell i on row j at (j + 1) (NX + 1) + i, rows -1 .. NY), then 6
  // groups for the y edges (plane size uyp, edge below cell j on column i at j (NX + 2) +
  // i + 1, columns -1 .. NX). Groups: the fluctuation into the lower-index cell (with the
  // correction flux), into the higher-index cell, and the transverse parts of each towards
  // +t and -t; fields in (h, hu, hv) order. Null for the split step.
  double* ue;
  long long uxp, uyp;
  // Copy of the patch cells of this level (level >= 1) taken before a coarse-step attempt of
  // mlswe_advance, layout of q; a rejected attempt restores it. Null until advance needs it.
  double* snap;
};

// One tile of a sweep: `nlines` lines of `len` cells, along x (x sweep: rows
// j0.., cells i0..) or along y (y sweep: columns i0.., cells j0..).
struct SweepItem {
  int desc;
  int i0, j0;
  int len;
  int nlines;
  int flags;  // bit 0: interior lines (count CFL, record interface fluxes); bit 1: the tile
              // ends its patch line (its last edge is the patch boundary)
};

// Raises a kernel's dynamic shared-memory limit once per device: the attribute belongs
// to the device that is current when it is set, so a process that launches on several
// devices sets it on each (bit d of `flags` marks device d; devices past 63 set it on
// every launch). Safe to call from several host threads: setting it twice is harmless.
template <class K>
cudaError_t set_smem_limit_once(std::atomic<unsigned long long>& flags, K* kernel, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (flags.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) flags.fetch_or(bit, std::memory_order_release);
  return e;
}

__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

// ---- helpers that keep comparisons off the FP64 pipe (integer work is nearly free) ----

// -1, 0, +1 for s < 0, s == 0 (either sign of zero), s > 0 (finite or infinite s).
__device__ __forceinline__ int sign_class(double s) {
  const long long b = __double_as_longlong(s);
  if ((b << 1) == 0) return 0;
  return b < 0 ? -1 : 1;
}

// Bit pattern of |s|; for non-negative doubles the unsigned order is the numeric order.
__device__ __forceinline__ unsigned long long abs_bits(double s) {
  return (unsigned long long)__double_as_longlong(s) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

__device__ __forceinline__ double pos_min(double a, double b) {  // both > 0
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x < y ? x : y);
}

// Share of a wave of speed s that goes to the left cell, second-order correction included:
//   c = (1 if s < 0, 0 if s > 0, 1/2 if s = 0) + sign(s) (1 - nu |s|) phi(theta) / 2
// (the correction only where act). For the MC limiter phi / 2 = min((1 + theta) / 4, 1,
// theta) exactly (scalings by powers of two), so its factor 2 goes into the weight
// sign(s) (1 - nu |s|) and the correction costs one FMA for the weight, one for the
// limiter and one to add it. theta = num * iden; limiters: 0 none (phi = 1), 1 minmod, 2 MC;
// the minima of positive numbers are taken on their bit patterns.
__device__ __forceinline__ double left_share(int kind, int sc, bool act, double num, double iden, double s,
                                             double nu) {
  const double base = sc < 0 ? 1.0 : (sc > 0 ? 0.0 : 0.5);
  if (!act) return base;
  const double th = num * iden;
  if (kind == 2) {
    if (__double_as_longlong(th) <= 0) return base;  // phi = 0
    const double ph = pos_min(pos_min(fma(0.25, th, 0.25), 1.0), th);
    const double w = sc > 0 ? fma(-nu, fabs(s), 1.0) : fma(nu, fabs(s), -1.0);
    return fma(w, ph, base);
  }
  double ph = 1.0;
  if (kind == 1) {
    if (__double_as_longlong(th) <= 0) return base;
    ph = pos_min(1.0, th);
  }
  const double w = sc > 0 ? fma(-0.5 * nu, fabs(s), 0.5) : fma(0.5 * nu, fabs(s), -0.5);
  return fma(w, ph, base);
}

// |x| in [2^-160, 2^160), read from the exponent field (integer unit, not the FP64 pipe).
__device__ __forceinline__ bool moderate(double x) {
  const unsigned e = (unsigned)(__double_as_longlong(x) >> 52) & 0x7ffu;
  return e - 863u <= 320u;
}

// Reciprocal and reciprocal square root by iteration (Newton-Raphson family; see Muller et
// al., Handbook of Floating-Point Arithmetic, ch. 5 on iterations for division and square
// root), cheaper on the FP64 pipe than the correctly rounded functions. The seed is the FP32
// reciprocal (square root) of the leading 20 significand bits, scaled by integer arithmetic
// on the exponent field: relative error eta below 2^-19. One third-order (Householder) step
// follows; its truncation error is O(eta^3) < 2^-56, so the result is within about one unit
// in the last place of the exact value (not always the correctly rounded one).
//
// FP32 seeds: the hardware approximations (relative error about 2^-23), arguments in [1, 4)
// (never subnormal, so flushing them to zero changes nothing).
__device__ __forceinline__ float seed_rcp(float m) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(m));
  return r;
}
__device__ __forceinline__ float seed_rsqrt(float m) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(m));
  return r;
}

// 1/x for a normal x with |x| < 2^1022: with e = 1 - x y, y' = y + y (e + e^2).
__device__ __forceinline__ double rcp_iter(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int ex = (int)((hi >> 20) & 0x7ffu);                          // biased exponent of x
  const float m = __uint_as_float(0x3f800000u | ((hi & 0xfffffu) << 3));  // significand in [1, 2)
  const unsigned r = __float_as_uint(seed_rcp(m));                     // 1/m in (1/2, 1]
  const int re = (int)(r >> 23) - 127;                                  // its exponent: 0 or -1
  // 1/x = sign(x) (1/m) 2^(1023 - ex): biased exponent 2046 - ex + re
  const unsigned long long yb = (b & 0x8000000000000000ull) | ((unsigned long long)(2046 - ex + re) << 52) |
                                ((unsigned long long)(r & 0x7fffffu) << 29);
  const double y = __longlong_as_double((long long)yb);
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// 1/sqrt(x) for any positive normal x: x = s 2^(2k) with s in [1, 4) (the
// significand, doubled when the exponent is odd); with e = 1 - x y^2,
// y' = y + y e (1/2 + 3 e / 8).
__device__ __forceinline__ double rsqrt_iter(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int E = (int)(hi >> 20) - 1023;  // unbiased exponent (x > 0: no sign bit)
  const int odd = E & 1;
  const float s = __uint_as_float((odd ? 0x40000000u : 0x3f800000u) | ((hi & 0xfffffu) << 3));
  const unsigned r = __float_as_uint(seed_rsqrt(s));  // in (1/2, 1]
  const int re = (int)(r >> 23) - 127;            // 0 or -1
  const int k = (E - odd) / 2;                     // exact: E - odd is even
  const unsigned long long yb = ((unsigned long long)(1023 + re - k) << 52) | ((unsigned long long)(r & 0x7fffffu) << 29);
  const double y = __longlong_as_double((long long)yb);
  const double xy = x * y;
  const double e = fma(-xy, y, 1.0);
  return fma(y, e * fma(0.375, e, 0.5), y);
}

// 1/x to about 2^-44 relative for a normal x with |x| < 2^1022: the FP32 seed of the leading
// 23 significand bits (relative error below 2^-22) and one second-order Newton-Raphson step,
// y' = y + y e with e = 1 - x y (error e^2), 2 FP64 instructions. Only for factors whose own
// error is multiplied by a small quantity: the Newton corrections of the eigenvalues (their
// error is the correction times 2^-44, below the rounding of the eigenvalue) and the
// limiter ratios (an error of 2^-44 in theta moves the limited correction by as little).
__device__ __forceinline__ double rcp2_iter(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int ex = (int)((hi >> 20) & 0x7ffu);
  const float m = __uint_as_float(0x3f800000u | ((hi & 0xfffffu) << 3) | (lo >> 29));  // in [1, 2)
  const unsigned r = __float_as_uint(seed_rcp(m));
  const int re = (int)(r >> 23) - 127;
  const unsigned long long yb = (b & 0x8000000000000000ull) | ((unsigned long long)(2046 - ex + re) << 52) |
                                ((unsigned long long)(r & 0x7fffffu) << 29);
  const double y = __longlong_as_double((long long)yb);
  return fma(y, fma(-x, y, 1.0), y);
}

// 1/sqrt(x) to about 2^-43 relative for any positive normal x: the FP32 seed of the leading
// 23 significand bits and one second-order step, y' = y + (y e) / 2 with e = 1 - x y^2
// (error 3 e^2 / 8), 4 FP64 instructions. For the eigenvalue guesses of the coupled branch,
// which the Newton steps then correct (and which stand as they are only where
// hyperbolicity is lost, to that accuracy).
__device__ __forceinline__ double rsqrt2_iter(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int E = (int)(hi >> 20) - 1023;
  const int odd = E & 1;
  const float sg = __uint_as_float((odd ? 0x40000000u : 0x3f800000u) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  const unsigned r = __float_as_uint(seed_rsqrt(sg));
  const int re = (int)(r >> 23) - 127;
  const int k = (E - odd) / 2;
  const unsigned long long yb = ((unsigned long long)(1023 + re - k) << 52) | ((unsigned long long)(r & 0x7fffffu) << 29);
  const double y = __longlong_as_double((long long)yb);
  const double e = fma(-(x * y), y, 1.0);
  return fma(y * e, 0.5, y);
}

// rcp2_iter of N numbers when every |x_p| lies in [2^-160, 2^160) (one range test for the
// group), one division each otherwise.
template <int N>
__device__ __forceinline__ void reciprocal2_group(const double* x, double* inv) {
  bool safe = true;
#pragma unroll
  for (int p = 0; p < N; ++p) safe = safe && moderate(x[p]);
  if (safe) {
#pragma unroll
    for (int p = 0; p < N; ++p) inv[p] = rcp2_iter(x[p]);
  } else {
#pragma unroll
    for (int p = 0; p < N; ++p) inv[p] = rcp(x[p]);
  }
}

// 0.5 / x_p the same way; the factor 1/2 lowers the exponent field of the iterate (exact: for
// |x_p| in [2^-160, 2^160) the result is a normal number far from the subnormal range).
template <int N>
__device__ __forceinline__ void half_reciprocal2_group(const double* x, double* inv) {
  bool safe = true;
#pragma unroll
  for (int p = 0; p < N; ++p) safe = safe && moderate(x[p]);
  if (safe) {
#pragma unroll
    for (int p = 0; p < N; ++p) inv[p] = __longlong_as_double(__double_as_longlong(rcp2_iter(x[p])) - (1ll << 52));
  } else {
#pragma unroll
    for (int p = 0; p < N; ++p) inv[p] = 0.5 * rcp(x[p]);
  }
}

// The iterations where |x| lies in [2^-160, 2^160) (x > 0 for the square root), the
// library functions elsewhere (zero, subnormal, huge, infinite, NaN or negative arguments).
__device__ __forceinline__ double rcp_fast(double x) { return moderate(x) ? rcp_iter(x) : rcp(x); }
// 0.5 / x: the iteration's result with its exponent field lowered by one (exact: the result
// of a moderate argument is a normal number far from the subnormal range).
__device__ __forceinline__ double half_rcp_fast(double x) {
  if (moderate(x)) return __longlong_as_double(__double_as_longlong(rcp_iter(x)) - (1ll << 52));
  return 0.5 * rcp(x);
}
__device__ __forceinline__ double rsqrt_fast(double x) {
  return __double_as_longlong(x) >= 0 && moderate(x) ? rsqrt_iter(x) : rsqrt(x);
}
__device__ __forceinline__ double sqrt_fast(double x) {
  return __double_as_longlong(x) >= 0 && moderate(x) ? x * rsqrt_iter(x) : sqrt(x);
}

// Reciprocals of N <= 6 nonzero numbers: when every |x_p| lies in [2^-160, 2^160), each by
// the seeded iteration (3 FP64 instructions; an earlier form shared one reciprocal of the
// product among the N values, which costs about 4N + 1); otherwise one division each. One
// range test for the group keeps the branch structure of the caller simple.
template <int N>
__device__ __forceinline__ void batched_reciprocal(const double* x, double* inv) {
  static_assert(N <= 6, "groups of at most six");
  bool safe = true;
#pragma unroll
  for (int p = 0; p < N; ++p) safe = safe && moderate(x[p]);
  if (safe) {
#pragma unroll
    for (int p = 0; p < N; ++p) inv[p] = rcp_iter(x[p]);
  } else {
#pragma unroll
    for (int p = 0; p < N; ++p) inv[p] = rcp(x[p]);
  }
}


// batched_reciprocal for any N, in groups of at most six.
template <int N>
__device__ __forceinline__ void batched_reciprocal_groups(const double* x, double* inv) {
  if constexpr (N <= 6) {
    batched_reciprocal<N>(x, inv);
  } else {
    batched_reciprocal<6>(x, inv);
    batched_reciprocal_groups<N - 6>(x + 6, inv + 6);
  }
}

// ----------------------------------------------------------------------------
// Cell record staged in shared memory (fields already permuted to normal /
// transverse for the sweep direction).
// ----------------------------------------------------------------------------
template <int M>
struct Rec {
  static constexpr int H = 0;             // h_m at 3m, hn_m at 3m+1, ht_m at 3m+2
  static constexpr int UN = 3 * M;        // sqrt(h_m) un_m at UN + 2m, sqrt(h_m) ut_m at UN + 2m + 1
                                          // (0 where not wet): the Roe-average numerators
  static constexpr int SQ = 5 * M;        // sqrt(h_m)
  static constexpr int ETA = 6 * M;       // eta_m
  static constexpr int BB = 7 * M;        // B
  static constexpr int N = 7 * M + 1;
};

// Compressed waves of one edge: acoustic wave p carries in layer m the mass mass[m][p], so
//   Z_p = (mass[m][p], mass[m][p] s_p, mass[m][p] vh_m) for m = 1 .. M,
// shear wave of layer m is (0, 0, z_m) on layer m with speed us_m.
template <int M>
struct EdgeW {
  static constexpr int NA = 2 * M;
  double mass[M][NA], s[NA];
  double z[M], us[M], vh[M];
  // What the acoustic waves of layer m sum to: its mass and normal-momentum flux jumps
  // (sum_p Z_p = jump exactly for the f-wave split, up to rounding).
  double t0[M], t1[M];
  double hbt[M];  // depth whose gravity speed the transverse split of this edge takes
  double muk[M];  // M >= 3, coupled edges: eigenvalues of the coupling matrix G (velocity-free)
  int wall;  // bit 2m: layer m reflects into the left cell (left is dry), bit 2m+1: right
};

template <int M>
struct WRec {  // shared-memory layout of EdgeW: mass of layer m, wave p at A + 2M m + p
  static constexpr int A = 0, S = 2 * M * M, Z = S + 2 * M, US = Z + M, VH = US + M, T0 = VH + M, T1 = T0 + M,
                       N = T1 + M;
};

// Per-edge record of a coupled two-layer edge that the adjoint's reverse pass reads instead
// of rebuilding it (field offsets; each field is one plane over the edges of a sweep):
// reciprocals of the Roe weights (sqrt hL + sqrt hR per layer), of hbar_1 + hbar_2 and of
// c1 = g hbar_1; reciprocal square roots of the discriminant and of mu_+, mu_-; the
// eigenvalue guesses, the iterate after the first Newton step and the final eigenvalues;
// 1/P'(lambda) of both Newton steps; reciprocals of prod_{q != p}(lambda_p - lambda_q); the
// wave strengths beta_p; 1.0 if the Newton steps ran, else 0.0.
struct FwdRec {
  static constexpr int IS0 = 0, IS1 = 1, IH = 2, IC1 = 3, IDISC = 4, ISP = 5, ISM = 6, LAM0 = 7, LAM1 = 11,
                       LAM = 15, ID0 = 19, ID1 = 23, IDEN = 27, BETA = 31, NEWTON = 35, N = 36;
};

// Layer of acoustic slot p in the per-layer (decoupled) branch: layer m owns slots m
// (left-going) and 2M - 1 - m (right-going).
template <int M>
__device__ __forceinline__ int layer_of_slot(int p) {
  return p < M ? p : 2 * M - 1 - p;
}

// rho_n / rho_m: weight of the depth jump of the lighter layer n above in layer m's pressure.
template <int M>
__device__ __forceinline__ double density_ratio(const DevParams& P, int n, int m) {
  if constexpr (M == 2) return P.r;
  return P.rr[n][m];
}

// Single-layer f-wave split of (d0, d1, d2) with speeds s1 < s2 (inv_ds: 1/(s2 - s1) when
// known, else 0).
template <int M>
__device__ __forceinline__ void split_single(int m, int pa, int pb, double d0, double d1, double d2,
                                             double s1, double s2, double vh, double us, EdgeW<M>& W,
                                             double inv_ds = 0.0) {
  const double inv = inv_ds != 0.0 ? inv_ds : rcp_fast(s2 - s1);
  const double b1 = (s2 * d0 - d1) * inv;
  const double b2 = (d1 - s1 * d0) * inv;
  W.mass[m][pa] = b1;
  W.mass[m][pb] = b2;
  W.s[pa] = s1; W.s[pb] = s2;
  W.z[m] = d2 - vh * d0;
  W.us[m] = us;
  W.vh[m] = vh;
  W.t0[m] = d0;
  W.t1[m] = d1;
}

// ---- general coupled branch (M >= 3 layers, all wet on both sides) ----

// Eigenvalues of the symmetric M x M matrix K by cyclic Jacobi rotations (each rotation
// zeroes one off-diagonal pair: tan phi = sgn(theta) / (|theta| + sqrt(theta^2 + 1)),
// theta = (K_qq - K_pp) / (2 K_pq)), until the off-diagonal part is below 1e-32 of the
// diagonal or 10 sweeps; mu in descending order.
template <int M>
__device__ __forceinline__ void jacobi_eigenvalues(double K[M][M], double mu[M]) {
  for (int sweep = 0; sweep < 10; ++sweep) {
    double off = 0.0, dg = 0.0;
#pragma unroll
    for (int i = 0; i < M; ++i) {
      dg = fma(K[i][i], K[i][i], dg);
#pragma unroll
      for (int j = i + 1; j < M; ++j) off = fma(K[i][j], K[i][j], off);
    }
    if (off <= 1e-32 * dg) break;
#pragma unroll
    for (int p = 0; p < M - 1; ++p)
#pragma unroll
      for (int q = p + 1; q < M; ++q) {
        const double kpq = K[p][q];
        if (kpq == 0.0) continue;
        const double theta = (K[q][q] - K[p][p]) * (0.5 * rcp_fast(kpq));
        const double t = copysign(rcp_fast(fabs(theta) + sqrt_fast(fma(theta, theta, 1.0))), theta);
        const double c = rsqrt_fast(fma(t, t, 1.0)), sn = t * c;
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const double kp = K[k][p], kq = K[k][q];
          K[k][p] = c * kp - sn * kq;
          K[k][q] = sn * kp + c * kq;
        }
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const double pk = K[p][k], qk = K[q][k];
          K[p][k] = c * pk - sn * qk;
          K[q][k] = sn * pk + c * qk;
        }
      }
  }
#pragma unroll
  for (int i = 0; i < M; ++i) mu[i] = K[i][i];
#pragma unroll
  for (int i = 0; i < M; ++i)
#pragma unroll
    for (int j = i + 1; j < M; ++j) {
      const double a = mu[i], b = mu[j];
      mu[i] = fmax(a, b);
      mu[j] = fmin(a, b);
    }
}

// One elimination step (pivot column K, a compile-time index, so every access below is to a
// fixed register): partial pivoting (ties: lowest row), the row exchange as selects, then
// the elimination of column K below the pivot; recurses to K + 1.
template <int N, int K>
__device__ __forceinline__ void gauss_step(double (&A)[N][N], double (&b)[N]) {
  if constexpr (K < N) {
    int piv = K;
    unsigned long long best = abs_bits(A[K][K]);
#pragma unroll
    for (int i = K + 1; i < N; ++i) {
      const unsigned long long v = abs_bits(A[i][K]);
      if (v > best) { best = v; piv = i; }
    }
#pragma unroll
    for (int i = K + 1; i < N; ++i) {
      const bool sw = i == piv;
#pragma unroll
      for (int j = K; j < N; ++j) {
        const double t = A[K][j];
        A[K][j] = sw ? A[i][j] : t;
        A[i][j] = sw ? t : A[i][j];
      }
      const double tb = b[K];
      b[K] = sw ? b[i] : tb;
      b[i] = sw ? tb : b[i];
    }
    const double ip = rcp_fast(A[K][K]);
#pragma unroll
    for (int i = K + 1; i < N; ++i) {
      const double f = A[i][K] * ip;
#pragma unroll
      for (int j = K + 1; j < N; ++j) A[i][j] = fma(-f, A[K][j], A[i][j]);
      b[i] = fma(-f, b[K], b[i]);
    }
    gauss_step<N, K + 1>(A, b);
  }
}

// Solve A x = b (N x N) by Gaussian elimination with partial pivoting. The steps are
// instantiated per pivot column, so every index is a compile-time constant and A stays in
// registers (a loop over the pivot column left A in local memory for N = 6).
template <int N>
__device__ __forceinline__ void gauss_solve(double (&A)[N][N], double (&b)[N], double (&x)[N]) {
  gauss_step<N, 0>(A, b);
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    double sum = b[k];
#pragma unroll
    for (int j = k + 1; j < N; ++j) sum = fma(-A[k][j], x[j], sum);
    x[k] = sum * rcp_fast(A[k][k]);
  }
}

// The same elimination for R right-hand sides at once (rows b[r]): the pivots depend on A
// only, so each right-hand side goes through exactly the operations of gauss_solve alone,
// while A is eliminated once.
template <int N, int R, int K>
__device__ __forceinline__ void gauss_step_multi(double (&A)[N][N], double (&b)[R][N]) {
  if constexpr (K < N) {
    int piv = K;
    unsigned long long best = abs_bits(A[K][K]);
#pragma unroll
    for (int i = K + 1; i < N; ++i) {
      const unsigned long long v = abs_bits(A[i][K]);
      if (v > best) { best = v; piv = i; }
    }
#pragma unroll
    for (int i = K + 1; i < N; ++i) {
      const bool sw = i == piv;
#pragma unroll
      for (int j = K; j < N; ++j) {
        const double t = A[K][j];
        A[K][j] = sw ? A[i][j] : t;
        A[i][j] = sw ? t : A[i][j];
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const double tb = b[r][K];
        b[r][K] = sw ? b[r][i] : tb;
        b[r][i] = sw ? tb : b[r][i];
      }
    }
    const double ip = rcp_fast(A[K][K]);
#pragma unroll
    for (int i = K + 1; i < N; ++i) {
      const double f = A[i][K] * ip;
#pragma unroll
      for (int j = K + 1; j < N; ++j) A[i][j] = fma(-f, A[K][j], A[i][j]);
#pragma unroll
      for (int r = 0; r < R; ++r) b[r][i] = fma(-f, b[r][K], b[r][i]);
    }
    gauss_step_multi<N, R, K + 1>(A, b);
  }
}

template <int N, int R>
__device__ __forceinline__ void gauss_solve_multi(double (&A)[N][N], double (&b)[R][N], double (&x)[R][N]) {
  gauss_step_multi<N, R, 0>(A, b);
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    const double id = rcp_fast(A[k][k]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      double sum = b[r][k];
#pragma unroll
      for (int j = k + 1; j < N; ++j) sum = fma(-A[k][j], x[r][j], sum);
      x[r][k] = sum * id;
    }
  }
}

// Coupled branch for M = 3 layers. The eigenvalues of the normal system at the Roe state are
// the roots of P(l) = det(A(l)), A(l) = diag((l - u_m)^2) - G, G_mn = g hbar_m C_mn with
// C_mn = 1 for n >= m and rho_n / rho_m for the lighter layers n < m. Guesses: the roots for
// equal velocities, ubar -+ sqrt(mu_k), mu_k the eigenvalues of G (similar to the symmetric
// K_mn = sqrt(w_m w_n) rho_min(m,n), w_m = g hbar_m / rho_m); then 2 Newton steps with
// P' = sum_m 2 (l - u_m) cof_mm(A). Eigenvectors: dh_1 = 1 and the first two rows of
// A(l) dh = 0 (Cramer); momenta l dh; strengths from the 6 x 6 system of the flux jumps.
// Loss of hyperbolicity: some adjacent pair with (u_m - u_{m+1})^2 >= (1 - rho_m/rho_{m+1})
// g (hbar_m + hbar_{m+1}); the guesses are used then (and for P.eigen = 1).
// Eigenvalues lam (guess order: external -, ..., external +) and eigenvector depths dh (dh_1
// = 1) of the coupled three-layer system with velocities u, mean depths hb and coupling G,
// from mu_k (the eigenvalues of G): the guesses, the loss-of-hyperbolicity test (returned),
// two Newton steps and Cramer's rule, as described above.
__device__ __forceinline__ double det3(double a00, double a01, double a02, double a10, double a11, double a12,
                                      double a20, double a21, double a22) {
  return a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) + a02 * (a10 * a21 - a11 * a20);
}

// Determinant of the 3 x 3 matrix of A without row r and column c (4 x 4 A; r, c compile-time
// constants after unrolling).
template <int R, int C>
__device__ __forceinline__ double minor4(const double A[4][4]) {
  constexpr int r0 = R == 0 ? 1 : 0, r1 = R <= 1 ? 2 : 1, r2 = R <= 2 ? 3 : 2;
  constexpr int c0 = C == 0 ? 1 : 0, c1 = C <= 1 ? 2 : 1, c2 = C <= 2 ? 3 : 2;
  return det3(A[r0][c0], A[r0][c1], A[r0][c2], A[r1][c0], A[r1][c1], A[r1][c2], A[r2][c0], A[r2][c1], A[r2][c2]);
}

template <int M>
__device__ __forceinline__ bool general_eig(const DevParams& P, const double G[M][M], const double* u,
                                            const double* hb, const double* mu, double* lam, double dh[][M]) {
  static_assert(M == 3 || M == 4, "general coupled branch written for three and four layers");
  constexpr int N = 2 * M;
  const double g = P.g;
  double hs = 0.0, hus = 0.0;
#pragma unroll
  for (int m = 0; m < M; ++m) { hs += hb[m]; hus = fma(hb[m], u[m], hus); }
  const double ubar = hus * rcp_fast(hs);
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const double sq = sqrt_fast(mu[k]);
    lam[k] = ubar - sq;
    lam[N - 1 - k] = ubar + sq;
  }
  bool lst = false;
#pragma unroll
  for (int m = 0; m + 1 < M; ++m) {
    const double du = u[m] - u[m + 1];
    lst = lst || (du * du >= P.gap_g[m] * (hb[m] + hb[m + 1]));
  }
  auto build_A = [&](double l, double A[M][M]) {
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int n = 0; n < M; ++n) {
        const double am = l - u[m];
        A[m][n] = (m == n ? am * am : 0.0) - G[m][n];
      }
  };
  if (!lst && P.eigen == 0) {
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      double Pl[N], dP[N], idP[N];
#pragma unroll
      for (int p = 0; p < N; ++p) {
        double A[M][M];
        build_A(lam[p], A);
        if constexpr (M == 3) {
          const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
          const double c11 = A[0][0] * A[2][2] - A[0][2] * A[2][0];
          const double c22 = A[0][0] * A[1][1] - A[0][1] * A[1][0];
          Pl[p] = A[0][0] * c00 - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                  A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
          dP[p] = 2.0 * ((lam[p] - u[0]) * c00 + (lam[p] - u[1]) * c11 + (lam[p] - u[2]) * c22);
        } else {
          // det A by the first row; P' = sum_m 2 (l - u_m) cof_mm (d/dl of the diagonal)
          const double c00 = minor4<0, 0>(A), c11 = minor4<1, 1>(A), c22 = minor4<2, 2>(A), c33 = minor4<3, 3>(A);
          Pl[p] = A[0][0] * c00 - A[0][1] * minor4<0, 1>(A) + A[0][2] * minor4<0, 2>(A) - A[0][3] * minor4<0, 3>(A);
          dP[p] = 2.0 * ((lam[p] - u[0]) * c00 + (lam[p] - u[1]) * c11 + (lam[p] - u[2]) * c22 +
                         (lam[p] - u[3]) * c33);
        }
      }
      batched_reciprocal_groups<N>(dP, idP);
#pragma unroll
      for (int p = 0; p < N; ++p) lam[p] -= Pl[p] * idP[p];
    }
  }
#pragma unroll
  for (int p = 0; p < N; ++p) {
    double A[M][M];
    build_A(lam[p], A);
    dh[p][0] = 1.0;
    if constexpr (M == 3) {
      const double det2 = A[0][1] * A[1][2] - A[0][2] * A[1][1];
      const double id2 = rcp_fast(det2);
      dh[p][1] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id2;
      dh[p][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id2;
    } else {
      // rows 0..2 of A dh = 0 with dh_1 = 1: sum_{c >= 1} A[r][c] dh_c = -A[r][0], by Cramer
      const double id = rcp_fast(det3(A[0][1], A[0][2], A[0][3], A[1][1], A[1][2], A[1][3], A[2][1], A[2][2], A[2][3]));
      dh[p][1] = -det3(A[0][0], A[0][2], A[0][3], A[1][0], A[1][2], A[1][3], A[2][0], A[2][2], A[2][3]) * id;
      dh[p][2] = -det3(A[0][1], A[0][0], A[0][3], A[1][1], A[1][0], A[1][3], A[2][1], A[2][0], A[2][3]) * id;
      dh[p][3] = -det3(A[0][1], A[0][2], A[0][0], A[1][1], A[1][2], A[1][0], A[2][1], A[2][2], A[2][0]) * id;
    }
  }
  return lst;
}

template <int M>
__device__ __forceinline__ void coupling_matrix(const DevParams& P, const double* hb, double G[M][M]) {
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int n = 0; n < M; ++n) G[m][n] = P.g * hb[m] * (n >= m ? 1.0 : density_ratio<M>(P, n, m));
}

template <int M, class CRec>
__device__ __forceinline__ void coupled_general(const DevParams& P, const CRec cL, const CRec cR,
                                                const double* hb, const double* d0, const double* d1,
                                                const double* d2, EdgeW<M>& W, int& lost) {
  static_assert(M == 3 || M == 4, "general coupled branch written for three and four layers");
  using R = Rec<M>;
  constexpr int N = 2 * M;
  const double g = P.g;
  double uh[M], vh[M], G[M][M], K[M][M], wq[M], mu[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const double sl = cL[R::SQ + m], sr = cR[R::SQ + m];
    const double inv = rcp_fast(sl + sr);
    uh[m] = (cL[R::UN + 2 * m] + cR[R::UN + 2 * m]) * inv;
    vh[m] = (cL[R::UN + 2 * m + 1] + cR[R::UN + 2 * m + 1]) * inv;
    wq[m] = sqrt_fast(g * hb[m] * P.irho[m]);
  }
  coupling_matrix<M>(P, hb, G);
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int n = 0; n < M; ++n) K[m][n] = wq[m] * wq[n] * P.rho[m < n ? m : n];  // densities increase downwards
  jacobi_eigenvalues<M>(K, mu);
  double lam[N], dh[N][M];
  lost += general_eig<M>(P, G, uh, hb, mu, lam, dh) ? 1 : 0;
  // the strengths
  double Rm[N][N], rhs[N], beta[N];
#pragma unroll
  for (int p = 0; p < N; ++p)
#pragma unroll
    for (int m = 0; m < M; ++m) {
      Rm[2 * m][p] = dh[p][m];
      Rm[2 * m + 1][p] = lam[p] * dh[p][m];
    }
#pragma unroll
  for (int m = 0; m < M; ++m) { rhs[2 * m] = d0[m]; rhs[2 * m + 1] = d1[m]; }
  gauss_solve<N>(Rm, rhs, beta);
#pragma unroll
  for (int p = 0; p < N; ++p) {
#pragma unroll
    for (int m = 0; m < M; ++m) W.mass[m][p] = beta[p] * dh[p][m];
    W.s[p] = lam[p];
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    W.z[m] = d2[m] - vh[m] * d0[m];
    W.us[m] = uh[m];
    W.vh[m] = vh[m];
    W.t0[m] = d0[m];
    W.t1[m] = d1[m];
    W.hbt[m] = hb[m];
    W.muk[m] = mu[m];
  }
}

// A cell record read in place from the tile's shared-memory records (field f at
// p[f * kMaxCells]): fields are loaded where the solver uses them instead of all up front,
// which keeps fewer values live in registers.
struct SmemRec {
  const double* p;
  __device__ __forceinline__ double operator[](int f) const { return p[f * kMaxCells]; }
};

// Riemann solve at one edge. cL, cR: cell records (arrays or SmemRec views); wL, wR: wet
// bits (bit m = layer m).
// STORE: a coupled two-layer edge also writes its FwdRec record to st (field k at
// st[k * sstride]). The stores are unconditional (st must be valid), so the arithmetic is
// compiled in the same basic blocks, and therefore rounds the same, as without STORE.
template <int M, bool STORE = false, class CRec = const double*>
__device__ __forceinline__ void solve_edge(const DevParams& P, const CRec cL, const CRec cR,
                                           int wL, int wR, EdgeW<M>& W, int& lost, double* st = nullptr,
                                           long long sstride = 0) {
  auto put = [&](int k, double v) {
    if constexpr (STORE) st[(long long)k * sstride] = v;
  };
  using R = Rec<M>;
  const double g = P.g;
#pragma unroll
  for (int p = 0; p < 2 * M; ++p) {
    W.s[p] = 0.0;
#pragma unroll
    for (int m = 0; m < M; ++m) W.mass[m][p] = 0.0;
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    W.z[m] = 0.0; W.us[m] = 0.0; W.vh[m] = 0.0; W.t0[m] = 0.0; W.t1[m] = 0.0; W.hbt[m] = 0.0; W.muk[m] = 0.0;
  }
  W.wall = 0;

  double d0[M], d1[M], d2[M], hb[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const double hL = cL[3 * m], hR = cR[3 * m];
    const double hnL = cL[3 * m + 1], hnR = cR[3 * m + 1];
    hb[m] = 0.5 * (hL + hR);
    double coup = cR[R::ETA + m] - cL[R::ETA + m];
#pragma unroll
    for (int n = 0; n < m; ++n) coup += density_ratio<M>(P, n, m) * (cR[3 * n] - cL[3 * n]);
    d0[m] = hnR - hnL;
    // hn u = (sqrt(h) u)^2 and hn v = (sqrt(h) u)(sqrt(h) v) from the records
    const double wL = cL[R::UN + 2 * m], wR = cR[R::UN + 2 * m];
    d1[m] = (wR * wR - wL * wL) + g * hb[m] * coup;
    d2[m] = wR * cR[R::UN + 2 * m + 1] - wL * cL[R::UN + 2 * m + 1];
  }
  const int full = (1 << M) - 1;
  if constexpr (M == 2) if (wL == full && wR == full) {
    // ---- coupled two-layer branch ----
    const double c1 = g * hb[0], c2 = g * hb[1];
    // one reciprocal for the Roe weights of both layers, the depth sum and c1
    double den4[4] = {cL[R::SQ] + cR[R::SQ], cL[R::SQ + 1] + cR[R::SQ + 1], hb[0] + hb[1], c1}, inv4[4];
    batched_reciprocal<4>(den4, inv4);
    put(FwdRec::IS0, inv4[0]);
    put(FwdRec::IS1, inv4[1]);
    put(FwdRec::IH, inv4[2]);
    put(FwdRec::IC1, inv4[3]);
    double uh[2], vh[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      uh[m] = (cL[R::UN + 2 * m] + cR[R::UN + 2 * m]) * inv4[m];
      vh[m] = (cL[R::UN + 2 * m + 1] + cR[R::UN + 2 * m + 1]) * inv4[m];
    }
    const double ubar = (hb[0] * uh[0] + hb[1] * uh[1]) * inv4[2];
    const double dc = c1 - c2;
    // X, mu_+ and mu_- are positive normal numbers here (both layers wet: c1, c2 > 0), where
    // the iteration holds for any exponent: no range branch. (A branch at these three calls
    // made the recording form of the kernel (STORE) round the surrounding arithmetic
    // differently from the plain one; recorded steps must equal plain steps bit for bit.)
    const double c12 = c1 * c2;
    const double X = dc * dc + P.four_r * c12;
    const double rX = rsqrt2_iter(X);
    const double disc = X * rX;
    const double csum = c1 + c2;
    // mu_+ mu_- = (1 - r) c1 c2: mu_- without the cancellation of (csum - disc)/2
    const double mup = 0.5 * (csum + disc);
    const double tp = rsqrt2_iter(mup);
    const double sp = mup * tp;
    const double mum = (P.omr * c12) * (tp * tp);
    const double rmum = rsqrt2_iter(mum);
    const double sm = mum * rmum;
    double lam[4] = {ubar - sp, ubar - sm, ubar + sm, ubar + sp};
    put(FwdRec::IDISC, rX);
    put(FwdRec::ISP, tp);
    put(FwdRec::ISM, rmum);
#pragma unroll
    for (int p = 0; p < 4; ++p) put(FwdRec::LAM0 + p, lam[p]);
    const double du = uh[0] - uh[1];
    const bool lst = du * du >= P.omr_g * (hb[0] + hb[1]);
    lost += lst ? 1 : 0;
    const bool newton = !lst && P.eigen == 0;
    put(FwdRec::NEWTON, newton ? 1.0 : 0.0);
    if (newton) {
      const double rc = P.r * c12;
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        if (it == 1) {
#pragma unroll
          for (int p = 0; p < 4; ++p) put(FwdRec::LAM1 + p, lam[p]);
        }
        double Pl[4], dP[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const double a1 = lam[p] - uh[0], a2 = lam[p] - uh[1];
          const double f1 = a1 * a1 - c1, f2 = a2 * a2 - c2;
          Pl[p] = f1 * f2 - rc;
          dP[p] = a1 * f2 + a2 * f1;  // P'(l) / 2
        }
        // The four Newton quotients 1/P'(lambda_p) = (1/2) / dP_p by second-order reciprocals
        // (the quotient multiplies the correction P / P').
        double q[4];
        half_reciprocal2_group<4>(dP, q);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          lam[p] -= Pl[p] * q[p];
          put((it == 0 ? FwdRec::ID0 : FwdRec::ID1) + p, q[p]);
        }
      }
    } else {
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        put(FwdRec::LAM1 + p, lam[p]);
        put(FwdRec::ID0 + p, 0.0);
        put(FwdRec::ID1 + p, 0.0);
      }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) put(FwdRec::LAM + p, lam[p]);
    // Wave strengths. With a(l) = (l^2 + p1 l + p0) / c1 (p1 = -2 u1, p0 = u1^2 - c1) the rows
    // of R beta = delta give the power moments m_k = sum_p beta_p l_p^k, k = 0..3, and
    // beta_p follows from the Lagrange basis of the four eigenvalues.
    const double p1 = -2.0 * uh[0], p0 = uh[0] * uh[0] - c1;
    const double m0 = d0[0], m1 = d1[0];
    const double m2 = c1 * d0[1] - p1 * m1 - p0 * m0;
    const double m3 = c1 * d1[1] - p1 * m2 - p0 * m1;
    const double ic1 = inv4[3];
    const double l01 = lam[0] - lam[1], l02 = lam[0] - lam[2], l03 = lam[0] - lam[3];
    const double l12 = lam[1] - lam[2], l13 = lam[1] - lam[3], l23 = lam[2] - lam[3];
    double den[4];
    den[0] = l01 * l02 * l03;
    den[1] = -l01 * l12 * l13;
    den[2] = l02 * l12 * l23;
    den[3] = -l03 * l13 * l23;
    double iden[4];
    batched_reciprocal<4>(den, iden);
    // Numerators: prod_{q != p}(x - l_q) = Q(x)/(x - l_p), Q(x) = x^4 - S1 x^3 + S2 x^2 - S3 x + S4,
    // by synthetic division: coefficients 1, l_p - S1, S2 + l_p (l_p - S1), l_p (...) - S3.
    const double s01 = lam[0] + lam[1], s23 = lam[2] + lam[3];
    const double q0 = lam[0] * lam[1], q1 = lam[2] * lam[3];
    const double S1 = s01 + s23, S2 = q0 + q1 + s01 * s23, S3 = q0 * s23 + q1 * s01;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const double k2 = lam[p] - S1;
      const double k1 = S2 + lam[p] * k2;
      const double k0 = lam[p] * k1 - S3;
      const double num = m3 + k2 * m2 + k1 * m1 + k0 * m0;
      const double beta = num * iden[p];
      put(FwdRec::IDEN + p, iden[p]);
      put(FwdRec::BETA + p, beta);
      const double al = lam[p] - uh[0];
      const double alpha = (al * al - c1) * ic1;
      W.mass[0][p] = beta;
      W.mass[M - 1][p] = beta * alpha;
      W.s[p] = lam[p];
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      W.z[m] = d2[m] - vh[m] * d0[m];
      W.us[m] = uh[m];
      W.vh[m] = vh[m];
      W.t0[m] = d0[m];
      W.t1[m] = d1[m];
      W.hbt[m] = hb[m];
    }
    return;
  }
  if constexpr (M >= 3) {
    if (wL == full && wR == full) {
      coupled_general<M>(P, cL, cR, hb, d0, d1, d2, W, lost);
      return;
    }
  }
  // ---- per-layer branch ----
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int pa = m;
    const int pb = 2 * M - 1 - m;
    const bool wl = (wL >> m) & 1, wr = (wR >> m) & 1;
    const double hL = cL[3 * m], hR = cR[3 * m];
    if (wl && wr) {
      const double sl = cL[R::SQ + m], sr = cR[R::SQ + m];
      const double inv = rcp_fast(sl + sr);
      const double uh = (cL[R::UN + 2 * m] + cR[R::UN + 2 * m]) * inv;
      const double vh = (cL[R::UN + 2 * m + 1] + cR[R::UN + 2 * m + 1]) * inv;
      // one reciprocal square root gives c = sqrt(g hbar) and 1/(s2 - s1) = 1/(2c)
      const double gh = g * hb[m];
      const double tc = rsqrt_fast(gh);
      const double ch = gh * tc;
      split_single<M>(m, pa, pb, d0[m], d1[m], d2[m], uh - ch, uh + ch, vh, uh, W, 0.5 * tc);
      W.hbt[m] = hb[m];
    } else if (wl || wr) {
      const CRec cw = wl ? cL : cR;
      const CRec cd = wl ? cR : cL;
      const double bhat_d = (m == M - 1) ? cd[R::BB] : cd[R::ETA + m + 1];
      if (cw[R::ETA + m] < bhat_d) {
        // Wall for this layer: mirror of the wet side, coupling dropped.
        const double hw = cw[3 * m], hnw = cw[3 * m + 1];
        const double isw = rcp_fast(cw[R::SQ + m]);  // wet side: u = (sqrt(h) u) / sqrt(h)
        const double unw = cw[R::UN + 2 * m] * isw, utw = cw[R::UN + 2 * m + 1] * isw;
        // Oriented left -> right: wet left gives (hn, -hn), wet right gives (-hn, hn).
        const double sgn = wl ? 1.0 : -1.0;
        const double e0 = -2.0 * sgn * hnw;
        const double e1 = 0.0 * hnw * unw;
        const double e2 = -2.0 * sgn * hnw * utw;
        const double ch = sqrt(g * hw);
        split_single<M>(m, pa, pb, e0, e1, e2, -ch, ch, utw, 0.0, W);
        W.wall |= 1 << (2 * m + (wl ? 1 : 0));
        W.hbt[m] = hw;
      } else {
        const double sl = cL[R::SQ + m], sr = cR[R::SQ + m];
        const double inv = rcp_fast(sl + sr);
        const double uh = (cL[R::UN + 2 * m] + cR[R::UN + 2 * m]) * inv;
        const double vh = (cL[R::UN + 2 * m + 1] + cR[R::UN + 2 * m + 1]) * inv;
        const double ch = sqrt(g * hb[m]);
        double s1, s2;
        if (wl) {
          const double c = sqrt(g * hL), u = cL[R::UN + 2 * m] * rcp_fast(cL[R::SQ + m]);
          s1 = fmin(u - c, uh - ch);
          s2 = u + 2.0 * c;
        } else {
          const double c = sqrt(g * hR), u = cR[R::UN + 2 * m] * rcp_fast(cR[R::SQ + m]);
          s1 = u - 2.0 * c;
          s2 = fmax(u + c, uh + ch);
        }
        split_single<M>(m, pa, pb, d0[m], d1[m], d2[m], s1, s2, vh, uh, W);
        W.hbt[m] = hb[m];
      }
    }
  }
}

// ---- transverse split of the unsplit step ----
// The fluctuation dq (normal-frame order (h, hn, ht) per layer) that an edge sends into one
// of its cells is split into the waves of the transverse direction, at the state the edge
// was solved at: per layer the depth hb, the normal Roe velocity un and the transverse one
// ut. The transverse system is the normal one with un and ut exchanged: acoustic eigenvalues
// mu_p of the (h, ht) block, eigenvectors (dh_m, un_m dh_m, mu_p dh_m), and a shear wave
// in hn_m with speed ut_m whose strength is what the acoustic waves leave of hn
// (dq_hn - un dq_h: the acoustic waves carry the whole depth change). up gathers mu beta r
// of the waves with mu > 0, dn those with mu < 0.

// Eigen data of a coupled two-layer edge in the transverse direction: eigenvalues (closed-form
// guesses for equal velocities, two Newton steps on the quartic unless hyperbolicity is lost
// or P.eigen = 1), and what the strengths of any dq need (Lagrange denominators of the
// eigenvalues, their elementary symmetric sums, the coefficients of a(mu)).
struct TransEig2 {
  double mu[4], iden[4], S1, S2, S3, c1, p1, p0, ic1;
};

__device__ __forceinline__ void trans_eigen2(const DevParams& P, const double* hb, const double* ut, TransEig2& E) {
  const double g = P.g;
  const double c1 = g * hb[0], c2 = g * hb[1];
  double den2[2] = {hb[0] + hb[1], c1}, inv2[2];
  batched_reciprocal<2>(den2, inv2);
  const double ubar = (hb[0] * ut[0] + hb[1] * ut[1]) * inv2[0];
  const double dc = c1 - c2;
  const double c12 = c1 * c2;
  const double X = dc * dc + P.four_r * c12;
  const double disc = X * rsqrt_fast(X);
  const double mup = 0.5 * ((c1 + c2) + disc);
  const double tp = rsqrt_fast(mup);
  const double sp = mup * tp;
  const double mum = (P.omr * c12) * (tp * tp);
  const double sm = mum * rsqrt_fast(mum);
  double lam[4] = {ubar - sp, ubar - sm, ubar + sm, ubar + sp};
  const double du = ut[0] - ut[1];
  const bool lst = du * du >= P.omr_g * (hb[0] + hb[1]);
  if (!lst && P.eigen == 0) {
    const double rc = P.r * c12;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      double Pl[4], dP[4], q[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const double a1 = lam[p] - ut[0], a2 = lam[p] - ut[1];
        const double f1 = a1 * a1 - c1, f2 = a2 * a2 - c2;
        Pl[p] = f1 * f2 - rc;
        dP[p] = a1 * f2 + a2 * f1;  // P'(l) / 2
      }
      half_reciprocal2_group<4>(dP, q);  // 1/P': its error only scales the correction
#pragma unroll
      for (int p = 0; p < 4; ++p) lam[p] -= Pl[p] * q[p];
    }
  }
  const double l01 = lam[0] - lam[1], l02 = lam[0] - lam[2], l03 = lam[0] - lam[3];
  const double l12 = lam[1] - lam[2], l13 = lam[1] - lam[3], l23 = lam[2] - lam[3];
  double den[4] = {l01 * l02 * l03, -l01 * l12 * l13, l02 * l12 * l23, -l03 * l13 * l23};
  batched_reciprocal<4>(den, E.iden);
  const double s01 = lam[0] + lam[1], s23 = lam[2] + lam[3];
  const double q0 = lam[0] * lam[1], q1 = lam[2] * lam[3];
  E.S1 = s01 + s23;
  E.S2 = q0 + q1 + s01 * s23;
  E.S3 = q0 * s23 + q1 * s01;
#pragma unroll
  for (int p = 0; p < 4; ++p) E.mu[p] = lam[p];
  E.c1 = c1;
  E.ic1 = inv2[1];
  E.p1 = -2.0 * ut[0];
  E.p0 = ut[0] * ut[0] - c1;
}

// Adds speed * (v_h, un v_h, speed v_h) to fields f .. f+2 of up (speed > 0) or dn (speed <
// 0). f is a compile-time constant after unrolling, so up and dn stay in registers.
__device__ __forceinline__ void trans_send(double speed, double v_h, double un, double* up, double* dn, int f) {
  const int sc = sign_class(speed);
  const double a = speed * v_h, b = speed * (un * v_h), c = speed * (speed * v_h);
  if (sc > 0) { up[f] += a; up[f + 1] += b; up[f + 2] += c; }
  else if (sc < 0) { dn[f] += a; dn[f + 1] += b; dn[f + 2] += c; }
}

__device__ __forceinline__ void trans_shear(double ut, double z, double* up, double* dn, int f) {
  const int sc = sign_class(ut);
  const double a = ut * z;
  if (sc > 0) up[f] += a;
  else if (sc < 0) dn[f] += a;
}

// Coupled two-layer edge: strengths from the moments of the (h, ht) rows (the normal solve's
// Vandermonde form with ut in place of un), then the parts towards +t and -t.
__device__ __forceinline__ void trans_apply2(const TransEig2& E, const double* un, const double* ut,
                                             const double* dq, double* up, double* dn) {
#pragma unroll
  for (int f = 0; f < 6; ++f) { up[f] = 0.0; dn[f] = 0.0; }
  const double m0 = dq[0], m1 = dq[2];
  const double m2 = E.c1 * dq[3] - E.p1 * m1 - E.p0 * m0;
  const double m3 = E.c1 * dq[5] - E.p1 * m2 - E.p0 * m1;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const double mu = E.mu[p];
    const double k2 = mu - E.S1;
    const double k1 = E.S2 + mu * k2;
    const double k0 = mu * k1 - E.S3;
    const double beta = (m3 + k2 * m2 + k1 * m1 + k0 * m0) * E.iden[p];
    const double al = mu - ut[0];
    const double alpha = (al * al - E.c1) * E.ic1;
    trans_send(mu, beta, un[0], up, dn, 0);
    trans_send(mu, beta * alpha, un[1], up, dn, 3);
  }
#pragma unroll
  for (int m = 0; m < 2; ++m) trans_shear(ut[m], dq[3 * m + 1] - un[m] * dq[3 * m], up, dn, 3 * m + 1);
}

// Layers on their own (one layer, or an edge where some layer is dry on a side): speeds
// ut_m -+ sqrt(g hb_m) for every layer wet on a side (bit m of act).
template <int M>
__device__ __forceinline__ void trans_apply_layers(const DevParams& P, int act, const double* hb, const double* un,
                                                   const double* ut, const double* dq, double* up, double* dn) {
#pragma unroll
  for (int f = 0; f < 3 * M; ++f) { up[f] = 0.0; dn[f] = 0.0; }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    if (!((act >> m) & 1)) continue;
    const double gh = P.g * hb[m];
    const double tc = rsqrt_fast(gh);
    const double c = gh * tc;
    const double inv = 0.5 * tc;  // 1 / (s2 - s1)
    const double s1 = ut[m] - c, s2 = ut[m] + c;
    const double dh = dq[3 * m], dht = dq[3 * m + 2];
    const double b1 = (s2 * dh - dht) * inv;
    const double b2 = (dht - s1 * dh) * inv;
    trans_send(s1, b1, un[m], up, dn, 3 * m);
    trans_send(s2, b2, un[m], up, dn, 3 * m);
    trans_shear(ut[m], dq[3 * m + 1] - un[m] * dh, up, dn, 3 * m + 1);
  }
}

// Coupled edge of M >= 3 layers: the transverse eigenvalues are the roots of
// det(diag((mu - ut_m)^2) - G) with the same G as the normal solve, so the guesses reuse its
// eigenvalues mu_k of G around the transverse mean velocity; then general_eig's Newton steps
// and eigenvectors, and the 2M x 2M elimination for the strengths of each fluctuation.
template <int M>
__device__ __forceinline__ void trans_apply_general(const DevParams& P, const double* hb, const double* un,
                                                    const double* ut, const double* muk, const double* dqa,
                                                    const double* dqb, double* upa, double* dna, double* upb,
                                                    double* dnb) {
  constexpr int N = 2 * M;
  double G[M][M], lam[N], dh[N][M];
  coupling_matrix<M>(P, hb, G);
  general_eig<M>(P, G, ut, hb, muk, lam, dh);
  // one elimination of the eigenvector matrix for the strengths of both fluctuations
  double Rm[N][N], rhs[2][N], beta[2][N];
#pragma unroll
  for (int p = 0; p < N; ++p)
#pragma unroll
    for (int m = 0; m < M; ++m) {
      Rm[2 * m][p] = dh[p][m];
      Rm[2 * m + 1][p] = lam[p] * dh[p][m];
    }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    rhs[0][2 * m] = dqa[3 * m]; rhs[0][2 * m + 1] = dqa[3 * m + 2];
    rhs[1][2 * m] = dqb[3 * m]; rhs[1][2 * m + 1] = dqb[3 * m + 2];
  }
  gauss_solve_multi<N, 2>(Rm, rhs, beta);
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    const double* dq = v == 0 ? dqa : dqb;
    double* up = v == 0 ? upa : upb;
    double* dn = v == 0 ? dna : dnb;
#pragma unroll
    for (int f = 0; f < 3 * M; ++f) { up[f] = 0.0; dn[f] = 0.0; }
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
      for (int m = 0; m < M; ++m) trans_send(lam[p], beta[v][p] * dh[p][m], un[m], up, dn, 3 * m);
#pragma unroll
    for (int m = 0; m < M; ++m) trans_shear(ut[m], dq[3 * m + 1] - un[m] * dq[3 * m], up, dn, 3 * m + 1);
  }
}

}  // namespace mlswe
