// Multilayer shallow-water AMR: FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow reference that the
// CUDA library is checked against. Only tests/, the smoke check and the CPU
// baseline leg of bench.py load it. It shares no code with the CUDA library.
//
// Paper: Schwarzschild & Mandli, "An Implementation of Adaptive Mesh
// Refinement for Shallow Water Equations" (arXiv:1803.01450).
//   Sec. 2, Eqs. (1)-(2)   level spacing  dx^{l+1} = dx^l / r_x^l
//   Sec. 2.1, Eq. (3)      eta = h + B
//   Sec. 2.1, Eq. (4)      eta_{m,k} = B_k + h_{M,k} + ... + h_{m,k}
//   Sec. 2.1, Eq. (5)      effective bathymetry Bhat_{m,k} = sum_{n>m} h_{n,k} + B_k
//   Sec. 2.1, Eq. (10)     sigma_k = minmod(eta_k - eta_{k-1}, eta_{k+1} - eta_k) / dx
//   Sec. 2.1 (last para)   bottom-up layer loop of the refinement
//   Sec. 2.1 (first para)  top-down wet rule: a layer is wet only if all layers above are
//   Sec. 2.2, Eq. (11)     coarsening: fine cells averaged onto the coarse cell, all components
//
// The paper does not write out the per-patch solver (Sec. 1 cites the
// multilayer GeoClaw solver without equations). The finite-volume step here is
// this project's reading: an f-wave Riemann solver with the non-conservative
// layer coupling folded into the momentum flux jump, Godunov dimensional
// splitting (x sweep, then y sweep), an MC-limited second-order wave
// correction and a positivity fix. Every choice is listed in the design notes
// and is shared, as a specification only, with the CUDA path.
//
// Parity pins for this file live in tests/test_oracle_*.py.
//
// Storage used throughout: a "line" or "patch" array holds 3M conserved fields
// per cell in the order (h_1, hu_1, hv_1, h_2, hu_2, hv_2); layer 1 is the top
// layer (Sec. 2.1). Patch arrays carry a ghost ring of NG = 2 cells and are
// stored field-major: q[f][j + 2][i + 2], row length nx + 4.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#include <omp.h>

namespace {

constexpr int NG = 2;
constexpr int MAXM = 4;
constexpr int MAXF = 3 * MAXM;
constexpr int MAXW = 3 * MAXM;

struct Params {
  int M;          // number of layers, 1 .. MAXM
  double g;       // gravity
  double r;       // density ratio rho_1 / rho_2 (M = 2)
  double rho[MAXM];  // layer densities, top (lightest) first (M >= 3)
  double dry_tol; // a layer is wet where h > dry_tol (and every layer above is wet)
  int order;      // 1 or 2
  int limiter;    // 0 none, 1 minmod, 2 MC
  int eigen;      // 0: guesses + 2 Newton steps, 1: guesses only
  int force_general = 0;  // 1: the general coupled branch also for M = 2 (a check of it)
  int unsplit = 0;        // 1: unsplit step with transverse Riemann solves (else split)
};

// ---------------------------------------------------------------------------
// Scalar helpers written for both double and the dual number used by the
// adjoint check. Comparisons look at values only.
// ---------------------------------------------------------------------------
inline double val(double x) { return x; }

template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int k = 0; k < N; ++k) d[k] = 0.0; }
  Dual(double x) : v(x) { for (int k = 0; k < N; ++k) d[k] = 0.0; }
};
template <int N> inline double val(const Dual<N>& x) { return x.v; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> c; c.v = a.v + b.v; for (int k = 0; k < N; ++k) c.d[k] = a.d[k] + b.d[k]; return c; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> c; c.v = a.v - b.v; for (int k = 0; k < N; ++k) c.d[k] = a.d[k] - b.d[k]; return c; }
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> c; c.v = -a.v; for (int k = 0; k < N; ++k) c.d[k] = -a.d[k]; return c; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> c; c.v = a.v * b.v; for (int k = 0; k < N; ++k) c.d[k] = a.d[k] * b.v + a.v * b.d[k]; return c; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> c; c.v = a.v / b.v;
  for (int k = 0; k < N; ++k) c.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
  return c; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) { return a * Dual<N>(b); }
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) { return Dual<N>(a) * b; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> inline Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> c; c.v = std::sqrt(a.v);
  for (int k = 0; k < N; ++k) c.d[k] = a.d[k] / (2.0 * c.v);
  return c; }
using std::sqrt;

// Operation-counting scalar: every +, -, *, / and sqrt on it increments a global counter
// (used only to count the floating-point work of the method per cell update).
struct OpCount { long long add = 0, mul = 0, div = 0, sqrt = 0; };
static OpCount g_ops;
struct Cnt {
  double v;
  Cnt() : v(0.0) {}
  Cnt(double x) : v(x) {}
};
inline double val(const Cnt& x) { return x.v; }
inline Cnt operator+(const Cnt& a, const Cnt& b) { g_ops.add++; return Cnt(a.v + b.v); }
inline Cnt operator-(const Cnt& a, const Cnt& b) { g_ops.add++; return Cnt(a.v - b.v); }
inline Cnt operator-(const Cnt& a) { return Cnt(-a.v); }
inline Cnt operator*(const Cnt& a, const Cnt& b) { g_ops.mul++; return Cnt(a.v * b.v); }
inline Cnt operator/(const Cnt& a, const Cnt& b) { g_ops.div++; return Cnt(a.v / b.v); }
inline Cnt operator+(const Cnt& a, double b) { return a + Cnt(b); }
inline Cnt operator+(double a, const Cnt& b) { return Cnt(a) + b; }
inline Cnt operator-(const Cnt& a, double b) { return a - Cnt(b); }
inline Cnt operator-(double a, const Cnt& b) { return Cnt(a) - b; }
inline Cnt operator*(const Cnt& a, double b) { return a * Cnt(b); }
inline Cnt operator*(double a, const Cnt& b) { return Cnt(a) * b; }
inline Cnt operator/(const Cnt& a, double b) { return a / Cnt(b); }
inline Cnt operator/(double a, const Cnt& b) { return Cnt(a) / b; }
inline Cnt sqrt(const Cnt& a) { g_ops.sqrt++; return Cnt(std::sqrt(a.v)); }

template <class T> inline T tmin(const T& a, const T& b) { return val(b) < val(a) ? b : a; }
template <class T> inline T tmax(const T& a, const T& b) { return val(b) > val(a) ? b : a; }
template <class T> inline T tabs(const T& a) { return val(a) < 0.0 ? -a : a; }

// ---------------------------------------------------------------------------
// Riemann solver at one edge, normal direction n, transverse direction t.
// Inputs per side: (h_m, hn_m, ht_m) for each layer, and the bathymetry B.
// Output: waves Z[p][3M] with speeds s[p]; per-layer wall marks.
// ---------------------------------------------------------------------------
template <class T>
struct Waves {
  T Z[MAXW][MAXF];
  T s[MAXW];
  int nw;
  int wall_into[MAXM];  // -1 none, 0: the left cell is the dry wall side, 1: the right cell
  int hyperbolicity_lost;
  // State of the edge that the transverse solve decomposes in (per layer): the depth whose
  // gravity speed it takes, the normal and the transverse velocity; whether the layers were
  // solved together, and which layers had a wet side.
  T hbt[MAXM], unt[MAXM], utt[MAXM];
  T muk[MAXM];  // coupled edges of M >= 3 layers: the eigenvalues of the coupling matrix G
  int coupled;
  int active[MAXM];
};

// Eigenvalue guesses and Newton steps for the coupled two-layer system.
// The characteristic polynomial of the normal 4x4 system at the Roe state is
//   P(l) = ((l - u1)^2 - c1)((l - u2)^2 - c2) - r c1 c2,   c_m = g hbar_m.
// Guesses are the exact roots for u1 = u2 = ubar (mass-weighted mean):
//   l = ubar -+ sqrt(mu_+-),  mu_+- = ((c1 + c2) +- sqrt((c1 - c2)^2 + 4 r c1 c2)) / 2,
// ordered (external -, internal -, internal +, external +).
template <class T>
void two_layer_eigen(const Params& P, const T& u1, const T& u2, const T& hb1, const T& hb2,
                     T lam[4], int* lost) {
  const T c1 = P.g * hb1, c2 = P.g * hb2;
  const T ubar = (hb1 * u1 + hb2 * u2) / (hb1 + hb2);
  const T disc = sqrt((c1 - c2) * (c1 - c2) + 4.0 * P.r * c1 * c2);
  const T mup = 0.5 * ((c1 + c2) + disc);
  const T mum = 0.5 * ((c1 + c2) - disc);
  const T sp = sqrt(mup), sm = sqrt(mum);
  lam[0] = ubar - sp;
  lam[1] = ubar - sm;
  lam[2] = ubar + sm;
  lam[3] = ubar + sp;
  const T du = u1 - u2;
  *lost = val(du * du) >= val((1.0 - P.r) * P.g * (hb1 + hb2)) ? 1 : 0;
  if (*lost || P.eigen == 1) return;
  for (int p = 0; p < 4; ++p) {
    T l = lam[p];
    for (int it = 0; it < 2; ++it) {
      const T a1 = l - u1, a2 = l - u2;
      const T f1 = a1 * a1 - c1, f2 = a2 * a2 - c2;
      const T Pl = f1 * f2 - P.r * c1 * c2;
      const T dP = 2.0 * a1 * f2 + 2.0 * a2 * f1;
      l = l - Pl / dP;
    }
    lam[p] = l;
  }
}

// Dense 4x4 solve by Gaussian elimination with partial pivoting (ties: lowest row).
template <class T>
void solve4(T A[4][4], T b[4], T x[4]) {
  int perm[4] = {0, 1, 2, 3};
  for (int k = 0; k < 4; ++k) {
    int piv = k;
    for (int i = k + 1; i < 4; ++i)
      if (std::fabs(val(A[perm[i]][k])) > std::fabs(val(A[perm[piv]][k]))) piv = i;
    std::swap(perm[k], perm[piv]);
    for (int i = k + 1; i < 4; ++i) {
      const T f = A[perm[i]][k] / A[perm[k]][k];
      for (int j = k; j < 4; ++j) A[perm[i]][j] = A[perm[i]][j] - f * A[perm[k]][j];
      b[perm[i]] = b[perm[i]] - f * b[perm[k]];
    }
  }
  for (int k = 3; k >= 0; --k) {
    T s = b[perm[k]];
    for (int j = k + 1; j < 4; ++j) s = s - A[perm[k]][j] * x[j];
    x[k] = s / A[perm[k]][k];
  }
}

// Single-layer f-wave split of delta = (d0, d1, d2) on layer m with speeds s1 < s2,
// transverse velocity vhat and shear speed ushear. Writes waves pa, pb (acoustic) and
// pshear into W.
template <class T>
void single_layer_waves(int m, const T& d0, const T& d1, const T& d2, const T& s1, const T& s2,
                        const T& vhat, const T& ushear, int pa, int pb, int pshear, Waves<T>& W) {
  const T b1 = (s2 * d0 - d1) / (s2 - s1);
  const T b2 = (d1 - s1 * d0) / (s2 - s1);
  W.Z[pa][3 * m + 0] = b1; W.Z[pa][3 * m + 1] = b1 * s1; W.Z[pa][3 * m + 2] = b1 * vhat;
  W.Z[pb][3 * m + 0] = b2; W.Z[pb][3 * m + 1] = b2 * s2; W.Z[pb][3 * m + 2] = b2 * vhat;
  W.s[pa] = s1; W.s[pb] = s2;
  W.Z[pshear][3 * m + 2] = d2 - vhat * d0;
  W.s[pshear] = ushear;
}

// rho_n / rho_m: the weight of layer n's depth jump in layer m's pressure (n above m).
inline double density_ratio(const Params& P, int n, int m) {
  if (P.M == 2) return P.r;
  return P.rho[n] / P.rho[m];
}

// Dense n x n solve by Gaussian elimination with partial pivoting (ties: lowest row).
template <class T>
void solve_n(int n, T A[2 * MAXM][2 * MAXM], T b[2 * MAXM], T x[2 * MAXM]) {
  int perm[2 * MAXM];
  for (int i = 0; i < n; ++i) perm[i] = i;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(val(A[perm[i]][k])) > std::fabs(val(A[perm[piv]][k]))) piv = i;
    std::swap(perm[k], perm[piv]);
    for (int i = k + 1; i < n; ++i) {
      const T f = A[perm[i]][k] / A[perm[k]][k];
      for (int j = k; j < n; ++j) A[perm[i]][j] = A[perm[i]][j] - f * A[perm[k]][j];
      b[perm[i]] = b[perm[i]] - f * b[perm[k]];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    T sum = b[perm[k]];
    for (int j = k + 1; j < n; ++j) sum = sum - A[perm[k]][j] * x[j];
    x[k] = sum / A[perm[k]][k];
  }
}

// Determinant of the n x n matrix A with row `skip` and column `skip` removed (skip < 0:
// none), by Gaussian elimination with partial pivoting.
template <class T>
T det_minor(int n, const T A[MAXM][MAXM], int skip) {
  T B[MAXM][MAXM];
  int k = 0;
  for (int i = 0; i < n; ++i) {
    if (i == skip) continue;
    int l = 0;
    for (int j = 0; j < n; ++j) {
      if (j == skip) continue;
      B[k][l++] = A[i][j];
    }
    ++k;
  }
  T det = T(1.0);
  for (int c = 0; c < k; ++c) {
    int piv = c;
    for (int i = c + 1; i < k; ++i)
      if (std::fabs(val(B[i][c])) > std::fabs(val(B[piv][c]))) piv = i;
    if (piv != c) {
      for (int j = 0; j < k; ++j) std::swap(B[c][j], B[piv][j]);
      det = -det;
    }
    det = det * B[c][c];
    for (int i = c + 1; i < k; ++i) {
      const T f = B[i][c] / B[c][c];
      for (int j = c; j < k; ++j) B[i][j] = B[i][j] - f * B[c][j];
    }
  }
  return det;
}

// Eigenvalues of the symmetric n x n matrix K by cyclic Jacobi rotations (each rotation
// zeroes one off-diagonal pair), repeated until the off-diagonal part is below 1e-30 of
// the diagonal; returned in descending order.
template <class T>
void jacobi_eigenvalues(int n, T K[MAXM][MAXM], T mu[MAXM]) {
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += val(K[i][i]) * val(K[i][i]);
      for (int j = 0; j < n; ++j)
        if (i != j) off += val(K[i][j]) * val(K[i][j]);
    }
    if (off <= 1e-30 * diag) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (val(K[p][q]) == 0.0) continue;
        // rotation angle: tan(2 phi) = 2 K_pq / (K_qq - K_pp); t = tan(phi), smaller root
        const T theta = (K[q][q] - K[p][p]) / (2.0 * K[p][q]);
        const T t = (val(theta) >= 0.0 ? T(1.0) : T(-1.0)) / (tabs(theta) + sqrt(theta * theta + 1.0));
        const T c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const T kp = K[k][p], kq = K[k][q];
          K[k][p] = c * kp - sn * kq;
          K[k][q] = sn * kp + c * kq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const T pk = K[p][k], qk = K[q][k];
          K[p][k] = c * pk - sn * qk;
          K[q][k] = sn * pk + c * qk;
        }
      }
  }
  for (int i = 0; i < n; ++i) mu[i] = K[i][i];
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (val(mu[j]) > val(mu[i])) std::swap(mu[i], mu[j]);
}

// Coupled branch for M >= 2 layers, all wet on both sides (the general form of the
// two-layer branch). For an eigenvalue l the layer depths of the eigenvector solve
//   ((l - u_m)^2) dh_m = sum_n G_mn dh_n,   G_mn = g hbar_m C_mn,
//   C_mn = 1 (n >= m: own layer and the layers below), rho_n / rho_m (n < m: lighter above),
// so the 2M eigenvalues are the roots of P(l) = det(diag((l - u_m)^2) - G). Guesses: the
// exact roots for equal velocities, l = ubar -+ sqrt(mu_k) with mu_k the eigenvalues of G
// (G = diag(g hbar / rho) S with S_mn = rho_min(m,n) symmetric, so G is similar to the
// symmetric K = W^(1/2) S W^(1/2)), then 2 Newton steps with P'(l) = sum_m 2 (l - u_m) A~_mm
// (A~_mm the diagonal cofactors of A(l) = diag((l - u_m)^2) - G). Eigenvectors: dh_1 = 1
// and rows 1 .. M-1 of A(l) dh = 0; momenta l dh. Strengths from the 2M x 2M system.
// Loss of hyperbolicity: some adjacent pair with (u_m - u_{m+1})^2 >= (1 - rho_m/rho_{m+1})
// g (hbar_m + hbar_{m+1}); then the guesses are used.
// Eigenvalues lam[0 .. 2M-1] (ascending guesses order) and eigenvector depths dh[p][m]
// (dh_1 = 1) of the coupled M-layer system with velocities uh and mean depths hbar, as
// described above; returns 1 when hyperbolicity is lost (the guesses are kept).
// mu: the eigenvalues of G (they depend on hbar and the densities only); mu_known = false
// computes them here (and returns them in mu), true takes them as given.
template <class T>
int general_eigen(const Params& P, const T uh[MAXM], const T hbar[MAXM], T lam[2 * MAXM],
                  T dh[2 * MAXM][MAXM], T mu[MAXM], bool mu_known) {
  const int M = P.M, N = 2 * M;
  const double g = P.g;
  T G[MAXM][MAXM];
  for (int m = 0; m < M; ++m)
    for (int n = 0; n < M; ++n) G[m][n] = g * hbar[m] * (n >= m ? 1.0 : density_ratio(P, n, m));
  // guesses
  if (!mu_known) {
    T K[MAXM][MAXM], wq[MAXM];
    for (int m = 0; m < M; ++m) wq[m] = sqrt(g * hbar[m] / P.rho[m]);
    for (int m = 0; m < M; ++m)
      for (int n = 0; n < M; ++n) K[m][n] = wq[m] * wq[n] * std::min(P.rho[m], P.rho[n]);
    jacobi_eigenvalues(M, K, mu);
  }
  T hsum = T(0.0), husum = T(0.0);
  for (int m = 0; m < M; ++m) { hsum = hsum + hbar[m]; husum = husum + hbar[m] * uh[m]; }
  const T ubar = husum / hsum;
  for (int k = 0; k < M; ++k) {
    const T sq = sqrt(mu[k]);
    lam[k] = ubar - sq;
    lam[N - 1 - k] = ubar + sq;
  }
  int lost = 0;
  for (int m = 0; m + 1 < M; ++m) {
    const T du = uh[m] - uh[m + 1];
    if (val(du * du) >= val((1.0 - P.rho[m] / P.rho[m + 1]) * g * (hbar[m] + hbar[m + 1]))) lost = 1;
  }
  T A[MAXM][MAXM];
  if (!lost && P.eigen == 0) {
    for (int p = 0; p < N; ++p) {
      T l = lam[p];
      for (int it = 0; it < 2; ++it) {
        for (int m = 0; m < M; ++m)
          for (int n = 0; n < M; ++n) A[m][n] = (m == n ? (l - uh[m]) * (l - uh[m]) : T(0.0)) - G[m][n];
        const T Pl = det_minor(M, A, -1);
        T dP = T(0.0);
        for (int m = 0; m < M; ++m) dP = dP + 2.0 * (l - uh[m]) * det_minor(M, A, m);
        l = l - Pl / dP;
      }
      lam[p] = l;
    }
  }
  // eigenvectors
  for (int p = 0; p < N; ++p) {
    const T l = lam[p];
    for (int m = 0; m < M; ++m)
      for (int n = 0; n < M; ++n) A[m][n] = (m == n ? (l - uh[m]) * (l - uh[m]) : T(0.0)) - G[m][n];
    dh[p][0] = T(1.0);
    // rows 0 .. M-2 for dh_1 .. dh_{M-1}: A[i][1..] x = -A[i][0]
    T S[2 * MAXM][2 * MAXM], b[2 * MAXM], x[2 * MAXM];
    for (int i = 0; i < M - 1; ++i) {
      for (int j = 1; j < M; ++j) S[i][j - 1] = A[i][j];
      b[i] = -A[i][0];
    }
    solve_n(M - 1, S, b, x);
    for (int m = 1; m < M; ++m) dh[p][m] = x[m - 1];
  }
  return lost;
}

template <class T>
void coupled_waves_general(const Params& P, T h[2][MAXM], T hn[2][MAXM], T un[2][MAXM], T ut[2][MAXM],
                           const T hbar[MAXM], const T d0[MAXM], const T d1[MAXM], const T d2[MAXM], Waves<T>& W) {
  const int M = P.M, N = 2 * M;
  T uh[MAXM], vh[MAXM];
  for (int m = 0; m < M; ++m) {
    const T sl = sqrt(h[0][m]), sr = sqrt(h[1][m]);
    uh[m] = (sl * un[0][m] + sr * un[1][m]) / (sl + sr);
    vh[m] = (sl * ut[0][m] + sr * ut[1][m]) / (sl + sr);
  }
  T lam[2 * MAXM], dh[2 * MAXM][MAXM];
  W.hyperbolicity_lost = general_eigen(P, uh, hbar, lam, dh, W.muk, false);
  // the strengths
  T R[2 * MAXM][2 * MAXM], rhs[2 * MAXM], beta[2 * MAXM];
  for (int p = 0; p < N; ++p)
    for (int m = 0; m < M; ++m) {
      R[2 * m][p] = dh[p][m];
      R[2 * m + 1][p] = lam[p] * dh[p][m];
    }
  for (int m = 0; m < M; ++m) { rhs[2 * m] = d0[m]; rhs[2 * m + 1] = d1[m]; }
  solve_n(N, R, rhs, beta);
  for (int p = 0; p < N; ++p) {
    for (int m = 0; m < M; ++m) {
      const T mass = beta[p] * dh[p][m];
      W.Z[p][3 * m] = mass;
      W.Z[p][3 * m + 1] = mass * lam[p];
      W.Z[p][3 * m + 2] = mass * vh[m];
    }
    W.s[p] = lam[p];
  }
  for (int m = 0; m < M; ++m) {
    W.Z[N + m][3 * m + 2] = d2[m] - vh[m] * d0[m];
    W.s[N + m] = uh[m];
  }
  W.coupled = 1;
  for (int m = 0; m < M; ++m) { W.hbt[m] = hbar[m]; W.unt[m] = uh[m]; W.utt[m] = vh[m]; W.active[m] = 1; }
}

template <class T>
void riemann(const Params& P, const T* qL, const T* qR, const T& BL, const T& BR, Waves<T>& W) {
  const int M = P.M;
  const double g = P.g;
  W.nw = 3 * M;
  W.hyperbolicity_lost = 0;
  for (int p = 0; p < MAXW; ++p) {
    W.s[p] = T(0.0);
    for (int f = 0; f < MAXF; ++f) W.Z[p][f] = T(0.0);
  }
  for (int m = 0; m < MAXM; ++m) {
    W.wall_into[m] = -1;
    W.hbt[m] = T(0.0); W.unt[m] = T(0.0); W.utt[m] = T(0.0); W.muk[m] = T(0.0);
    W.active[m] = 0;
  }
  W.coupled = 0;

  // Per-side cell quantities.
  T h[2][MAXM], hn[2][MAXM], ht[2][MAXM], un[2][MAXM], ut[2][MAXM], eta[2][MAXM], Bhat[2][MAXM];
  bool wet[2][MAXM];
  for (int sd = 0; sd < 2; ++sd) {
    const T* q = sd ? qR : qL;
    const T& B = sd ? BR : BL;
    for (int m = 0; m < M; ++m) {
      h[sd][m] = q[3 * m]; hn[sd][m] = q[3 * m + 1]; ht[sd][m] = q[3 * m + 2];
      // Top-down wet rule (Sec. 2.1): wet only if every layer above is wet.
      wet[sd][m] = val(h[sd][m]) > P.dry_tol && (m == 0 || wet[sd][m - 1]);
      if (wet[sd][m]) { un[sd][m] = hn[sd][m] / h[sd][m]; ut[sd][m] = ht[sd][m] / h[sd][m]; }
      else { un[sd][m] = T(0.0); ut[sd][m] = T(0.0); }
    }
    // Eq. (4): eta_m = B + h_M + ... + h_m, summed from the bottom; Eq. (5): Bhat_m = eta_{m+1}.
    T acc = B;
    for (int m = M - 1; m >= 0; --m) {
      Bhat[sd][m] = acc;
      acc = acc + h[sd][m];
      eta[sd][m] = acc;
    }
  }

  // Flux jumps with the layer coupling folded into the momentum row:
  //   d1_m = D(hn un) + g hbar_m (D eta_m + sum_{n<m} (rho_n/rho_m) D h_n)
  // (g hbar D h_m is exactly (g/2) D(h_m^2); the remaining terms are the pressure of
  // the layers below through D eta_m and of the lighter layers above).
  T d0[MAXM], d1[MAXM], d2[MAXM], hbar[MAXM];
  for (int m = 0; m < M; ++m) {
    hbar[m] = 0.5 * (h[0][m] + h[1][m]);
    T coup = eta[1][m] - eta[0][m];
    for (int n = 0; n < m; ++n) coup = coup + density_ratio(P, n, m) * (h[1][n] - h[0][n]);
    d0[m] = hn[1][m] - hn[0][m];
    d1[m] = (hn[1][m] * un[1][m] - hn[0][m] * un[0][m]) + g * hbar[m] * coup;
    d2[m] = hn[1][m] * ut[1][m] - hn[0][m] * ut[0][m];
  }

  bool all_wet = true;
  for (int m = 0; m < M; ++m) all_wet = all_wet && wet[0][m] && wet[1][m];

  if ((M >= 3 || (M == 2 && P.force_general)) && all_wet) {
    coupled_waves_general(P, h, hn, un, ut, hbar, d0, d1, d2, W);
    return;
  }
  if (M == 2 && all_wet) {
    // Coupled branch: 4 acoustic f-waves of the 4x4 normal system, plus 2 shear waves.
    T uh[2], vh[2], c[2];
    for (int m = 0; m < 2; ++m) {
      const T sl = sqrt(h[0][m]), sr = sqrt(h[1][m]);
      uh[m] = (sl * un[0][m] + sr * un[1][m]) / (sl + sr);
      vh[m] = (sl * ut[0][m] + sr * ut[1][m]) / (sl + sr);
      c[m] = g * hbar[m];
    }
    T lam[4];
    int lost = 0;
    two_layer_eigen(P, uh[0], uh[1], hbar[0], hbar[1], lam, &lost);
    W.hyperbolicity_lost = lost;
    // Right eigenvectors (1, l, a, a l), a = ((l - u1)^2 - c1) / c1.
    T alpha[4];
    for (int p = 0; p < 4; ++p) alpha[p] = ((lam[p] - uh[0]) * (lam[p] - uh[0]) - c[0]) / c[0];
    T A[4][4], rhs[4], beta[4];
    for (int p = 0; p < 4; ++p) {
      A[0][p] = T(1.0); A[1][p] = lam[p]; A[2][p] = alpha[p]; A[3][p] = alpha[p] * lam[p];
    }
    rhs[0] = d0[0]; rhs[1] = d1[0]; rhs[2] = d0[1]; rhs[3] = d1[1];
    solve4(A, rhs, beta);
    for (int p = 0; p < 4; ++p) {
      W.Z[p][0] = beta[p];
      W.Z[p][1] = beta[p] * lam[p];
      W.Z[p][2] = beta[p] * vh[0];
      W.Z[p][3] = beta[p] * alpha[p];
      W.Z[p][4] = beta[p] * alpha[p] * lam[p];
      W.Z[p][5] = beta[p] * alpha[p] * vh[1];
      W.s[p] = lam[p];
    }
    W.Z[4][2] = d2[0] - vh[0] * d0[0]; W.s[4] = uh[0];
    W.Z[5][5] = d2[1] - vh[1] * d0[1]; W.s[5] = uh[1];
    W.coupled = 1;
    for (int m = 0; m < 2; ++m) { W.hbt[m] = hbar[m]; W.unt[m] = uh[m]; W.utt[m] = vh[m]; W.active[m] = 1; }
    return;
  }

  // Decoupled branch: every layer on its own. Wave slots of layer m: m (left-going),
  // 2M - 1 - m (right-going), 2M + m (shear): M = 1 -> (0, 1, 2); M = 2 -> layer 1 (0, 3, 4),
  // layer 2 (1, 2, 5).
  for (int m = 0; m < M; ++m) {
    const int pa = m;
    const int pb = 2 * M - 1 - m;
    const int ps = 2 * M + m;
    const bool wl = wet[0][m], wr = wet[1][m];
    if (wl && wr) {
      const T sl = sqrt(h[0][m]), sr = sqrt(h[1][m]);
      const T uh = (sl * un[0][m] + sr * un[1][m]) / (sl + sr);
      const T vh = (sl * ut[0][m] + sr * ut[1][m]) / (sl + sr);
      const T ch = sqrt(g * hbar[m]);
      single_layer_waves(m, d0[m], d1[m], d2[m], uh - ch, uh + ch, vh, uh, pa, pb, ps, W);
      W.hbt[m] = hbar[m]; W.unt[m] = uh; W.utt[m] = vh; W.active[m] = 1;
    } else if (!wl && !wr) {
      // Both sides dry: no waves for this layer.
    } else {
      const int w = wl ? 0 : 1, d = 1 - w;
      if (val(eta[w][m]) < val(Bhat[d][m])) {
        // Wall for this layer only: the dry side becomes the mirror of the wet side
        // (same depth, normal momentum negated); the layer coupling is dropped.
        const T hw = h[w][m], hnw = hn[w][m], htw = ht[w][m], unw = un[w][m], utw = ut[w][m];
        T hs[2], hns[2], uns[2], uts[2];
        hs[w] = hw; hns[w] = hnw; uns[w] = unw; uts[w] = utw;
        hs[d] = hw; hns[d] = -hnw; uns[d] = -unw; uts[d] = utw;
        (void)htw;
        const T e0 = hns[1] - hns[0];
        const T e1 = hns[1] * uns[1] - hns[0] * uns[0];
        const T e2 = hns[1] * uts[1] - hns[0] * uts[0];
        const T sq = sqrt(hs[0]);
        const T uh = (sq * uns[0] + sq * uns[1]) / (sq + sq);
        const T vh = (sq * uts[0] + sq * uts[1]) / (sq + sq);
        const T ch = sqrt(g * (0.5 * (hs[0] + hs[1])));
        single_layer_waves(m, e0, e1, e2, uh - ch, uh + ch, vh, uh, pa, pb, ps, W);
        W.wall_into[m] = d;
        W.hbt[m] = 0.5 * (hs[0] + hs[1]); W.unt[m] = uh; W.utt[m] = vh; W.active[m] = 1;
      } else {
        // Flow onto a dry cell: real states, dry-front speed bound on the dry side.
        const T sl = sqrt(h[0][m]), sr = sqrt(h[1][m]);
        const T uh = (sl * un[0][m] + sr * un[1][m]) / (sl + sr);
        const T vh = (sl * ut[0][m] + sr * ut[1][m]) / (sl + sr);
        const T ch = sqrt(g * hbar[m]);
        const T cw = sqrt(g * h[w][m]);
        T s1, s2;
        if (d == 1) { s1 = tmin(un[0][m] - cw, uh - ch); s2 = un[0][m] + 2.0 * cw; }
        else { s1 = un[1][m] - 2.0 * cw; s2 = tmax(un[1][m] + cw, uh + ch); }
        single_layer_waves(m, d0[m], d1[m], d2[m], s1, s2, vh, uh, pa, pb, ps, W);
        W.hbt[m] = hbar[m]; W.unt[m] = uh; W.utt[m] = vh; W.active[m] = 1;
      }
    }
  }
}

// First-order fluctuations: A-dQ gathers left-going waves, A+dQ right-going ones,
// a wave of speed exactly 0 is split half and half. A wall layer sends nothing into
// its dry cell.
template <class T>
void fluctuations(const Params& P, const Waves<T>& W, T* amdq, T* apdq) {
  const int F = 3 * P.M;
  for (int f = 0; f < F; ++f) { amdq[f] = T(0.0); apdq[f] = T(0.0); }
  for (int p = 0; p < W.nw; ++p) {
    const double sv = val(W.s[p]);
    for (int f = 0; f < F; ++f) {
      if (sv < 0.0) amdq[f] = amdq[f] + W.Z[p][f];
      else if (sv > 0.0) apdq[f] = apdq[f] + W.Z[p][f];
      else { amdq[f] = amdq[f] + 0.5 * W.Z[p][f]; apdq[f] = apdq[f] + 0.5 * W.Z[p][f]; }
    }
  }
  for (int m = 0; m < P.M; ++m) {
    if (W.wall_into[m] == 0) for (int k = 0; k < 3; ++k) amdq[3 * m + k] = T(0.0);
    if (W.wall_into[m] == 1) for (int k = 0; k < 3; ++k) apdq[3 * m + k] = T(0.0);
  }
}

template <class T>
T limiter_phi(int kind, const T& th) {
  if (kind == 0) return T(1.0);
  if (kind == 1) return tmax(T(0.0), tmin(T(1.0), th));
  // MC: max(0, min((1 + theta)/2, 2, 2 theta))
  return tmax(T(0.0), tmin(tmin(0.5 * (1.0 + th), T(2.0)), 2.0 * th));
}

// Second-order correction flux at an edge, from its waves and the waves at the
// neighbouring edges (wave limiter with the upwind neighbour of each family).
template <class T>
void correction(const Params& P, const Waves<T>& W, const Waves<T>& Wleft, const Waves<T>& Wright,
                double nu, T* ftil) {
  const int F = 3 * P.M;
  for (int f = 0; f < F; ++f) ftil[f] = T(0.0);
  if (P.order < 2) return;
  for (int p = 0; p < W.nw; ++p) {
    const double sv = val(W.s[p]);
    if (sv == 0.0) continue;
    const Waves<T>& U = sv > 0.0 ? Wleft : Wright;
    T zz(0.0), zu(0.0);
    for (int f = 0; f < F; ++f) { zz = zz + W.Z[p][f] * W.Z[p][f]; zu = zu + U.Z[p][f] * W.Z[p][f]; }
    T th(0.0);
    if (val(zz) > 0.0) th = zu / zz;
    const T phi = limiter_phi(P.limiter, th);
    const T sa = tabs(W.s[p]);
    const double sg = sv > 0.0 ? 1.0 : -1.0;
    const T coef = 0.5 * sg * (1.0 - nu * sa) * phi;
    for (int f = 0; f < F; ++f) ftil[f] = ftil[f] + coef * W.Z[p][f];
  }
  for (int m = 0; m < P.M; ++m)
    if (W.wall_into[m] >= 0) for (int k = 0; k < 3; ++k) ftil[3 * m + k] = T(0.0);
}

// Positivity fix: negative depths are clipped, momentum of a thin layer is removed.
template <class T>
void positivity(const Params& P, T* q) {
  for (int m = 0; m < P.M; ++m) {
    if (val(q[3 * m]) < 0.0) q[3 * m] = T(0.0);
    if (val(q[3 * m]) <= P.dry_tol) { q[3 * m + 1] = T(0.0); q[3 * m + 2] = T(0.0); }
  }
}

// Transverse Riemann solve (unsplit form): the fluctuation dq (3M, normal-frame order
// (h, hn, ht) per layer) that an edge sends into one of its cells is split into the waves of
// the transverse direction, at the state the edge was solved at (Roe velocities unt, utt and
// depth hbt per layer). The transverse system is the normal one with the roles of the
// velocities exchanged: acoustic eigenvalues mu_p of the (h, ht) block (the same coupled
// problem with utt in place of unt), eigenvectors (dh_m, unt_m dh_m, mu_p dh_m) per layer,
// and a shear wave per layer in hn with speed utt_m. bp gathers mu beta r of the waves with
// mu > 0 (towards +t), bm those with mu < 0. Coupled edges decompose all layers together
// (two layers: the closed-form guesses plus Newton steps of the normal solve; more layers:
// the general branch), otherwise each layer with a wet side alone with speeds
// utt_m -+ sqrt(g hbt_m); a layer dry on both sides sends nothing.
template <class T>
void transverse(const Params& P, const Waves<T>& W, int nv, const T* const* dq, T* const* bp, T* const* bm) {
  // nv fluctuations of the same edge share its eigen-decomposition
  const int M = P.M, F = 3 * M;
  for (int v = 0; v < nv; ++v)
    for (int f = 0; f < F; ++f) { bp[v][f] = T(0.0); bm[v][f] = T(0.0); }
  auto send = [&](int v, const T& speed, int f, const T& amount) {
    const double sv = val(speed);
    if (sv > 0.0) bp[v][f] = bp[v][f] + speed * amount;
    else if (sv < 0.0) bm[v][f] = bm[v][f] + speed * amount;
  };
  if (W.coupled) {
    const int N = 2 * M;
    T mu[2 * MAXM], dh[2 * MAXM][MAXM];
    if (M == 2 && !P.force_general) {
      int lost = 0;
      two_layer_eigen(P, W.utt[0], W.utt[1], W.hbt[0], W.hbt[1], mu, &lost);
      const T c1 = P.g * W.hbt[0];
      for (int p = 0; p < 4; ++p) {
        dh[p][0] = T(1.0);
        dh[p][1] = ((mu[p] - W.utt[0]) * (mu[p] - W.utt[0]) - c1) / c1;
      }
    } else {
      // G and so its eigenvalues are the normal solve's: only the velocities differ
      T muk[MAXM];
      for (int m = 0; m < M; ++m) muk[m] = W.muk[m];
      general_eigen(P, W.utt, W.hbt, mu, dh, muk, true);
    }
    for (int v = 0; v < nv; ++v) {
      // strengths from the (h, ht) rows: sum_p beta_p (dh_m, mu_p dh_m) = (dq_h, dq_ht)_m
      T R[2 * MAXM][2 * MAXM], rhs[2 * MAXM], beta[2 * MAXM];
      for (int p = 0; p < N; ++p)
        for (int m = 0; m < M; ++m) { R[2 * m][p] = dh[p][m]; R[2 * m + 1][p] = mu[p] * dh[p][m]; }
      for (int m = 0; m < M; ++m) { rhs[2 * m] = dq[v][3 * m]; rhs[2 * m + 1] = dq[v][3 * m + 2]; }
      solve_n(N, R, rhs, beta);
      // shear strength: what the acoustic waves leave of hn; they carry the whole depth
      // change dq_h of every layer (the h rows of the system) and un dq_h of hn
      for (int m = 0; m < M; ++m) {
        for (int p = 0; p < N; ++p) {
          const T a = beta[p] * dh[p][m];
          send(v, mu[p], 3 * m, a);
          send(v, mu[p], 3 * m + 1, W.unt[m] * a);
          send(v, mu[p], 3 * m + 2, mu[p] * a);
        }
        send(v, W.utt[m], 3 * m + 1, dq[v][3 * m + 1] - W.unt[m] * dq[v][3 * m]);
      }
    }
    return;
  }
  for (int m = 0; m < M; ++m) {
    if (!W.active[m]) continue;
    const T c = sqrt(P.g * W.hbt[m]);
    const T s1 = W.utt[m] - c, s2 = W.utt[m] + c;
    for (int v = 0; v < nv; ++v) {
      const T b1 = (s2 * dq[v][3 * m] - dq[v][3 * m + 2]) / (s2 - s1);
      const T b2 = (dq[v][3 * m + 2] - s1 * dq[v][3 * m]) / (s2 - s1);
      send(v, s1, 3 * m, b1); send(v, s1, 3 * m + 1, W.unt[m] * b1); send(v, s1, 3 * m + 2, s1 * b1);
      send(v, s2, 3 * m, b2); send(v, s2, 3 * m + 1, W.unt[m] * b2); send(v, s2, 3 * m + 2, s2 * b2);
      send(v, W.utt[m], 3 * m + 1, dq[v][3 * m + 1] - W.unt[m] * dq[v][3 * m]);
    }
  }
}

// One 1-D sweep along a line of n cells with two ghost cells at each end.
// line[(k)*F + f] for k in [0, n + 4) holds cell k - 2 in (h, hn, ht) order per layer.
// Writes out[i*F + f] for cells i in [0, n). Returns the largest wave speed at the
// edges i - 1/2, i in [0, n], and (optionally) the mass flux of every layer there.
template <class T>
double sweep_line(const Params& P, int n, const T* line, const T* Bline, double nu, T* out,
                  T* massflux /*[(n+1)*M] or null*/, int* lost_count) {
  const int F = 3 * P.M;
  // Edges e = i - 1/2 for i in [-1, n + 1]: index k = i + 1 in [0, n + 2].
  std::vector<Waves<T>> W(n + 3);
  for (int k = 0; k < n + 3; ++k) {
    const int i = k - 1;  // cells i - 1 and i, stored at i + 1 and i + 2
    riemann(P, &line[(i + 1) * F], &line[(i + 2) * F], Bline[i + 1], Bline[i + 2], W[k]);
  }
  double smax = 0.0;
  std::vector<T> amdq((n + 1) * F), apdq((n + 1) * F), ftil((n + 1) * F);
  for (int i = 0; i <= n; ++i) {
    const int k = i + 1;
    fluctuations(P, W[k], &amdq[i * F], &apdq[i * F]);
    correction(P, W[k], W[k - 1], W[k + 1], nu, &ftil[i * F]);
    for (int p = 0; p < W[k].nw; ++p) smax = std::max(smax, std::fabs(val(W[k].s[p])));
    if (lost_count) *lost_count += W[k].hyperbolicity_lost;
    if (massflux) {
      // Flux through edge i - 1/2 as seen from the left cell i - 1.
      for (int m = 0; m < P.M; ++m)
        massflux[i * P.M + m] = line[(i + 1) * F + 3 * m + 1] + amdq[i * F + 3 * m] + ftil[i * F + 3 * m];
    }
  }
  for (int i = 0; i < n; ++i) {
    T q[MAXF];
    for (int f = 0; f < F; ++f) {
      q[f] = line[(i + 2) * F + f]
             - nu * (apdq[i * F + f] + amdq[(i + 1) * F + f])
             - nu * (ftil[(i + 1) * F + f] - ftil[i * F + f]);
    }
    positivity(P, q);
    for (int f = 0; f < F; ++f) out[i * F + f] = q[f];
  }
  return smax;
}

inline size_t pidx(int nx, int i, int j) { return (size_t)(j + NG) * (nx + 2 * NG) + (i + NG); }

// Wall ghost cells on all four sides: mirror the state, negate the normal momentum of
// every layer, mirror B. x ghosts of the interior rows first, then full-width y ghost rows
// (corners therefore carry both negations).
template <class T>
void fill_walls_t(int M, int nx, int ny, T* q, T* B, int sides /*bit0 W, bit1 E, bit2 S, bit3 N*/) {
  const int F = 3 * M;
  const size_t plane = (size_t)(nx + 2 * NG) * (ny + 2 * NG);
  for (int j = 0; j < ny; ++j)
    for (int gI = 1; gI <= NG; ++gI) {
      if (sides & 1) {
        const int dst = -gI, src = gI - 1;
        for (int f = 0; f < F; ++f) {
          const double sgn = (f % 3 == 1) ? -1.0 : 1.0;
          q[f * plane + pidx(nx, dst, j)] = sgn * q[f * plane + pidx(nx, src, j)];
        }
        if (B) B[pidx(nx, dst, j)] = B[pidx(nx, src, j)];
      }
      if (sides & 2) {
        const int dst = nx - 1 + gI, src = nx - gI;
        for (int f = 0; f < F; ++f) {
          const double sgn = (f % 3 == 1) ? -1.0 : 1.0;
          q[f * plane + pidx(nx, dst, j)] = sgn * q[f * plane + pidx(nx, src, j)];
        }
        if (B) B[pidx(nx, dst, j)] = B[pidx(nx, src, j)];
      }
    }
  for (int i = -NG; i < nx + NG; ++i)
    for (int gJ = 1; gJ <= NG; ++gJ) {
      if (sides & 4) {
        const int dst = -gJ, src = gJ - 1;
        for (int f = 0; f < F; ++f) {
          const double sgn = (f % 3 == 2) ? -1.0 : 1.0;
          q[f * plane + pidx(nx, i, dst)] = sgn * q[f * plane + pidx(nx, i, src)];
        }
        if (B) B[pidx(nx, i, dst)] = B[pidx(nx, i, src)];
      }
      if (sides & 8) {
        const int dst = ny - 1 + gJ, src = ny - gJ;
        for (int f = 0; f < F; ++f) {
          const double sgn = (f % 3 == 2) ? -1.0 : 1.0;
          q[f * plane + pidx(nx, i, dst)] = sgn * q[f * plane + pidx(nx, i, src)];
        }
        if (B) B[pidx(nx, i, dst)] = B[pidx(nx, i, src)];
      }
    }
}

void fill_walls_impl(int M, int nx, int ny, double* q, double* B, int sides) {
  fill_walls_t<double>(M, nx, ny, q, B, sides);
}

// One dimensionally split step on a patch whose ghost ring is filled.
// x sweep over every row j in [-2, ny + 2) (ghost rows included, so the y sweep sees
// swept ghost rows), then y sweep over the interior columns.
template <class T>
void step_patch_impl(const Params& P, int nx, int ny, double dx, double dy, double dt,
                     T* q, const T* B, double* smax, T* fx, T* fy, int* lost) {
  const int F = 3 * P.M;
  const int W = nx + 2 * NG, H = ny + 2 * NG;
  const size_t plane = (size_t)W * H;
  std::vector<T> qs(q, q + plane * F);  // q* (ghost columns keep Q^n; unused by the y sweep)
  double sx = 0.0, sy = 0.0;
  int lost_x = 0, lost_y = 0;
  #pragma omp parallel for reduction(max : sx) reduction(+ : lost_x) schedule(static)
  for (int j = -NG; j < ny + NG; ++j) {
    std::vector<T> line((nx + 4) * F), Bl(nx + 4), out(nx * F), mf((nx + 1) * P.M);
    for (int i = -NG; i < nx + NG; ++i) {
      Bl[i + NG] = B[pidx(nx, i, j)];
      for (int m = 0; m < P.M; ++m) {
        line[(i + NG) * F + 3 * m + 0] = q[(3 * m + 0) * plane + pidx(nx, i, j)];
        line[(i + NG) * F + 3 * m + 1] = q[(3 * m + 1) * plane + pidx(nx, i, j)];
        line[(i + NG) * F + 3 * m + 2] = q[(3 * m + 2) * plane + pidx(nx, i, j)];
      }
    }
    const bool interior = (j >= 0 && j < ny);
    int lc = 0;
    const double s = sweep_line(P, nx, line.data(), Bl.data(), dt / dx, out.data(),
                                (interior && fx) ? mf.data() : nullptr, &lc);
    if (interior) { sx = std::max(sx, s); lost_x += lc; }
    for (int i = 0; i < nx; ++i)
      for (int m = 0; m < P.M; ++m) {
        qs[(3 * m + 0) * plane + pidx(nx, i, j)] = out[i * F + 3 * m + 0];
        qs[(3 * m + 1) * plane + pidx(nx, i, j)] = out[i * F + 3 * m + 1];
        qs[(3 * m + 2) * plane + pidx(nx, i, j)] = out[i * F + 3 * m + 2];
      }
    if (interior && fx)
      for (int i = 0; i <= nx; ++i)
        for (int m = 0; m < P.M; ++m) fx[((size_t)m * ny + j) * (nx + 1) + i] = mf[i * P.M + m];
  }
  #pragma omp parallel for reduction(max : sy) reduction(+ : lost_y) schedule(static)
  for (int i = 0; i < nx; ++i) {
    std::vector<T> line((ny + 4) * F), Bl(ny + 4), out(ny * F), mf((ny + 1) * P.M);
    for (int j = -NG; j < ny + NG; ++j) {
      Bl[j + NG] = B[pidx(nx, i, j)];
      for (int m = 0; m < P.M; ++m) {
        // normal = hv, transverse = hu
        line[(j + NG) * F + 3 * m + 0] = qs[(3 * m + 0) * plane + pidx(nx, i, j)];
        line[(j + NG) * F + 3 * m + 1] = qs[(3 * m + 2) * plane + pidx(nx, i, j)];
        line[(j + NG) * F + 3 * m + 2] = qs[(3 * m + 1) * plane + pidx(nx, i, j)];
      }
    }
    int lc = 0;
    const double s = sweep_line(P, ny, line.data(), Bl.data(), dt / dy, out.data(),
                                fy ? mf.data() : nullptr, &lc);
    sy = std::max(sy, s);
    lost_y += lc;
    for (int j = 0; j < ny; ++j)
      for (int m = 0; m < P.M; ++m) {
        q[(3 * m + 0) * plane + pidx(nx, i, j)] = out[j * F + 3 * m + 0];
        q[(3 * m + 2) * plane + pidx(nx, i, j)] = out[j * F + 3 * m + 1];
        q[(3 * m + 1) * plane + pidx(nx, i, j)] = out[j * F + 3 * m + 2];
      }
    if (fy)
      for (int j = 0; j <= ny; ++j)
        for (int m = 0; m < P.M; ++m) fy[((size_t)m * (ny + 1) + j) * nx + i] = mf[j * P.M + m];
  }
  if (smax) { smax[0] = sx; smax[1] = sy; }
  if (lost) *lost = lost_x + lost_y;
}

// Unsplit step on a patch whose ghost ring is filled (wave propagation with transverse
// Riemann solves, the corner-transport form of the book's Ch. 21): every edge is solved on
// Q^n; an x edge (i - 1/2, j) sends ap = A+dQ - Ft into cell (i, j) and am = A-dQ + Ft into
// cell (i - 1, j) (Ft: its limited correction flux, so ap and am are what the cells receive);
// each is split by the transverse solve, and the parts moving up / down correct the y-edge
// fluxes above / below the receiving cell by -(dt / 2 dx) B+- (.) ; y edges likewise. Then
//   Q_ij -= dt/dx (ap_{i-1/2} + am_{i+1/2}) + dt/dy (bp_{j-1/2} + bm_{j+1/2})
//         + dt/dx (Gx_{i+1/2} - Gx_{i-1/2}) + dt/dy (Gy_{j+1/2} - Gy_{j-1/2})
// and the positivity fix. Rows j in [-1, ny] and columns i in [-1, nx] are solved, so that
// the corrections at the patch's own edges are complete.
template <class T>
void step_patch_unsplit_impl(const Params& P, int nx, int ny, double dx, double dy, double dt,
                             T* q, const T* B, double* smax, T* fx, T* fy, int* lost,
                             OpCount* snaps = nullptr /* counting runs: counter after each phase */) {
  const int M = P.M, F = 3 * M;
  const int PW = nx + 2 * NG, PH = ny + 2 * NG;
  const size_t plane = (size_t)PW * PH;
  const double nux = dt / dx, nuy = dt / dy;
  // x edges i - 1/2, i in [0, nx], rows j in [-1, ny]: am, ap and their transverse parts
  // (stored in (h, hu, hv) order); row r = j + 1.
  const size_t XE = (size_t)(ny + 2) * (nx + 1);
  std::vector<T> xam(XE * F), xap(XE * F), xamU(XE * F), xamD(XE * F), xapU(XE * F), xapD(XE * F);
  // y edges j - 1/2, j in [0, ny], columns i in [-1, nx]: col c = i + 1
  const size_t YE = (size_t)(nx + 2) * (ny + 1);
  std::vector<T> ybm(YE * F), ybp(YE * F), ybmR(YE * F), ybmL(YE * F), ybpR(YE * F), ybpL(YE * F);
  double sx = 0.0, sy = 0.0;
  int lost_x = 0, lost_y = 0;
  for (int dir = 0; dir < 2; ++dir) {
    const int nlines = dir == 0 ? ny + 2 : nx + 2;  // lines -1 .. n
    const int n = dir == 0 ? nx : ny;                // cells along a line
    const double nu = dir == 0 ? nux : nuy;
    #pragma omp parallel for reduction(max : sx, sy) reduction(+ : lost_x, lost_y) schedule(static)
    for (int li = 0; li < nlines; ++li) {
      const int ln = li - 1;
      std::vector<T> line((n + 4) * F), Bl(n + 4);
      for (int k = -NG; k < n + NG; ++k) {
        const size_t o = dir == 0 ? pidx(nx, k, ln) : pidx(nx, ln, k);
        Bl[k + NG] = B[o];
        for (int m = 0; m < M; ++m) {
          line[(k + NG) * F + 3 * m + 0] = q[(3 * m + 0) * plane + o];
          line[(k + NG) * F + 3 * m + 1] = q[(3 * m + (dir == 0 ? 1 : 2)) * plane + o];
          line[(k + NG) * F + 3 * m + 2] = q[(3 * m + (dir == 0 ? 2 : 1)) * plane + o];
        }
      }
      std::vector<Waves<T>> W(n + 3);
      for (int k = 0; k < n + 3; ++k) {
        const int i = k - 1;
        riemann(P, &line[(i + 1) * F], &line[(i + 2) * F], Bl[i + 1], Bl[i + 2], W[k]);
      }
      const bool interior = ln >= 0 && ln < (dir == 0 ? ny : nx);
      for (int i = 0; i <= n; ++i) {
        const int k = i + 1;
        T amdq[MAXF], apdq[MAXF], ft[MAXF], am[MAXF], ap[MAXF], u[4][MAXF];
        fluctuations(P, W[k], amdq, apdq);
        correction(P, W[k], W[k - 1], W[k + 1], nu, ft);
        for (int f = 0; f < F; ++f) { am[f] = amdq[f] + ft[f]; ap[f] = apdq[f] - ft[f]; }
        {  // am, ap: their parts towards +t and -t
          const T* in[2] = {am, ap};
          T* up[2] = {u[0], u[2]};
          T* dn[2] = {u[1], u[3]};
          transverse(P, W[k], 2, in, up, dn);
        }
        if (interior) {
          double s = 0.0;
          for (int p = 0; p < W[k].nw; ++p) s = std::max(s, std::fabs(val(W[k].s[p])));
          if (dir == 0) { sx = std::max(sx, s); lost_x += W[k].hyperbolicity_lost; }
          else { sy = std::max(sy, s); lost_y += W[k].hyperbolicity_lost; }
        }
        // back to (h, hu, hv) order
        const size_t e = (size_t)li * (n + 1) + i;
        T* dst[6];
        if (dir == 0) { dst[0] = &xam[e * F]; dst[1] = &xap[e * F]; dst[2] = &xamU[e * F]; dst[3] = &xamD[e * F];
                        dst[4] = &xapU[e * F]; dst[5] = &xapD[e * F]; }
        else { dst[0] = &ybm[e * F]; dst[1] = &ybp[e * F]; dst[2] = &ybmR[e * F]; dst[3] = &ybmL[e * F];
               dst[4] = &ybpR[e * F]; dst[5] = &ybpL[e * F]; }
        const T* src[6] = {am, ap, u[0], u[1], u[2], u[3]};
        for (int v = 0; v < 6; ++v)
          for (int m = 0; m < M; ++m) {
            dst[v][3 * m] = src[v][3 * m];
            dst[v][3 * m + (dir == 0 ? 1 : 2)] = src[v][3 * m + 1];
            dst[v][3 * m + (dir == 0 ? 2 : 1)] = src[v][3 * m + 2];
          }
      }
    }
    if (snaps) snaps[dir] = g_ops;
  }
  // Transverse correction fluxes: Gy at y edges (i, j - 1/2), j in [0, ny], i in [0, nx);
  // Gx at x edges (i - 1/2, j), i in [0, nx], j in [0, ny).
  std::vector<T> Gy((size_t)(ny + 1) * nx * F, T(0.0)), Gx((size_t)ny * (nx + 1) * F, T(0.0));
  const double hx = 0.5 * nux, hy = 0.5 * nuy;
  auto gy = [&](int i, int jj) -> T* { return &Gy[((size_t)jj * nx + i) * F]; };
  auto gx = [&](int ii, int j) -> T* { return &Gx[((size_t)j * (nx + 1) + ii) * F]; };
  for (int j = -1; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      const size_t e = (size_t)(j + 1) * (nx + 1) + i;
      // ap enters cell (i, j); am enters cell (i - 1, j); up: edge j + 1/2 (index j + 1), down: j - 1/2 (j)
      for (int side = 0; side < 2; ++side) {
        const int ci = side == 0 ? i : i - 1;
        if (ci < 0 || ci >= nx) continue;
        const T* up = side == 0 ? &xapU[e * F] : &xamU[e * F];
        const T* dn = side == 0 ? &xapD[e * F] : &xamD[e * F];
        if (j + 1 <= ny) { T* g = gy(ci, j + 1); for (int f = 0; f < F; ++f) g[f] = g[f] - hx * up[f]; }
        if (j >= 0) { T* g = gy(ci, j); for (int f = 0; f < F; ++f) g[f] = g[f] - hx * dn[f]; }
      }
    }
  for (int i = -1; i <= nx; ++i)
    for (int j = 0; j <= ny; ++j) {
      const size_t e = (size_t)(i + 1) * (ny + 1) + j;
      // bp enters cell (i, j); bm enters cell (i, j - 1); right: edge i + 1/2, left: i - 1/2
      for (int side = 0; side < 2; ++side) {
        const int cj = side == 0 ? j : j - 1;
        if (cj < 0 || cj >= ny) continue;
        const T* rt = side == 0 ? &ybpR[e * F] : &ybmR[e * F];
        const T* lt = side == 0 ? &ybpL[e * F] : &ybmL[e * F];
        if (i + 1 <= nx) { T* g = gx(i + 1, cj); for (int f = 0; f < F; ++f) g[f] = g[f] - hy * rt[f]; }
        if (i >= 0) { T* g = gx(i, cj); for (int f = 0; f < F; ++f) g[f] = g[f] - hy * lt[f]; }
      }
    }
  if (snaps) snaps[2] = g_ops;
  // mass flux of every layer through the interior edges, seen from the lower-index cell:
  // its normal momentum + (A-dQ + Ft)_h + the transverse correction flux
  if (fx)
    for (int m = 0; m < M; ++m)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
          const size_t e = (size_t)(j + 1) * (nx + 1) + i;
          fx[((size_t)m * ny + j) * (nx + 1) + i] =
              q[(3 * m + 1) * plane + pidx(nx, i - 1, j)] + xam[e * F + 3 * m] + gx(i, j)[3 * m];
        }
  if (fy)
    for (int m = 0; m < M; ++m)
      for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const size_t e = (size_t)(i + 1) * (ny + 1) + j;
          fy[((size_t)m * (ny + 1) + j) * nx + i] =
              q[(3 * m + 2) * plane + pidx(nx, i, j - 1)] + ybm[e * F + 3 * m] + gy(i, j)[3 * m];
        }
  #pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t exl = (size_t)(j + 1) * (nx + 1) + i, exr = exl + 1;
      const size_t eyb = (size_t)(i + 1) * (ny + 1) + j, eyt = eyb + 1;
      T qn[MAXF];
      for (int f = 0; f < F; ++f) {
        const size_t o = (size_t)f * plane + pidx(nx, i, j);
        qn[f] = q[o] - nux * (xap[exl * F + f] + xam[exr * F + f]) - nuy * (ybp[eyb * F + f] + ybm[eyt * F + f])
                - nux * (gx(i + 1, j)[f] - gx(i, j)[f]) - nuy * (gy(i, j + 1)[f] - gy(i, j)[f]);
      }
      positivity(P, qn);
      // written after every read of this cell's old state (the loops above read q only)
      for (int f = 0; f < F; ++f) q[(size_t)f * plane + pidx(nx, i, j)] = qn[f];
    }
  if (snaps) snaps[3] = g_ops;
  if (smax) { smax[0] = sx; smax[1] = sy; }
  if (lost) *lost = lost_x + lost_y;
}

inline double minmod(double a, double b) {
  // Sec. 2.1: the argument of smaller modulus, zero when the signs differ.
  if (a * b <= 0.0) return 0.0;
  return std::fabs(a) <= std::fabs(b) ? a : b;
}

}  // namespace

extern "C" {

struct or_params {
  int M; double g; double r; double dry_tol; int order; int limiter; int eigen;
  double rho[4];  // layer densities, top first (read for M >= 3 and by the general branch)
  int unsplit;    // 1: unsplit step with transverse Riemann solves
};

static Params to_params(const or_params* p) {
  Params P;
  P.M = p->M; P.g = p->g; P.r = p->r; P.dry_tol = p->dry_tol;
  P.order = p->order; P.limiter = p->limiter; P.eigen = p->eigen;
  for (int m = 0; m < MAXM; ++m) P.rho[m] = p->rho[m];
  P.unsplit = p->unsplit;
  return P;
}

// Waves and fluctuations at one edge (normal direction n): Z[MAXW][MAXF], s[MAXW],
// amdq[MAXF], apdq[MAXF]; info[0 .. MAXM-1] wall marks per layer, info[MAXM] the
// hyperbolicity-loss flag. general = 1 takes the general coupled branch also for M = 2.
static void riemann_out(const Params& P, const double* qL, const double* qR, double BL, double BR, double* Z,
                        double* s, double* amdq, double* apdq, int* info) {
  Waves<double> W;
  riemann(P, qL, qR, BL, BR, W);
  for (int p = 0; p < MAXW; ++p) {
    s[p] = W.s[p];
    for (int f = 0; f < MAXF; ++f) Z[p * MAXF + f] = W.Z[p][f];
  }
  fluctuations(P, W, amdq, apdq);
  for (int m = 0; m < MAXM; ++m) info[m] = W.wall_into[m];
  info[MAXM] = W.hyperbolicity_lost;
}

void or_riemann(const or_params* pp, const double* qL, const double* qR, double BL, double BR,
                double* Z, double* s, double* amdq, double* apdq, int* info) {
  riemann_out(to_params(pp), qL, qR, BL, BR, Z, s, amdq, apdq, info);
}

void or_riemann_general(const or_params* pp, const double* qL, const double* qR, double BL, double BR,
                        double* Z, double* s, double* amdq, double* apdq, int* info) {
  Params P = to_params(pp);
  P.force_general = 1;
  riemann_out(P, qL, qR, BL, BR, Z, s, amdq, apdq, info);
}

// Transverse split of dq (3M, normal-frame order) at the edge (qL, qR, BL, BR): bp, bm the
// parts moving towards +t and -t (see transverse above). general: the general coupled branch
// also for M = 2.
void or_transverse(const or_params* pp, const double* qL, const double* qR, double BL, double BR,
                   const double* dq, double* bp, double* bm, int general) {
  Params P = to_params(pp);
  P.force_general = general;
  Waves<double> W;
  riemann(P, qL, qR, BL, BR, W);
  const double* in[1] = {dq};
  double* up[1] = {bp};
  double* dn[1] = {bm};
  transverse(P, W, 1, in, up, dn);
}

void or_eigen(const or_params* pp, double u1, double u2, double hb1, double hb2, double* lam, int* lost) {
  const Params P = to_params(pp);
  two_layer_eigen(P, u1, u2, hb1, hb2, lam, lost);
}

// 1-D sweep on a line of n cells (plus 2 ghosts per end); test entry.
double or_sweep_line(const or_params* pp, int n, const double* line, const double* Bline, double nu,
                     double* out, double* massflux) {
  const Params P = to_params(pp);
  int lost = 0;
  return sweep_line(P, n, line, Bline, nu, out, massflux, &lost);
}

// Floating-point operations of one 1-D sweep over a line of n cells (two ghosts per end),
// counted with the counting scalar: out[0..3] = additions/subtractions, multiplications,
// divisions, square roots.
void or_count_sweep(const or_params* pp, int n, const double* line, const double* Bline, double nu, long long* out) {
  const Params P = to_params(pp);
  const int F = 3 * P.M;
  std::vector<Cnt> l((n + 4) * F), b(n + 4), o(n * F);
  for (int k = 0; k < (n + 4) * F; ++k) l[k] = Cnt(line[k]);
  for (int k = 0; k < n + 4; ++k) b[k] = Cnt(Bline[k]);
  g_ops = OpCount();
  int lost = 0;
  sweep_line(P, n, l.data(), b.data(), nu, o.data(), (Cnt*)nullptr, &lost);
  out[0] = g_ops.add; out[1] = g_ops.mul; out[2] = g_ops.div; out[3] = g_ops.sqrt;
}

// Floating-point operations of one unsplit step on a patch array (ghost ring filled),
// counted with the counting scalar on one thread: out[4k .. 4k+3] = additions, multiplications,
// divisions, square roots of phase k: 0 the x edges (rows -1 .. ny), 1 the y edges
// (columns -1 .. nx), 2 the transverse correction fluxes, 3 the update (and mass fluxes).
void or_count_unsplit(const or_params* pp, int nx, int ny, double dx, double dy, double dt, const double* q,
                      const double* B, long long* out) {
  Params P = to_params(pp);
  P.unsplit = 1;
  const size_t plane = (size_t)(nx + 2 * NG) * (ny + 2 * NG);
  std::vector<Cnt> qc(plane * 3 * P.M), bc(plane);
  for (size_t k = 0; k < qc.size(); ++k) qc[k] = Cnt(q[k]);
  for (size_t k = 0; k < plane; ++k) bc[k] = Cnt(B[k]);
  const int threads = omp_get_max_threads();
  omp_set_num_threads(1);  // one global counter
  g_ops = OpCount();
  OpCount snaps[4];
  int lost = 0;
  step_patch_unsplit_impl(P, nx, ny, dx, dy, dt, qc.data(), bc.data(), nullptr, (Cnt*)nullptr, (Cnt*)nullptr,
                          &lost, snaps);
  omp_set_num_threads(threads);
  OpCount prev;
  for (int k = 0; k < 4; ++k) {
    out[4 * k] = snaps[k].add - prev.add; out[4 * k + 1] = snaps[k].mul - prev.mul;
    out[4 * k + 2] = snaps[k].div - prev.div; out[4 * k + 3] = snaps[k].sqrt - prev.sqrt;
    prev = snaps[k];
  }
}

void or_fill_walls(int M, int nx, int ny, double* q, double* B, int sides) {
  fill_walls_impl(M, nx, ny, q, B, sides);
}

// One step on a patch array with a filled ghost ring; q is updated in place (interior).
// smax[2] receives the largest wave speeds of the x and y sweeps; fx [M][ny][nx+1] and
// fy [M][ny+1][nx] (either may be null) receive the mass flux of every layer at every
// interior edge. Returns the number of edges where hyperbolicity was lost.
int or_step_patch(const or_params* pp, int nx, int ny, double dx, double dy, double dt,
                  double* q, const double* B, double* smax, double* fx, double* fy) {
  const Params P = to_params(pp);
  int lost = 0;
  if (P.unsplit) step_patch_unsplit_impl(P, nx, ny, dx, dy, dt, q, B, smax, fx, fy, &lost);
  else step_patch_impl(P, nx, ny, dx, dy, dt, q, B, smax, fx, fy, &lost);
  return lost;
}

// Fixed grid with walls on all sides: fill ghosts, then one step.
int or_step_walled(const or_params* pp, int nx, int ny, double dx, double dy, double dt,
                   double* q, double* B, double* smax) {
  fill_walls_impl(pp->M, nx, ny, q, B, 15);
  return or_step_patch(pp, nx, ny, dx, dy, dt, q, B, smax, nullptr, nullptr);
}

// Refinement, Sec. 2.1 (Eqs. (4), (5), (10) and the bottom-up layer loop), in 2-D.
// qc: coarse patch array [3M][nyc+4][nxc+4] with its ghost ring filled (neighbours of
// every coarse cell in the box must be valid). Box: coarse cells [ci0, ci1) x [cj0, cj1).
// Bf: fine bathymetry for the fine cells of the box, [(cj1-cj0)*r][(ci1-ci0)*r].
// out: fine values [3M][(cj1-cj0)*r][(ci1-ci0)*r].
void or_interp_fine(const or_params* pp, int r, int nxc, int nyc, const double* qc, const double* Bc,
                    int ci0, int cj0, int ci1, int cj1, const double* Bf, double* out) {
  const Params P = to_params(pp);
  const int M = P.M;
  const size_t plane = (size_t)(nxc + 4) * (nyc + 4);
  const int nfx = (ci1 - ci0) * r, nfy = (cj1 - cj0) * r;
  const size_t fplane = (size_t)nfx * nfy;
  auto Q = [&](int f, int i, int j) { return qc[f * plane + pidx(nxc, i, j)]; };
  auto wetc = [&](int i, int j, int m) {
    for (int n = 0; n <= m; ++n) if (!(Q(3 * n, i, j) > P.dry_tol)) return false;
    return true;
  };
  auto etac = [&](int i, int j, int m) {
    double e = Bc[pidx(nxc, i, j)];
    for (int n = M - 1; n >= m; --n) e = e + Q(3 * n, i, j);
    return e;
  };
  std::vector<double> off(r);
  for (int a = 0; a < r; ++a) off[a] = (a + 0.5) / r - 0.5;
  for (int cj = cj0; cj < cj1; ++cj)
    for (int ci = ci0; ci < ci1; ++ci) {
      // Fine depths of the layers below, needed for the effective bathymetry (Eq. (5)).
      std::vector<double> hf((size_t)M * r * r, 0.0);
      for (int m = M - 1; m >= 0; --m) {  // bottom layer first (Sec. 2.1, last paragraph)
        const bool wk = wetc(ci, cj, m);
        double sx = 0.0, sy = 0.0;
        if (wk) {
          const double ek = etac(ci, cj, m);
          const double aL = wetc(ci - 1, cj, m) ? ek - etac(ci - 1, cj, m) : 0.0;
          const double aR = wetc(ci + 1, cj, m) ? etac(ci + 1, cj, m) - ek : 0.0;
          const double aS = wetc(ci, cj - 1, m) ? ek - etac(ci, cj - 1, m) : 0.0;
          const double aN = wetc(ci, cj + 1, m) ? etac(ci, cj + 1, m) - ek : 0.0;
          sx = minmod(aL, aR);  // Eq. (10) times dx: the slope in units of one coarse cell
          sy = minmod(aS, aN);
        }
        // Momentum: the same limited linear reconstruction on the conserved variables.
        double mx[2] = {0, 0}, my[2] = {0, 0}, mc[2] = {0, 0};
        for (int k = 0; k < 2 && wk; ++k) {
          const int f = 3 * m + 1 + k;
          const double c = Q(f, ci, cj);
          mc[k] = c;
          const double aL = wetc(ci - 1, cj, m) ? c - Q(f, ci - 1, cj) : 0.0;
          const double aR = wetc(ci + 1, cj, m) ? Q(f, ci + 1, cj) - c : 0.0;
          const double aS = wetc(ci, cj - 1, m) ? c - Q(f, ci, cj - 1) : 0.0;
          const double aN = wetc(ci, cj + 1, m) ? Q(f, ci, cj + 1) - c : 0.0;
          mx[k] = minmod(aL, aR);
          my[k] = minmod(aS, aN);
        }
        const double ek = wk ? etac(ci, cj, m) : 0.0;
        for (int b = 0; b < r; ++b)
          for (int a = 0; a < r; ++a) {
            const int fi = (ci - ci0) * r + a, fj = (cj - cj0) * r + b;
            const size_t fo = (size_t)fj * nfx + fi;
            double h = 0.0, hu = 0.0, hv = 0.0;
            if (wk) {
              const double ef = ek + sx * off[a] + sy * off[b];
              double bh = Bf[fo];
              for (int n = M - 1; n > m; --n) bh = bh + hf[(size_t)n * r * r + b * r + a];
              h = std::max(0.0, ef - bh);
              if (h > P.dry_tol) {
                hu = mc[0] + mx[0] * off[a] + my[0] * off[b];
                hv = mc[1] + mx[1] * off[a] + my[1] * off[b];
              }
            }
            hf[(size_t)m * r * r + b * r + a] = h;
            out[(3 * m + 0) * fplane + fo] = h;
            out[(3 * m + 1) * fplane + fo] = hu;
            out[(3 * m + 2) * fplane + fo] = hv;
          }
      }
    }
}

// Coarsening, Sec. 2.2, Eq. (11) in 2-D: every component of the coarse cell becomes the
// mean of its r x r fine cells (row-major sum, then times 1/(r r)).
// qf: [nf][nyf][nxf] (nf components), out: [nf][nyf/r][nxf/r].
void or_average_coarse(int nf, int r, int nxf, int nyf, const double* qf, double* out) {
  const int nxc = nxf / r, nyc = nyf / r;
  const double inv = 1.0 / (double)(r * r);
  for (int f = 0; f < nf; ++f)
    for (int j = 0; j < nyc; ++j)
      for (int i = 0; i < nxc; ++i) {
        double s = 0.0;
        for (int b = 0; b < r; ++b)
          for (int a = 0; a < r; ++a) s = s + qf[((size_t)f * nyf + (size_t)j * r + b) * nxf + (size_t)i * r + a];
        out[((size_t)f * nyc + j) * nxc + i] = s * inv;
      }
}

// Refinement flags from the gradient of the top surface eta_1 (Eq. (4) with m = 1):
// flag iff gx^2 + gy^2 > tol^2, central differences where both neighbours are usable
// (inside the domain, inside the level's patches and wet in layer 1), one-sided where
// only one is. q: [3M][ny][nx] dense level, B: [ny][nx], avail: [ny][nx] (1 = cell of
// the level). No fused multiply-add anywhere (compiled with -ffp-contract=off).
void or_flags(int M, int nx, int ny, const double* q, const double* B, const uint8_t* avail,
              double dry_tol, double inv_dx, double inv_dy, double tol2, uint8_t* flags) {
  const size_t plane = (size_t)nx * ny;
  auto usable = [&](int i, int j) {
    if (i < 0 || j < 0 || i >= nx || j >= ny) return false;
    const size_t c = (size_t)j * nx + i;
    return avail[c] != 0 && q[c] > dry_tol;
  };
  auto eta1 = [&](int i, int j) {
    const size_t c = (size_t)j * nx + i;
    double e = B[c];
    for (int n = M - 1; n >= 0; --n) e = e + q[(size_t)(3 * n) * plane + c];
    return e;
  };
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t c = (size_t)j * nx + i;
      flags[c] = 0;
      if (!usable(i, j)) continue;
      const double e = eta1(i, j);
      const bool l = usable(i - 1, j), rr = usable(i + 1, j), s = usable(i, j - 1), n = usable(i, j + 1);
      double gx = 0.0, gy = 0.0;
      if (l && rr) gx = (eta1(i + 1, j) - eta1(i - 1, j)) * (0.5 * inv_dx);
      else if (rr) gx = (eta1(i + 1, j) - e) * inv_dx;
      else if (l) gx = (e - eta1(i - 1, j)) * inv_dx;
      if (s && n) gy = (eta1(i, j + 1) - eta1(i, j - 1)) * (0.5 * inv_dy);
      else if (n) gy = (eta1(i, j + 1) - e) * inv_dy;
      else if (s) gy = (e - eta1(i, j - 1)) * inv_dy;
      const double g2 = gx * gx + gy * gy;
      flags[c] = g2 > tol2 ? 1 : 0;
    }
}

// Bathymetry of a coarser level: mean of the r x r cells of the next finer level
// (row-major sum, then times 1/(r r)), the same operator as Eq. (11).
void or_bathy_average(int r, int nxf, int nyf, const double* Bf, double* Bc) {
  or_average_coarse(1, r, nxf, nyf, Bf, Bc);
}

// Adjoint of one first-order, fixed-dt step on a walled grid (wet cells only), applied
// to the cotangent lam (in: d/dQ^{n+1}, out: d/dQ^n, [3M][ny][nx]) and accumulating the
// bathymetry cotangent into gB [ny][nx]. The local Jacobian of each edge is taken
// exactly by forward-mode dual numbers; its transpose is applied edge by edge.
// q: Q^n [3M][ny][nx], B [ny][nx].
void or_adjoint_step(const or_params* pp, int nx, int ny, double dx, double dy, double dt,
                     const double* qn, const double* Bd, double* lam, double* gB);

}  // extern "C"

// ---------------------------------------------------------------------------
// Adjoint (transpose of the step Jacobian) with dual numbers.
// ---------------------------------------------------------------------------
namespace {

constexpr int ND = 14;  // 6 + 6 state entries and 2 bathymetry values of one edge
using D14 = Dual<ND>;

// Jacobian of (A-dQ, A+dQ) of one edge with respect to (qL[6], qR[6], BL, BR):
// J[out 0..11][in 0..13].
void edge_jacobian(const Params& P, const double* qL, const double* qR, double BL, double BR,
                   double J[12][ND], double amdq_v[6], double apdq_v[6]) {
  const int F = 3 * P.M;
  D14 L[MAXF], R[MAXF], bl(BL), br(BR);
  for (int f = 0; f < F; ++f) {
    L[f] = D14(qL[f]); L[f].d[f] = 1.0;
    R[f] = D14(qR[f]); R[f].d[6 + f] = 1.0;
  }
  bl.d[12] = 1.0; br.d[13] = 1.0;
  Waves<D14> W;
  riemann(P, L, R, bl, br, W);
  D14 am[MAXF], ap[MAXF];
  fluctuations(P, W, am, ap);
  for (int o = 0; o < 12; ++o) for (int k = 0; k < ND; ++k) J[o][k] = 0.0;
  for (int f = 0; f < F; ++f) {
    amdq_v[f] = am[f].v; apdq_v[f] = ap[f].v;
    for (int k = 0; k < ND; ++k) { J[f][k] = am[f].d[k]; J[6 + f][k] = ap[f].d[k]; }
  }
}

// Map input slot k of an edge (L/R state entry f, or bathymetry) to the array index of the
// line it belongs to.
void adjoint_sweep_line(const Params& P, int n, const double* line, const double* Bline, double nu,
                        const double* lam_out /*[n][F]*/, double* lam_in /*[(n+4)][F]*/,
                        double* gB_line /*[n+4]*/) {
  const int F = 3 * P.M;
  // Q*_i = Q_i - nu (A+dQ_{i-1/2} + A-dQ_{i+1/2}) for i in [0, n).
  for (int i = 0; i < n; ++i)
    for (int f = 0; f < F; ++f) lam_in[(i + 2) * F + f] += lam_out[i * F + f];
  for (int i = 0; i <= n; ++i) {  // edge i - 1/2 between cells i - 1 and i
    double J[12][ND], am[6], ap[6];
    edge_jacobian(P, &line[(i + 1) * F], &line[(i + 2) * F], Bline[i + 1], Bline[i + 2], J, am, ap);
    double cot[12] = {0};
    // A-dQ at this edge enters cell i - 1, A+dQ enters cell i.
    if (i - 1 >= 0) for (int f = 0; f < F; ++f) cot[f] = -nu * lam_out[(i - 1) * F + f];
    if (i < n) for (int f = 0; f < F; ++f) cot[6 + f] = -nu * lam_out[i * F + f];
    for (int k = 0; k < ND; ++k) {
      double s = 0.0;
      for (int o = 0; o < 12; ++o) s += J[o][k] * cot[o];
      if (k < 6) { if (k < F) lam_in[(i + 1) * F + k] += s; }
      else if (k < 12) { if (k - 6 < F) lam_in[(i + 2) * F + (k - 6)] += s; }
      else if (k == 12) gB_line[i + 1] += s;
      else gB_line[i + 2] += s;
    }
  }
}

}  // namespace

// Jacobian of the first-order fluctuations of one edge, J[12][14]: rows A-dQ (6), A+dQ (6);
// columns qL (6), qR (6), BL, BR (dual numbers).
// OpenMP threads the oracle's parallel loops use (for reporting the CPU baseline).
extern "C" int or_threads() { return omp_get_max_threads(); }

extern "C" void or_edge_jacobian(const or_params* pp, const double* qL, const double* qR, double BL, double BR,
                                 double* J) {
  const Params P = to_params(pp);
  double Jm[12][ND], am[6], ap[6];
  edge_jacobian(P, qL, qR, BL, BR, Jm, am, ap);
  for (int o = 0; o < 12; ++o)
    for (int k = 0; k < ND; ++k) J[o * ND + k] = Jm[o][k];
}

extern "C" void or_adjoint_step(const or_params* pp, int nx, int ny, double dx, double dy, double dt,
                                const double* qn, const double* Bd, double* lam, double* gB) {
  Params P = to_params(pp);
  P.order = 1;
  const int F = 3 * P.M;
  const size_t plane = (size_t)nx * ny;
  // Rebuild the forward intermediates: padded Q^n with walls, and Q* with walls.
  const int W = nx + 4, H = ny + 4;
  const size_t pplane = (size_t)W * H;
  std::vector<double> qp(pplane * F), Bp(pplane);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      Bp[pidx(nx, i, j)] = Bd[(size_t)j * nx + i];
      for (int f = 0; f < F; ++f) qp[f * pplane + pidx(nx, i, j)] = qn[f * plane + (size_t)j * nx + i];
    }
  fill_walls_impl(P.M, nx, ny, qp.data(), Bp.data(), 15);
  std::vector<double> qs = qp;
  // x sweep (order 1) over all rows, as in the forward step, to rebuild Q*.
  for (int j = -NG; j < ny + NG; ++j) {
    std::vector<double> line((nx + 4) * F), Bl(nx + 4), out(nx * F);
    for (int i = -NG; i < nx + NG; ++i) {
      Bl[i + NG] = Bp[pidx(nx, i, j)];
      for (int m = 0; m < P.M; ++m)
        for (int k = 0; k < 3; ++k) line[(i + NG) * F + 3 * m + k] = qp[(3 * m + k) * pplane + pidx(nx, i, j)];
    }
    int lc = 0;
    sweep_line(P, nx, line.data(), Bl.data(), dt / dx, out.data(), (double*)nullptr, &lc);
    for (int i = 0; i < nx; ++i)
      for (int f = 0; f < F; ++f) qs[f * pplane + pidx(nx, i, j)] = out[i * F + f];
  }
  // Reverse of the y sweep: lam -> lam* on the padded Q* grid (rows -2..ny+1).
  std::vector<double> lams(pplane * F, 0.0), gBp(pplane, 0.0);
  for (int i = 0; i < nx; ++i) {
    std::vector<double> line((ny + 4) * F), Bl(ny + 4), lo(ny * F), li((ny + 4) * F, 0.0), gl(ny + 4, 0.0);
    for (int j = -NG; j < ny + NG; ++j) {
      Bl[j + NG] = Bp[pidx(nx, i, j)];
      for (int m = 0; m < P.M; ++m) {
        line[(j + NG) * F + 3 * m + 0] = qs[(3 * m + 0) * pplane + pidx(nx, i, j)];
        line[(j + NG) * F + 3 * m + 1] = qs[(3 * m + 2) * pplane + pidx(nx, i, j)];
        line[(j + NG) * F + 3 * m + 2] = qs[(3 * m + 1) * pplane + pidx(nx, i, j)];
      }
    }
    for (int j = 0; j < ny; ++j)
      for (int m = 0; m < P.M; ++m) {
        lo[j * F + 3 * m + 0] = lam[(3 * m + 0) * plane + (size_t)j * nx + i];
        lo[j * F + 3 * m + 1] = lam[(3 * m + 2) * plane + (size_t)j * nx + i];
        lo[j * F + 3 * m + 2] = lam[(3 * m + 1) * plane + (size_t)j * nx + i];
      }
    adjoint_sweep_line(P, ny, line.data(), Bl.data(), dt / dy, lo.data(), li.data(), gl.data());
    for (int j = -NG; j < ny + NG; ++j) {
      gBp[pidx(nx, i, j)] += gl[j + NG];
      for (int m = 0; m < P.M; ++m) {
        lams[(3 * m + 0) * pplane + pidx(nx, i, j)] += li[(j + NG) * F + 3 * m + 0];
        lams[(3 * m + 2) * pplane + pidx(nx, i, j)] += li[(j + NG) * F + 3 * m + 1];
        lams[(3 * m + 1) * pplane + pidx(nx, i, j)] += li[(j + NG) * F + 3 * m + 2];
      }
    }
  }
  // Reverse of the x sweep on every row: lam* (interior columns) -> cotangent of padded Q^n.
  std::vector<double> lamp(pplane * F, 0.0);
  for (int j = -NG; j < ny + NG; ++j) {
    std::vector<double> line((nx + 4) * F), Bl(nx + 4), lo(nx * F), li((nx + 4) * F, 0.0), gl(nx + 4, 0.0);
    for (int i = -NG; i < nx + NG; ++i) {
      Bl[i + NG] = Bp[pidx(nx, i, j)];
      for (int f = 0; f < F; ++f) line[(i + NG) * F + f] = qp[f * pplane + pidx(nx, i, j)];
    }
    for (int i = 0; i < nx; ++i)
      for (int f = 0; f < F; ++f) lo[i * F + f] = lams[f * pplane + pidx(nx, i, j)];
    adjoint_sweep_line(P, nx, line.data(), Bl.data(), dt / dx, lo.data(), li.data(), gl.data());
    for (int i = -NG; i < nx + NG; ++i) {
      gBp[pidx(nx, i, j)] += gl[i + NG];
      for (int f = 0; f < F; ++f) lamp[f * pplane + pidx(nx, i, j)] += li[(i + NG) * F + f];
    }
  }
  // Ghost cells of Q^n are mirrors of interior cells (x ghosts of interior rows first,
  // then y ghost rows over the full width): fold their cotangents back, in reverse order.
  for (int i = -NG; i < nx + NG; ++i)
    for (int gJ = NG; gJ >= 1; --gJ) {
      const int dN = ny - 1 + gJ, sN = ny - gJ, dS = -gJ, sS = gJ - 1;
      for (int f = 0; f < F; ++f) {
        const double sgn = (f % 3 == 2) ? -1.0 : 1.0;
        lamp[f * pplane + pidx(nx, i, sN)] += sgn * lamp[f * pplane + pidx(nx, i, dN)];
        lamp[f * pplane + pidx(nx, i, dN)] = 0.0;
        lamp[f * pplane + pidx(nx, i, sS)] += sgn * lamp[f * pplane + pidx(nx, i, dS)];
        lamp[f * pplane + pidx(nx, i, dS)] = 0.0;
      }
      gBp[pidx(nx, i, sN)] += gBp[pidx(nx, i, dN)]; gBp[pidx(nx, i, dN)] = 0.0;
      gBp[pidx(nx, i, sS)] += gBp[pidx(nx, i, dS)]; gBp[pidx(nx, i, dS)] = 0.0;
    }
  for (int j = 0; j < ny; ++j)
    for (int gI = NG; gI >= 1; --gI) {
      const int dE = nx - 1 + gI, sE = nx - gI, dW = -gI, sW = gI - 1;
      for (int f = 0; f < F; ++f) {
        const double sgn = (f % 3 == 1) ? -1.0 : 1.0;
        lamp[f * pplane + pidx(nx, sE, j)] += sgn * lamp[f * pplane + pidx(nx, dE, j)];
        lamp[f * pplane + pidx(nx, dE, j)] = 0.0;
        lamp[f * pplane + pidx(nx, sW, j)] += sgn * lamp[f * pplane + pidx(nx, dW, j)];
        lamp[f * pplane + pidx(nx, dW, j)] = 0.0;
      }
      gBp[pidx(nx, sE, j)] += gBp[pidx(nx, dE, j)]; gBp[pidx(nx, dE, j)] = 0.0;
      gBp[pidx(nx, sW, j)] += gBp[pidx(nx, dW, j)]; gBp[pidx(nx, dW, j)] = 0.0;
    }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      gB[(size_t)j * nx + i] += gBp[pidx(nx, i, j)];
      for (int f = 0; f < F; ++f) lam[f * plane + (size_t)j * nx + i] = lamp[f * pplane + pidx(nx, i, j)];
    }
}

// Tangent-linear run of the gauge misfit (forward-mode dual numbers through every step):
// J = sum_{n=1..N} sum_g (eta_1(cell_g, Q^n) - obs[n-1][g])^2 with eta_1 = (B + h_2) + h_1
// (Eq. (4)) for N walled, fixed-dt steps from Q^0, and its directional derivative along
// (dq0, dB). q0, dq0: [3M][ny][nx]; B, dB: [ny][nx]; gij: [n_g][2] (i, j); obs: [N][n_g].
extern "C" void or_tangent_loss(const or_params* pp, int nx, int ny, double dx, double dy, double dt, int n_steps,
                                const double* q0, const double* B, const double* dq0, const double* dB, int n_g,
                                const int* gij, const double* obs, double* J, double* dJ) {
  using D1 = Dual<1>;
  const Params P = to_params(pp);
  const int F = 3 * P.M;
  const int W = nx + 2 * NG, H = ny + 2 * NG;
  const size_t pplane = (size_t)W * H, plane = (size_t)nx * ny;
  std::vector<D1> q(pplane * F), Bp(pplane);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t o = (size_t)j * nx + i;
      Bp[pidx(nx, i, j)] = D1(B[o]);
      Bp[pidx(nx, i, j)].d[0] = dB[o];
      for (int f = 0; f < F; ++f) {
        q[f * pplane + pidx(nx, i, j)] = D1(q0[f * plane + o]);
        q[f * pplane + pidx(nx, i, j)].d[0] = dq0[f * plane + o];
      }
    }
  double j_val = 0.0, j_dot = 0.0;
  for (int n = 1; n <= n_steps; ++n) {
    fill_walls_t<D1>(P.M, nx, ny, q.data(), Bp.data(), 15);
    step_patch_impl<D1>(P, nx, ny, dx, dy, dt, q.data(), Bp.data(), nullptr, nullptr, nullptr, nullptr);
    for (int g = 0; g < n_g; ++g) {
      const int i = gij[2 * g], jj = gij[2 * g + 1];
      D1 eta = Bp[pidx(nx, i, jj)];
      for (int m = P.M - 1; m >= 0; --m) eta = eta + q[(3 * m) * pplane + pidx(nx, i, jj)];
      const D1 r = eta - obs[(size_t)(n - 1) * n_g + g];
      j_val += r.v * r.v;
      j_dot += 2.0 * r.v * r.d[0];
    }
  }
  *J = j_val;
  *dJ = j_dot;
}
