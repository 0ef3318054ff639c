// Host-side check of the hand-written edge vector-Jacobian products
// (paper_1803_01450_gb300/csrc/mlswe_adjoint.cuh) against the oracle's Jacobian of the
// first-order edge fluctuations, taken with forward-mode dual numbers
// (or_edge_jacobian in oracle/mlswe_oracle.cpp). Compiled as host code by nvcc; no GPU.
//
// For random wet edge states and random output cotangents (a-, a+), it compares
//   (qL_b, qR_b, BL_b, BR_b) = J^T (a-, a+)
// and prints the worst relative error per case family; exit status 1 if any exceeds the
// bound given as argv[2].
//
// usage: vjp_host_check <path of liboracle.so> <relative bound>
#include <dlfcn.h>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include "../paper_1803_01450_gb300/csrc/mlswe_adjoint.cuh"

using namespace mlswe;

struct OrParams {  // layout of the oracle's or_params
  int M;
  double g, r, dry_tol;
  int order, limiter, eigen;
  double rho[4];
  int unsplit;
};
typedef void (*JacFn)(const OrParams*, const double*, const double*, double, double, double*);

// The adjoint sweep's cell record (ARec<M>), built the way its load phase builds it.
template <int M>
static void cell_record(const double* q, double B, double tol, double* rec, int& wet) {
  using R = Rec<M>;
  wet = 0;
  bool above = true;
  for (int m = 0; m < M; ++m) {
    const double h = q[3 * m];
    rec[3 * m] = h;
    rec[3 * m + 1] = q[3 * m + 1];
    rec[3 * m + 2] = q[3 * m + 2];
    const bool w = above && h > tol;
    above = w;
    wet |= w ? (1 << m) : 0;
    rec[R::UN + 2 * m] = w ? q[3 * m + 1] / h : 0.0;
    rec[R::UN + 2 * m + 1] = w ? q[3 * m + 2] / h : 0.0;
    rec[R::SQ + m] = std::sqrt(h);
    rec[ARec<M>::IS + m] = w ? 1.0 / std::sqrt(h) : 0.0;
  }
  double eta = B;
  for (int m = M - 1; m >= 0; --m) {
    eta += rec[3 * m];
    rec[R::ETA + m] = eta;
  }
  rec[R::BB] = B;
}

// One case family: depths (d1, d2) with relative spread `spread`, velocities of scale
// `vel` (times the depth), bathymetry steps of `db`; eigen = 0 (Newton) or 1 (guesses).
template <int M>
static double family(JacFn jac, int eigen, double d1, double d2, double spread, double vel, double db,
                     double shear, int trials, unsigned seed) {
  const double g = 9.81, r = M == 2 ? 1025.0 / 1028.0 : 1.0;
  OrParams op{M, g, r, 1e-6, 1, 2, eigen, {1025.0, 1028.0, 0.0, 0.0}, 0};
  DevParams P{};
  P.M = M;
  P.g = g;
  P.r = r;
  P.rho[0] = 1025.0;
  P.rho[1] = 1028.0;
  P.dry_tol = 1e-6;
  P.order = 1;
  P.limiter = 2;
  P.eigen = eigen;
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> N01(0.0, 1.0);
  double worst = 0.0;
  for (int t = 0; t < trials; ++t) {
    double qL[6] = {0, 0, 0, 0, 0, 0}, qR[6] = {0, 0, 0, 0, 0, 0};
    const double depth[2] = {d1, d2};
    for (int m = 0; m < M; ++m) {
      qL[3 * m] = depth[m] * (1.0 + spread * N01(rng));
      qR[3 * m] = depth[m] * (1.0 + spread * N01(rng));
      const double u = (m == 0 ? shear : 0.0);  // mean shear between the layers
      for (int k = 1; k < 3; ++k) {
        qL[3 * m + k] = ((k == 1 ? u : 0.0) + vel * N01(rng)) * qL[3 * m];
        qR[3 * m + k] = ((k == 1 ? u : 0.0) + vel * N01(rng)) * qR[3 * m];
      }
    }
    const double BL = -(d1 + d2) + db * N01(rng), BR = -(d1 + d2) + db * N01(rng);
    double J[12 * 14];
    jac(&op, qL, qR, BL, BR, J);
    double amb[6] = {0, 0, 0, 0, 0, 0}, apb[6] = {0, 0, 0, 0, 0, 0};
    for (int f = 0; f < 3 * M; ++f) {
      amb[f] = N01(rng);
      apb[f] = N01(rng);
    }
    double ref[14];
    for (int k = 0; k < 14; ++k) {
      double s = 0.0;
      for (int o = 0; o < 6; ++o) s += J[o * 14 + k] * amb[o] + J[(6 + o) * 14 + k] * apb[o];
      ref[k] = s;
    }
    double cL[ARec<2>::N], cR[ARec<2>::N];
    int wL, wR;
    cell_record<M>(qL, BL, 1e-6, cL, wL);
    cell_record<M>(qR, BR, 1e-6, cR, wR);
    double qLb[6] = {0, 0, 0, 0, 0, 0}, qRb[6] = {0, 0, 0, 0, 0, 0}, BLb = 0.0, BRb = 0.0;
    const bool ok = M == 2 ? edge_vjp_2(P, cL, cR, wL, wR, amb, apb, qLb, qRb, BLb, BRb)
                           : edge_vjp_1(P, cL, cR, wL, wR, amb, apb, qLb, qRb, BLb, BRb);
    if (!ok) {
      std::printf("edge not in the wet branch\n");
      return 1.0;
    }
    double got[14] = {0};
    for (int f = 0; f < 3 * M; ++f) {
      got[f] = qLb[f];
      got[6 + f] = qRb[f];
    }
    got[12] = BLb;
    got[13] = BRb;
    double scale = 0.0, err = 0.0;
    for (int k = 0; k < 14; ++k) {
      scale = std::fmax(scale, std::fabs(ref[k]));
      err = std::fmax(err, std::fabs(got[k] - ref[k]));
    }
    worst = std::fmax(worst, err / scale);
  }
  return worst;
}

int main(int argc, char** argv) {
  if (argc < 3) {
    std::fprintf(stderr, "usage: %s liboracle.so bound\n", argv[0]);
    return 2;
  }
  void* lib = dlopen(argv[1], RTLD_NOW);
  if (!lib) {
    std::fprintf(stderr, "dlopen: %s\n", dlerror());
    return 2;
  }
  JacFn jac = (JacFn)dlsym(lib, "or_edge_jacobian");
  if (!jac) return 2;
  const double bound = std::atof(argv[2]);
  struct Fam {
    const char* name;
    double worst;
  } fams[] = {
      {"M=1 wet", family<1>(jac, 0, 0.6, 0.0, 0.1, 0.05, 0.05, 0.0, 2000, 1)},
      {"M=1 deep, strong flow", family<1>(jac, 0, 4000.0, 0.0, 0.15, 0.5, 10.0, 0.0, 2000, 2)},
      {"M=2 Newton", family<2>(jac, 0, 0.6, 0.4, 0.1, 0.05, 0.05, 0.0, 2000, 3)},
      {"M=2 Newton, ocean depths", family<2>(jac, 0, 200.0, 3800.0, 0.05, 0.01, 20.0, 0.0, 2000, 4)},
      {"M=2 Newton, sheared layers", family<2>(jac, 0, 0.6, 0.4, 0.1, 0.02, 0.05, 0.1, 2000, 5)},
      {"M=2 guesses only", family<2>(jac, 1, 0.6, 0.4, 0.1, 0.05, 0.05, 0.0, 2000, 6)},
  };
  int rc = 0;
  for (const Fam& f : fams) {
    std::printf("%-28s worst relative error %.3e\n", f.name, f.worst);
    if (!(f.worst <= bound)) rc = 1;
  }
  return rc;
}
