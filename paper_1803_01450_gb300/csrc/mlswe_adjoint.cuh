// Reverse-mode derivative (vector-Jacobian product) of the first-order edge
// fluctuations (A-dQ, A+dQ) of mlswe_device.cuh's Riemann solver, for wet
// states: the coupled two-layer branch (M = 2, both layers wet on both sides)
// and the one-layer branch (M = 1, wet on both sides). Hand-written: the
// forward quantities are recomputed, then every statement is differentiated in
// reverse order. Signs of the wave speeds select fluctuations and are treated
// as constant (the derivative of the selection is zero almost everywhere).
//
// Cell records are the forward sweep's (Rec<M>: h, hn, ht per layer, un, ut,
// sqrt(h), eta, B) followed by 1/sqrt(h) per layer (ARec<M>); bathymetry
// enters through eta. Reciprocals that share an edge are taken in batches of
// four with one division.
#pragma once
#include <cmath>
#include <cstring>
#include "mlswe_device.cuh"

namespace mlswe {

#ifdef __CUDACC__
#define MLSWE_HD __host__ __device__ __forceinline__
#else
#define MLSWE_HD inline
#endif

MLSWE_HD double adj_rcp(double x) {
#ifdef __CUDA_ARCH__
  return __drcp_rn(x);
#else
  return 1.0 / x;
#endif
}

MLSWE_HD double adj_rsqrt(double x) {
#ifdef __CUDA_ARCH__
  return rsqrt(x);
#else
  return 1.0 / std::sqrt(x);
#endif
}

MLSWE_HD long long adj_bits(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x);
#else
  long long b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}

// Sign of a wave speed from its bits (integer unit, not the FP64 pipe): -1, +1, or 0 for +-0.
MLSWE_HD int adj_sign(double s) {
  const long long b = adj_bits(s);
  return (b << 1) == 0 ? 0 : (b < 0 ? -1 : 1);
}

// |x| in [2^-199, 2^200), read from the exponent field.
MLSWE_HD bool adj_moderate(double x) {
  const unsigned e = (unsigned)((adj_bits(x) >> 52) & 0x7ff);
  return e - 824u <= 398u;
}

// Reciprocals of N <= 4 nonzero numbers with one division: 1/x_p = (1/prod x) * prod_{q != p} x_q.
// Used when every |x_p| lies in [2^-199, 2^200) (every partial product stays a normal FP64
// number); otherwise one division each.
template <int N>
MLSWE_HD void adj_batched_rcp(const double* x, double* inv) {
  bool safe = true;
  for (int p = 0; p < N; ++p) safe = safe && adj_moderate(x[p]);
  if (!safe) {
    for (int p = 0; p < N; ++p) inv[p] = adj_rcp(x[p]);
    return;
  }
  double pre[N], suf[N];
  pre[0] = 1.0;
  for (int p = 1; p < N; ++p) pre[p] = pre[p - 1] * x[p - 1];
  suf[N - 1] = 1.0;
  for (int p = N - 2; p >= 0; --p) suf[p] = suf[p + 1] * x[p + 1];
  const double ip = adj_rcp(pre[N - 1] * x[N - 1]);
  for (int p = 0; p < N; ++p) inv[p] = ip * (pre[p] * suf[p]);
}

// Cell record of the adjoint sweep: the forward record Rec<M> followed by 1/sqrt(h_m)
// (zero where layer m is not wet).
template <int M>
struct ARec {
  static constexpr int IS = Rec<M>::N;
  static constexpr int N = Rec<M>::N + M;
};

// Cotangent seen by a wave of speed s: a wave with s < 0 goes into A-dQ, s > 0 into A+dQ,
// s = 0 half into each.
template <int N>
MLSWE_HD void adj_pick(double s, const double* am_b, const double* ap_b, double* z) {
  const int sg = adj_sign(s);
  if (sg != 0) {
    for (int f = 0; f < N; ++f) z[f] = sg < 0 ? am_b[f] : ap_b[f];
  } else {
    for (int f = 0; f < N; ++f) z[f] = 0.5 * (am_b[f] + ap_b[f]);
  }
}

// Forward part of a coupled two-layer edge (M = 2, both layers wet on both sides): fills the
// record F (layout FwdRec) with what the reverse part needs. Returns false if the states are
// not in the coupled branch.
MLSWE_HD bool edge_fwd_2(const DevParams& P, const double* cL, const double* cR, int wL, int wR, double* F) {
  using R = Rec<2>;
  using FR = FwdRec;
  if (wL != 3 || wR != 3) return false;
  const double g = P.g, r = P.r;
  double hb[2], coup[2], d0[2], d1[2], uh[2];
  for (int m = 0; m < 2; ++m) {
    hb[m] = 0.5 * (cL[3 * m] + cR[3 * m]);
    coup[m] = cR[R::ETA + m] - cL[R::ETA + m];
    if (m == 1) coup[m] += r * (cR[0] - cL[0]);
    d0[m] = cR[3 * m + 1] - cL[3 * m + 1];
    d1[m] = (cR[3 * m + 1] * cR[R::UN + 2 * m] - cL[3 * m + 1] * cL[R::UN + 2 * m]) + g * hb[m] * coup[m];
  }
  const double c1 = g * hb[0], c2 = g * hb[1];
  // 1/(sqrt hL + sqrt hR) per layer, 1/(hbar_1 + hbar_2), 1/c1 in one division
  {
    const double den[4] = {cL[R::SQ] + cR[R::SQ], cL[R::SQ + 1] + cR[R::SQ + 1], hb[0] + hb[1], c1};
    adj_batched_rcp<4>(den, F + FR::IS0);
  }
  for (int m = 0; m < 2; ++m)
    uh[m] = (cL[R::SQ + m] * cL[R::UN + 2 * m] + cR[R::SQ + m] * cR[R::UN + 2 * m]) * F[FR::IS0 + m];
  const double ubar = (hb[0] * uh[0] + hb[1] * uh[1]) * F[FR::IH];
  const double dc = c1 - c2;
  const double X = dc * dc + 4.0 * r * c1 * c2;
  F[FR::IDISC] = adj_rsqrt(X);
  const double disc = X * F[FR::IDISC];
  // mu_+ = (csum + disc)/2; mu_- from mu_+ mu_- = (1 - r) c1 c2 (no cancellation)
  const double mup = 0.5 * ((c1 + c2) + disc);
  const double isp = adj_rsqrt(mup), sp = mup * isp;
  const double mum = ((1.0 - r) * c1 * c2) * (isp * isp);
  const double ism = adj_rsqrt(mum), sm = mum * ism;
  F[FR::ISP] = isp;
  F[FR::ISM] = ism;
  double lam[4] = {ubar - sp, ubar - sm, ubar + sm, ubar + sp};
  for (int p = 0; p < 4; ++p) F[FR::LAM0 + p] = lam[p];
  const double du = uh[0] - uh[1];
  const bool newton = !(du * du >= (1.0 - r) * g * (hb[0] + hb[1])) && P.eigen == 0;
  F[FR::NEWTON] = newton ? 1.0 : 0.0;
  const double rc = r * c1 * c2;
  if (newton) {
    for (int it = 0; it < 2; ++it) {
      double Pl[4], D[4];
      for (int p = 0; p < 4; ++p) {
        if (it == 1) F[FR::LAM1 + p] = lam[p];
        const double a1 = lam[p] - uh[0], a2 = lam[p] - uh[1];
        const double f1 = a1 * a1 - c1, f2 = a2 * a2 - c2;
        Pl[p] = f1 * f2 - rc;
        D[p] = 2.0 * (a1 * f2 + a2 * f1);
      }
      double* iD = F + (it == 0 ? FR::ID0 : FR::ID1);
      adj_batched_rcp<4>(D, iD);
      for (int p = 0; p < 4; ++p) lam[p] = lam[p] - Pl[p] * iD[p];
    }
  } else {
    for (int p = 0; p < 4; ++p) {
      F[FR::LAM1 + p] = lam[p];
      F[FR::ID0 + p] = 0.0;
      F[FR::ID1 + p] = 0.0;
    }
  }
  for (int p = 0; p < 4; ++p) F[FR::LAM + p] = lam[p];
  // wave strengths: Vandermonde form (see mlswe_device.cuh)
  const double p1 = -2.0 * uh[0], p0 = uh[0] * uh[0] - c1;
  const double m0 = d0[0], m1 = d1[0];
  const double m2 = c1 * d0[1] - p1 * m1 - p0 * m0;
  const double m3 = c1 * d1[1] - p1 * m2 - p0 * m1;
  double e1[4], e2[4], e3[4];
  {
    double den[4];
    for (int p = 0; p < 4; ++p) {
      const int qa = (p + 1) & 3, qb = (p + 2) & 3, qc = (p + 3) & 3;
      e1[p] = lam[qa] + lam[qb] + lam[qc];
      e2[p] = lam[qa] * lam[qb] + lam[qa] * lam[qc] + lam[qb] * lam[qc];
      e3[p] = lam[qa] * lam[qb] * lam[qc];
      den[p] = (lam[p] - lam[qa]) * (lam[p] - lam[qb]) * (lam[p] - lam[qc]);
    }
    adj_batched_rcp<4>(den, F + FR::IDEN);
  }
  for (int p = 0; p < 4; ++p)
    F[FR::BETA + p] = (m3 - e1[p] * m2 + e2[p] * m1 - e3[p] * m0) * F[FR::IDEN + p];
  return true;
}

// Reverse part of a coupled two-layer edge from its forward record F (filled by edge_fwd_2,
// or by the sweep kernel while it recomputed the step). cL, cR: cell records (ARec<2>).
// am_b, ap_b: cotangents of A-dQ and A+dQ (6 each, (h, hn, ht) per layer). Outputs
// (accumulated, +=): cotangents of the left and right conserved states qLb[6], qRb[6] and
// of BL, BR. The cheap forward quantities (Roe averages, flux jumps, alpha_p, the elementary
// symmetric polynomials of the other three eigenvalues) are rebuilt here.
MLSWE_HD void edge_rev_2(const DevParams& P, const double* cL, const double* cR, const double* F,
                         const double* am_b, const double* ap_b, double* qLb, double* qRb, double& BLb,
                         double& BRb) {
  using R = Rec<2>;
  using FR = FwdRec;
  const double g = P.g, r = P.r;
  double hb[2], coup[2], d0[2], uh[2], vh[2], iS[2];
  for (int m = 0; m < 2; ++m) {
    hb[m] = 0.5 * (cL[3 * m] + cR[3 * m]);
    coup[m] = cR[R::ETA + m] - cL[R::ETA + m];
    if (m == 1) coup[m] += r * (cR[0] - cL[0]);
    d0[m] = cR[3 * m + 1] - cL[3 * m + 1];
    iS[m] = F[FR::IS0 + m];
    uh[m] = (cL[R::SQ + m] * cL[R::UN + 2 * m] + cR[R::SQ + m] * cR[R::UN + 2 * m]) * iS[m];
    vh[m] = (cL[R::SQ + m] * cL[R::UN + 2 * m + 1] + cR[R::SQ + m] * cR[R::UN + 2 * m + 1]) * iS[m];
  }
  const double c1 = g * hb[0], c2 = g * hb[1];
  const double iH = F[FR::IH], ic1 = F[FR::IC1], idisc = F[FR::IDISC], isp = F[FR::ISP], ism = F[FR::ISM];
  const double ubar = (hb[0] * uh[0] + hb[1] * uh[1]) * iH;
  const double dc = c1 - c2;
  const bool newton = F[FR::NEWTON] != 0.0;
  const double rc = r * c1 * c2;
  double lam[4], beta[4], iden[4], al[4], tt[4], e1[4], e2[4], e3[4];
  for (int p = 0; p < 4; ++p) {
    lam[p] = F[FR::LAM + p];
    beta[p] = F[FR::BETA + p];
    iden[p] = F[FR::IDEN + p];
    tt[p] = lam[p] - uh[0];
    al[p] = (tt[p] * tt[p] - c1) * ic1;
  }
  // elementary symmetric polynomials of the three eigenvalues other than lam_p, from those of
  // all four: e1 = S1 - l, e2 = S2 - l e1, e3 = S3 - l e2
  {
    const double s01 = lam[0] + lam[1], s23 = lam[2] + lam[3];
    const double q01 = lam[0] * lam[1], q23 = lam[2] * lam[3];
    const double S1 = s01 + s23, S2 = q01 + q23 + s01 * s23, S3 = q01 * s23 + q23 * s01;
    for (int p = 0; p < 4; ++p) {
      e1[p] = S1 - lam[p];
      e2[p] = S2 - lam[p] * e1[p];
      e3[p] = S3 - lam[p] * e2[p];
    }
  }
  const double p1 = -2.0 * uh[0], p0 = uh[0] * uh[0] - c1;
  // ---------------- reverse ----------------
  double lamb[4] = {0, 0, 0, 0}, alb[4] = {0, 0, 0, 0}, betab[4];
  double vhb[2] = {0, 0}, uhb[2] = {0, 0}, d0b[2] = {0, 0}, d1b[2] = {0, 0}, d2b[2] = {0, 0};
  double c1b = 0.0, c2b = 0.0;
  for (int p = 0; p < 4; ++p) {
    double Zb[6];
    adj_pick<6>(lam[p], am_b, ap_b, Zb);
    betab[p] = Zb[0] + lam[p] * Zb[1] + vh[0] * Zb[2] + al[p] * (Zb[3] + lam[p] * Zb[4] + vh[1] * Zb[5]);
    lamb[p] += beta[p] * (Zb[1] + al[p] * Zb[4]);
    vhb[0] += beta[p] * Zb[2];
    alb[p] += beta[p] * (Zb[3] + lam[p] * Zb[4] + vh[1] * Zb[5]);
    vhb[1] += beta[p] * al[p] * Zb[5];
  }
  for (int m = 0; m < 2; ++m) {
    double zb;
    adj_pick<1>(uh[m], am_b + 3 * m + 2, ap_b + 3 * m + 2, &zb);
    d2b[m] += zb;
    vhb[m] -= d0[m] * zb;
    d0b[m] -= vh[m] * zb;
  }
  // beta = R^{-1} delta  ->  delta_b = R^{-T} beta_b (cubic through (lam_p, beta_b_p)), R_b = -delta_b beta^T
  double C3 = 0, C2 = 0, C1 = 0, C0 = 0;
  for (int p = 0; p < 4; ++p) {
    const double w = betab[p] * iden[p];
    C3 += w; C2 -= w * e1[p]; C1 += w * e2[p]; C0 -= w * e3[p];
  }
  const double db3 = c1 * C3;
  const double db2 = c1 * C2 - p1 * db3;
  const double db1 = C1 - (p1 * db2 + p0 * db3) * ic1;
  const double db0 = C0 - p0 * db2 * ic1;
  d0b[0] += db0; d1b[0] += db1; d0b[1] += db2; d1b[1] += db3;
  for (int p = 0; p < 4; ++p) {
    lamb[p] -= beta[p] * (db1 + al[p] * db3);
    alb[p] -= beta[p] * (db2 + lam[p] * db3);
  }
  // alpha_p = (t^2 - c1) / c1, t = lam_p - uh1
  for (int p = 0; p < 4; ++p) {
    const double g2 = 2.0 * tt[p] * ic1 * alb[p];
    lamb[p] += g2;
    uhb[0] -= g2;
    c1b -= alb[p] * tt[p] * tt[p] * ic1 * ic1;
  }
  // Newton steps in reverse. A step is l' = l - P/D with P(l) = f1 f2 - r c1 c2,
  // f_m = (l - u_m)^2 - c_m, D = dP/dl. For a parameter x, dl'/dx = -(P_x D - P D_x)/D^2 and
  // dl'/dl = P D_l / D^2. With w = lb/D and v = w P/D the cotangent of x is -(w P_x - v D_x);
  // P_u1 = -D - P_u2 and D_u1 = -D_l - D_u2 give the second velocity from the first.
  if (newton) {
    const double rc1 = r * c1, rc2 = r * c2;
    for (int it = 1; it >= 0; --it) {
      for (int p = 0; p < 4; ++p) {
        const double l = F[(it == 1 ? FR::LAM1 : FR::LAM0) + p];
        const double a1 = l - uh[0], a2 = l - uh[1];
        const double a12 = a1 * a2;
        const double f1 = a1 * a1 - c1, f2 = a2 * a2 - c2;
        const double Pl = f1 * f2 - rc;
        const double Dl = 2.0 * ((f1 + f2) + 4.0 * a12);
        const double lb = lamb[p];
        const double iD = F[(it == 1 ? FR::ID1 : FR::ID0) + p];
        const double w = lb * iD;
        const double v = (w * Pl) * iD;
        const double lnew = v * Dl;
        // P_u1 = -2 a1 f2, D_u1 = -2 (f2 + 2 a1 a2); P_c1 = -(f2 + r c2), D_c1 = -2 a2; P_c2, D_c2 alike
        const double gu0 = 2.0 * (v * (f2 + 2.0 * a12) - (w * a1) * f2);
        const double gc1 = 2.0 * v * a2 - w * (f2 + rc2);
        const double gc2 = 2.0 * v * a1 - w * (f1 + rc1);
        uhb[0] -= gu0;
        uhb[1] += (lb - lnew) + gu0;
        c1b -= gc1;
        c2b -= gc2;
        lamb[p] = lnew;
      }
    }
  }
  // guesses lam0 = ubar -+ sqrt(mu_+-)
  const double ubarb = lamb[0] + lamb[1] + lamb[2] + lamb[3];
  const double spb = lamb[3] - lamb[0], smb = lamb[2] - lamb[1];
  const double mupb = spb * 0.5 * isp, mumb = smb * 0.5 * ism;
  const double csumb = 0.5 * (mupb + mumb), discb = 0.5 * (mupb - mumb);
  c1b += csumb + discb * (dc + 2.0 * r * c2) * idisc;
  c2b += csumb + discb * (-dc + 2.0 * r * c1) * idisc;
  double hbb[2];
  uhb[0] += ubarb * hb[0] * iH;
  uhb[1] += ubarb * hb[1] * iH;
  hbb[0] = ubarb * (uh[0] - ubar) * iH + g * c1b;
  hbb[1] = ubarb * (uh[1] - ubar) * iH + g * c2b;
  // Roe averages and flux differences, per layer
  double unb[2][2] = {{0, 0}, {0, 0}}, utb[2][2] = {{0, 0}, {0, 0}}, sqb[2][2] = {{0, 0}, {0, 0}};
  double hnb[2][2] = {{0, 0}, {0, 0}}, hbar_b[2][2] = {{0, 0}, {0, 0}}, etab[2][2] = {{0, 0}, {0, 0}};
  for (int m = 0; m < 2; ++m) {
    const double* c[2] = {cL, cR};
    for (int s = 0; s < 2; ++s) {
      const double w = c[s][R::SQ + m] * iS[m];
      unb[s][m] += uhb[m] * w;
      utb[s][m] += vhb[m] * w;
      sqb[s][m] += (uhb[m] * (c[s][R::UN + 2 * m] - uh[m]) + vhb[m] * (c[s][R::UN + 2 * m + 1] - vh[m])) * iS[m];
    }
    // d0 = hnR - hnL
    hnb[1][m] += d0b[m]; hnb[0][m] -= d0b[m];
    // d1 = hnR unR - hnL unL + g hb coup
    hnb[1][m] += d1b[m] * cR[R::UN + 2 * m]; unb[1][m] += d1b[m] * cR[3 * m + 1];
    hnb[0][m] -= d1b[m] * cL[R::UN + 2 * m]; unb[0][m] -= d1b[m] * cL[3 * m + 1];
    hbb[m] += d1b[m] * g * coup[m];
    const double coupb = d1b[m] * g * hb[m];
    etab[1][m] += coupb; etab[0][m] -= coupb;
    if (m == 1) { hbar_b[1][0] += r * coupb; hbar_b[0][0] -= r * coupb; }
    // d2 = hnR utR - hnL utL
    hnb[1][m] += d2b[m] * cR[R::UN + 2 * m + 1]; utb[1][m] += d2b[m] * cR[3 * m + 1];
    hnb[0][m] -= d2b[m] * cL[R::UN + 2 * m + 1]; utb[0][m] -= d2b[m] * cL[3 * m + 1];
    // hb = (hL + hR) / 2
    hbar_b[0][m] += 0.5 * hbb[m]; hbar_b[1][m] += 0.5 * hbb[m];
  }
  // per cell: eta_2 = B + h_2, eta_1 = eta_2 + h_1; un = hn/h, ut = ht/h, sq = sqrt(h)
  for (int s = 0; s < 2; ++s) {
    const double* c = s ? cR : cL;
    double* qb = s ? qRb : qLb;
    double& Bb = s ? BRb : BLb;
    const double e2b = etab[s][1] + etab[s][0];
    double hbs[2] = {hbar_b[s][0] + etab[s][0], hbar_b[s][1] + e2b};
    Bb += e2b;
    for (int m = 0; m < 2; ++m) {
      const double is = c[ARec<2>::IS + m], ih = is * is;  // 1/sqrt(h), 1/h
      const double un = c[R::UN + 2 * m], ut = c[R::UN + 2 * m + 1];
      hbs[m] += -(unb[s][m] * un + utb[s][m] * ut) * ih + sqb[s][m] * 0.5 * is;
      qb[3 * m] += hbs[m];
      qb[3 * m + 1] += hnb[s][m] + unb[s][m] * ih;
      qb[3 * m + 2] += utb[s][m] * ih;
    }
  }
}

// Coupled two-layer edge, forward and reverse in one call. Returns false if the states are
// not in the coupled branch (some layer not wet on some side).
MLSWE_HD bool edge_vjp_2(const DevParams& P, const double* cL, const double* cR, int wL, int wR,
                         const double* am_b, const double* ap_b, double* qLb, double* qRb, double& BLb, double& BRb) {
  double F[FwdRec::N];
  if (!edge_fwd_2(P, cL, cR, wL, wR, F)) return false;
  edge_rev_2(P, cL, cR, F, am_b, ap_b, qLb, qRb, BLb, BRb);
  return true;
}

// One-layer edge (M = 1, wet on both sides): Roe speeds uh -+ sqrt(g hbar).
MLSWE_HD bool edge_vjp_1(const DevParams& P, const double* cL, const double* cR, int wL, int wR,
                         const double* am_b, const double* ap_b, double* qLb, double* qRb, double& BLb, double& BRb) {
  using R = Rec<1>;
  if (!(wL & 1) || !(wR & 1)) return false;
  const double g = P.g;
  const double hL = cL[0], hR = cR[0], hnL = cL[1], hnR = cR[1];
  const double unL = cL[R::UN], unR = cR[R::UN], utL = cL[R::UN + 1], utR = cR[R::UN + 1];
  const double sL = cL[R::SQ], sR = cR[R::SQ];
  const double hb = 0.5 * (hL + hR);
  const double coup = cR[R::ETA] - cL[R::ETA];
  const double d0 = hnR - hnL;
  const double d1 = (hnR * unR - hnL * unL) + g * hb * coup;
  const double iS = adj_rcp(sL + sR);
  const double uh = (sL * unL + sR * unR) * iS, vh = (sL * utL + sR * utR) * iS;
  const double ghb = g * hb, ich = adj_rsqrt(ghb), ch = ghb * ich;
  const double s1 = uh - ch, s2 = uh + ch;
  const double inv = 0.5 * ich;  // 1/(s2 - s1)
  const double b1 = (s2 * d0 - d1) * inv, b2 = (d1 - s1 * d0) * inv;
  // reverse
  double Z1b[3], Z2b[3], zb;
  adj_pick<3>(s1, am_b, ap_b, Z1b);
  adj_pick<3>(s2, am_b, ap_b, Z2b);
  adj_pick<1>(uh, am_b + 2, ap_b + 2, &zb);
  // Z1 = b1 (1, s1, vh), Z2 = b2 (1, s2, vh), shear = d2 - vh d0
  const double b1b = Z1b[0] + s1 * Z1b[1] + vh * Z1b[2];
  const double b2b = Z2b[0] + s2 * Z2b[1] + vh * Z2b[2];
  double s1b = b1 * Z1b[1], s2b = b2 * Z2b[1];
  double vhb = b1 * Z1b[2] + b2 * Z2b[2] - d0 * zb;
  double d0b = -vh * zb, d1b = 0.0, d2b = zb;
  // b1 = (s2 d0 - d1)/(s2 - s1), b2 = (d1 - s1 d0)/(s2 - s1)
  d0b += (b1b * s2 - b2b * s1) * inv;
  d1b += (-b1b + b2b) * inv;
  s2b += b1b * (d0 - b1) * inv - b2b * b2 * inv;
  s1b += b1b * b1 * inv + b2b * (-d0 + b2) * inv;
  // s1 = uh - ch, s2 = uh + ch, ch = sqrt(g hb)
  const double uhb = s1b + s2b;
  const double chb = s2b - s1b;
  double hbb = chb * g * 0.5 * ich;
  double unb[2], utb[2], sqb[2], hnb[2] = {0, 0};
  unb[0] = uhb * sL * iS; unb[1] = uhb * sR * iS;
  utb[0] = vhb * sL * iS; utb[1] = vhb * sR * iS;
  sqb[0] = (uhb * (unL - uh) + vhb * (utL - vh)) * iS;
  sqb[1] = (uhb * (unR - uh) + vhb * (utR - vh)) * iS;
  hnb[1] += d0b; hnb[0] -= d0b;
  hnb[1] += d1b * unR; unb[1] += d1b * hnR; hnb[0] -= d1b * unL; unb[0] -= d1b * hnL;
  hbb += d1b * g * coup;
  const double coupb = d1b * g * hb;
  hnb[1] += d2b * utR; utb[1] += d2b * hnR; hnb[0] -= d2b * utL; utb[0] -= d2b * hnL;
  const double* c[2] = {cL, cR};
  double* qb[2] = {qLb, qRb};
  double etab[2] = {-coupb, coupb};
  for (int s = 0; s < 2; ++s) {
    const double is = c[s][ARec<1>::IS], ih = is * is;  // 1/sqrt(h), 1/h
    double hsb = 0.5 * hbb + etab[s] - (unb[s] * c[s][R::UN] + utb[s] * c[s][R::UN + 1]) * ih + sqb[s] * 0.5 * is;
    qb[s][0] += hsb;
    qb[s][1] += hnb[s] + unb[s] * ih;
    qb[s][2] += utb[s] * ih;
  }
  BLb += etab[0];
  BRb += etab[1];
  return true;
}

}  // namespace mlswe
