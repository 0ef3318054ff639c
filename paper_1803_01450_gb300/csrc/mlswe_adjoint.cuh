// Reverse-mode derivative (vector-Jacobian product) of the first-order edge
// fluctuations (A-dQ, A+dQ) of mlswe_device.cuh's Riemann solver, for wet
// states: the coupled two-layer branch (M = 2, both layers wet on both sides)
// and the one-layer branch (M = 1, wet on both sides). Hand-written: the
// forward quantities are recomputed, then every statement is differentiated in
// reverse order. Signs of the wave speeds select fluctuations and are treated
// as constant (the derivative of the selection is zero almost everywhere).
//
// Cell records are the same as the forward sweep's (Rec<M>: h, hn, ht per
// layer, un, ut, sqrt(h), eta, B); bathymetry enters through eta.
#pragma once
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

// Selection weights of a wave of speed s into (A-dQ, A+dQ).
MLSWE_HD void adj_side_weights(double s, double& wl, double& wr) {
  wl = s < 0.0 ? 1.0 : (s > 0.0 ? 0.0 : 0.5);
  wr = 1.0 - wl;
}

// Coupled two-layer edge. cL, cR: cell records (Rec<2>). am_b, ap_b: cotangents of A-dQ and
// A+dQ (6 each, (h, hn, ht) per layer). Outputs (accumulated, +=): cotangents of the left and
// right conserved states qLb[6], qRb[6] and of BL, BR. Returns false if the states are not
// in the coupled branch (some layer not wet on some side).
MLSWE_HD bool edge_vjp_2(const DevParams& P, const double* cL, const double* cR, int wL, int wR,
                         const double* am_b, const double* ap_b, double* qLb, double* qRb, double& BLb, double& BRb) {
  using R = Rec<2>;
  if (wL != 3 || wR != 3) return false;
  const double g = P.g, r = P.r;
  // ---------------- forward recompute ----------------
  double hb[2], coup[2], d0[2], d1[2], d2[2], S[2], iS[2], uh[2], vh[2];
  for (int m = 0; m < 2; ++m) {
    hb[m] = 0.5 * (cL[3 * m] + cR[3 * m]);
    coup[m] = cR[R::ETA + m] - cL[R::ETA + m];
    if (m == 1) coup[m] += r * (cR[0] - cL[0]);
    d0[m] = cR[3 * m + 1] - cL[3 * m + 1];
    d1[m] = (cR[3 * m + 1] * cR[R::UN + 2 * m] - cL[3 * m + 1] * cL[R::UN + 2 * m]) + g * hb[m] * coup[m];
    d2[m] = cR[3 * m + 1] * cR[R::UN + 2 * m + 1] - cL[3 * m + 1] * cL[R::UN + 2 * m + 1];
    S[m] = cL[R::SQ + m] + cR[R::SQ + m];
    iS[m] = adj_rcp(S[m]);
    uh[m] = (cL[R::SQ + m] * cL[R::UN + 2 * m] + cR[R::SQ + m] * cR[R::UN + 2 * m]) * iS[m];
    vh[m] = (cL[R::SQ + m] * cL[R::UN + 2 * m + 1] + cR[R::SQ + m] * cR[R::UN + 2 * m + 1]) * iS[m];
  }
  const double c1 = g * hb[0], c2 = g * hb[1];
  const double Hs = hb[0] + hb[1], iH = adj_rcp(Hs);
  const double ubar = (hb[0] * uh[0] + hb[1] * uh[1]) * iH;
  const double dc = c1 - c2;
  const double disc = sqrt(dc * dc + 4.0 * r * c1 * c2);
  const double csum = c1 + c2;
  const double sp = sqrt(0.5 * (csum + disc)), sm = sqrt(0.5 * (csum - disc));
  double lam0[4] = {ubar - sp, ubar - sm, ubar + sm, ubar + sp};
  const double du = uh[0] - uh[1];
  const bool newton = !(du * du >= (1.0 - r) * g * (hb[0] + hb[1])) && P.eigen == 0;
  double lam1[4], lam[4];
  const double rc = r * c1 * c2;
  for (int p = 0; p < 4; ++p) {
    double l = lam0[p];
    if (newton) {
      for (int it = 0; it < 2; ++it) {
        if (it == 1) lam1[p] = l;
        const double a1 = l - uh[0], a2 = l - uh[1];
        const double f1 = a1 * a1 - c1, f2 = a2 * a2 - c2;
        const double Pl = f1 * f2 - rc;
        const double D = 2.0 * (a1 * f2 + a2 * f1);
        l = l - Pl * adj_rcp(D);
      }
    } else {
      lam1[p] = l;
    }
    lam[p] = l;
  }
  const double ic1 = adj_rcp(c1);
  double al[4], tt[4];
  for (int p = 0; p < 4; ++p) { tt[p] = lam[p] - uh[0]; al[p] = (tt[p] * tt[p] - c1) * ic1; }
  // wave strengths: Vandermonde form (see mlswe_device.cuh)
  const double p1 = -2.0 * uh[0], p0 = uh[0] * uh[0] - c1;
  const double m0 = d0[0], m1 = d1[0];
  const double m2 = c1 * d0[1] - p1 * m1 - p0 * m0;
  const double m3 = c1 * d1[1] - p1 * m2 - p0 * m1;
  double e1[4], e2[4], e3[4], iden[4], beta[4];
  for (int p = 0; p < 4; ++p) {
    const int qa = (p + 1) & 3, qb = (p + 2) & 3, qc = (p + 3) & 3;
    e1[p] = lam[qa] + lam[qb] + lam[qc];
    e2[p] = lam[qa] * lam[qb] + lam[qa] * lam[qc] + lam[qb] * lam[qc];
    e3[p] = lam[qa] * lam[qb] * lam[qc];
    const double den = (lam[p] - lam[qa]) * (lam[p] - lam[qb]) * (lam[p] - lam[qc]);
    iden[p] = adj_rcp(den);
    beta[p] = (m3 - e1[p] * m2 + e2[p] * m1 - e3[p] * m0) * iden[p];
  }
  // ---------------- reverse ----------------
  double lamb[4] = {0, 0, 0, 0}, alb[4] = {0, 0, 0, 0}, betab[4];
  double vhb[2] = {0, 0}, uhb[2] = {0, 0}, d0b[2] = {0, 0}, d1b[2] = {0, 0}, d2b[2] = {0, 0};
  double c1b = 0.0, c2b = 0.0;
  for (int p = 0; p < 4; ++p) {
    double wl, wr;
    adj_side_weights(lam[p], wl, wr);
    double Zb[6];
    for (int f = 0; f < 6; ++f) Zb[f] = wl * am_b[f] + wr * ap_b[f];
    betab[p] = Zb[0] + lam[p] * Zb[1] + vh[0] * Zb[2] + al[p] * (Zb[3] + lam[p] * Zb[4] + vh[1] * Zb[5]);
    lamb[p] += beta[p] * (Zb[1] + al[p] * Zb[4]);
    vhb[0] += beta[p] * Zb[2];
    alb[p] += beta[p] * (Zb[3] + lam[p] * Zb[4] + vh[1] * Zb[5]);
    vhb[1] += beta[p] * al[p] * Zb[5];
  }
  for (int m = 0; m < 2; ++m) {
    double wl, wr;
    adj_side_weights(uh[m], wl, wr);
    const double zb = wl * am_b[3 * m + 2] + wr * ap_b[3 * m + 2];
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
  // Newton steps in reverse
  if (newton) {
    for (int it = 1; it >= 0; --it) {
      for (int p = 0; p < 4; ++p) {
        const double l = it == 1 ? lam1[p] : lam0[p];
        const double a1 = l - uh[0], a2 = l - uh[1];
        const double f1 = a1 * a1 - c1, f2 = a2 * a2 - c2;
        const double Pl = f1 * f2 - rc;
        const double D = 2.0 * (a1 * f2 + a2 * f1);
        const double iD = adj_rcp(D), iD2 = iD * iD;
        const double Dl = 2.0 * (f1 + f2 + 4.0 * a1 * a2);
        const double Pu0 = -2.0 * a1 * f2, Du0 = -2.0 * (f2 + 2.0 * a1 * a2);
        const double Pu1 = -2.0 * a2 * f1, Du1 = -2.0 * (f1 + 2.0 * a1 * a2);
        const double Pc1 = -f2 - r * c2, Dc1 = -2.0 * a2;
        const double Pc2 = -f1 - r * c1, Dc2 = -2.0 * a1;
        const double lb = lamb[p];
        uhb[0] -= lb * (Pu0 * D - Pl * Du0) * iD2;
        uhb[1] -= lb * (Pu1 * D - Pl * Du1) * iD2;
        c1b -= lb * (Pc1 * D - Pl * Dc1) * iD2;
        c2b -= lb * (Pc2 * D - Pl * Dc2) * iD2;
        lamb[p] = lb * Pl * Dl * iD2;
      }
    }
  }
  // guesses lam0 = ubar -+ sqrt(mu_+-)
  const double ubarb = lamb[0] + lamb[1] + lamb[2] + lamb[3];
  const double spb = lamb[3] - lamb[0], smb = lamb[2] - lamb[1];
  const double mupb = spb * 0.5 * adj_rcp(sp), mumb = smb * 0.5 * adj_rcp(sm);
  const double csumb = 0.5 * (mupb + mumb), discb = 0.5 * (mupb - mumb);
  const double idisc = adj_rcp(disc);
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
      const double h = c[3 * m], ih = adj_rcp(h);
      const double un = c[R::UN + 2 * m], ut = c[R::UN + 2 * m + 1];
      hbs[m] += -(unb[s][m] * un + utb[s][m] * ut) * ih + sqb[s][m] * 0.5 * adj_rcp(c[R::SQ + m]);
      qb[3 * m] += hbs[m];
      qb[3 * m + 1] += hnb[s][m] + unb[s][m] * ih;
      qb[3 * m + 2] += utb[s][m] * ih;
    }
  }
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
  const double d2 = hnR * utR - hnL * utL;
  const double iS = adj_rcp(sL + sR);
  const double uh = (sL * unL + sR * unR) * iS, vh = (sL * utL + sR * utR) * iS;
  const double ch = sqrt(g * hb);
  const double s1 = uh - ch, s2 = uh + ch;
  const double inv = adj_rcp(s2 - s1);
  const double b1 = (s2 * d0 - d1) * inv, b2 = (d1 - s1 * d0) * inv;
  // reverse
  double w1l, w1r, w2l, w2r, wsl, wsr;
  adj_side_weights(s1, w1l, w1r);
  adj_side_weights(s2, w2l, w2r);
  adj_side_weights(uh, wsl, wsr);
  double Z1b[3], Z2b[3];
  for (int f = 0; f < 3; ++f) { Z1b[f] = w1l * am_b[f] + w1r * ap_b[f]; Z2b[f] = w2l * am_b[f] + w2r * ap_b[f]; }
  const double zb = wsl * am_b[2] + wsr * ap_b[2];
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
  double hbb = chb * g * 0.5 * adj_rcp(ch);
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
    const double h = c[s][0], ih = adj_rcp(h);
    double hsb = 0.5 * hbb + etab[s] - (unb[s] * c[s][R::UN] + utb[s] * c[s][R::UN + 1]) * ih +
                 sqb[s] * 0.5 * adj_rcp(c[s][R::SQ]);
    qb[s][0] += hsb;
    qb[s][1] += hnb[s] + unb[s] * ih;
    qb[s][2] += utb[s] * ih;
  }
  BLb += etab[0];
  BRb += etab[1];
  return true;
}

}  // namespace mlswe
