// integrals.cuh -- closed-form inner integrals of the retarded kernels over one
// source triangle (paper section 2.3, eq. layer_disc_tmp and the integrals I_d).
//
// For an observation point x and a source triangle T, with tau = m - r/(c dt)
// and the quadratic B-spline N (section 2.2), the library needs for each lag m
//     phi  = int_T N(tau)/r dS,     A0 = int_T Nddot(tau)/r dS,
//     A1   = int_T Nddot(tau)/r (y - x) dS,
//     P1   = int_T g'(r)/r (y - x) dS,   g(r) = (cdot Ndot(tau) + zeta N(tau)) / r,
// cdot = chi / dt (chi: weight of the time-differentiated MFIE).
// In polar coordinates about the projection p of x on the plane of T (height h,
// r dr = rho drho) the radial integral of F is an antiderivative Q(r) with
// Q' = F r; the in-plane part of the vector integrals is, by the divergence
// theorem in the plane, a sum over the sides of T of the outward side normal
// times the side integral of Q.  Along a side at signed distance d from p,
// parametrised by s (r^2 = h^2 + d^2 + s^2):
//     angular part  int (Q(r) - Q(|h|)) d/(d^2+s^2) ds
//     side part     int Q(r) ds
// Q is piecewise polynomial in r (times 1/r for g) between the light-cone
// circles r = j c dt, so each side is cut at those circles and every piece is
// integrated exactly with the primitives of r^n and (r^n - |h|^n) d/(d^2+s^2).
#pragma once

#include "internal.h"

namespace tdbem {

struct InnerOut {
  double phi[kMaxWin], A0[kMaxWin], Sn[kMaxWin];
  double EA[kMaxWin][3], EP[kMaxWin][3];
  double h;
  bool hasP;
};

// Pieces of the quadratic B-spline on [k, k+1] in the local variable
// u = tau - k in [0, 1]: N, Ndot, and C = int_{-inf}^{tau} N (textbook form).
__device__ __forceinline__ void bspline_piece_coeffs(int k, double* Np, double* Ndp, double* Cp) {
  // polynomials in u, ascending powers
  if (k == 0) {
    Np[0] = 0; Np[1] = 0; Np[2] = 0.5;
    Ndp[0] = 0; Ndp[1] = 1; Ndp[2] = 0;
    Cp[0] = 0; Cp[1] = 0; Cp[2] = 0; Cp[3] = 1.0 / 6.0;
  } else if (k == 1) {
    Np[0] = 0.5; Np[1] = 1; Np[2] = -1;
    Ndp[0] = 1; Ndp[1] = -2; Ndp[2] = 0;
    Cp[0] = 1.0 / 6.0; Cp[1] = 0.5; Cp[2] = 0.5; Cp[3] = -1.0 / 3.0;
  } else {
    Np[0] = 0.5; Np[1] = -1; Np[2] = 0.5;
    Ndp[0] = -1; Ndp[1] = 1; Ndp[2] = 0;
    Cp[0] = 5.0 / 6.0; Cp[1] = 0.5; Cp[2] = -0.5; Cp[3] = 1.0 / 6.0;
  }
}

// N, Ndot and C at tau (any real)
__device__ __forceinline__ void bspline_eval(double tau, double* N, double* Nd, double* C) {
  if (tau <= 0.0) { *N = 0; *Nd = 0; *C = 0; return; }
  if (tau >= 3.0) { *N = 0; *Nd = 0; *C = 1; return; }
  int k = (int)tau;
  if (k > 2) k = 2;
  double u = tau - k;
  double Np[3], Ndp[3], Cp[4];
  bspline_piece_coeffs(k, Np, Ndp, Cp);
  *N = Np[0] + u * (Np[1] + u * Np[2]);
  *Nd = Ndp[0] + u * Ndp[1];
  *C = Cp[0] + u * (Cp[1] + u * (Cp[2] + u * Cp[3]));
}

// A B-spline piece is a polynomial in u = tau - k; with tau = m - r/a this is
// u = u0 + beta r (u0 = m - k, beta = -1/a).  Returns the coefficients of the
// same polynomial in ascending powers of r.
template <int K>
__device__ __forceinline__ void poly_u_to_r(const double* pu, double u0, double beta, double* qr) {
  // binomial expansion of (u0 + beta r)^k
  const double binom[4][4] = {{1, 0, 0, 0}, {1, 1, 0, 0}, {1, 2, 1, 0}, {1, 3, 3, 1}};
  double bp[K + 1];
  bp[0] = 1.0;
  for (int n = 1; n <= K; ++n) bp[n] = bp[n - 1] * beta;
  for (int n = 0; n <= K; ++n) {
    double s = 0.0;
    double u0p = 1.0;  // u0^(k-n)
    for (int k = n; k <= K; ++k) {
      s += pu[k] * binom[k][n] * u0p;
      u0p *= u0;
    }
    qr[n] = s * bp[n];
  }
}

// Primitives along one side at parameter s.  E[n+1] = int r^n ds,
// At[n+1] = int (r^n - |h|^n) d/(d^2+s^2) ds, n = -1..3.
__device__ __forceinline__ void side_primitives(double s, double d, double hh, double R0sq, bool ang, bool hasP,
                                                double* E, double* At) {
  double r = sqrt(R0sq + s * s);
  double R0 = sqrt(R0sq);
  double ash = (R0 > 0.0) ? asinh(s / R0) : 0.0;
  E[1] = s;
  E[2] = (R0 > 0.0) ? 0.5 * (s * r + R0sq * ash) : 0.5 * s * fabs(s);
  E[3] = R0sq * s + s * s * s / 3.0;
  E[4] = 0.25 * s * r * r * r + 0.75 * R0sq * E[2];
  E[0] = hasP ? ash : 0.0;
  if (ang) {
    double T = 0.0;
    if (hh > 0.0) {
      double num = -s * d * (d * d + s * s);
      double den = (r + hh) * (d * d * r + hh * s * s);
      T = atan(num / den);
    }
    At[1] = 0.0;
    At[2] = d * ash + hh * T;
    At[3] = d * s;
    At[4] = d * E[2] + hh * hh * At[2];
    At[0] = hasP ? T / hh : 0.0;
  } else {
    for (int n = 0; n < 5; ++n) At[n] = 0.0;
  }
}

// Lag window of (x, T): lags with a possibly non-zero kernel anywhere on T.
__device__ __forceinline__ void lag_window(double rlo, double rhi, double a, int* m0, int* nm) {
  int lo = (int)floor(rlo / a) + 1;
  if (lo < 1) lo = 1;
  int hi = (int)ceil(rhi / a + 3.0) - 1;
  *m0 = lo;
  *nm = hi - lo + 1;
}

// Inner integrals for lags m0 .. m0+nm-1 (nm <= kMaxWin).  v: 3 vertices
// (row-major), nT: unit normal of the winding, lmax: longest side.
// Returns false if the number of light-cone pieces exceeds the local buffers.
__device__ bool inner_integrals(const double* x, const double* v, const double* nT, double lmax, double a,
                                double cdot, double zeta, int m0, int nm, InnerOut& o) {
  double h = (x[0] - v[0]) * nT[0] + (x[1] - v[1]) * nT[1] + (x[2] - v[2]) * nT[2];
  bool hasP = fabs(h) > 1e-10 * lmax;
  if (!hasP) h = 0.0;
  double hh = fabs(h);
  o.h = h;
  o.hasP = hasP;
  double p[3] = {x[0] - h * nT[0], x[1] - h * nT[1], x[2] - h * nT[2]};
  for (int i = 0; i < nm; ++i) {
    o.phi[i] = o.A0[i] = o.Sn[i] = 0.0;
    for (int q = 0; q < 3; ++q) o.EA[i][q] = o.EP[i][q] = 0.0;
  }
  // values at r = |h| of Q_phi = -a C, Q_A = -a Ndot, g
  double Qh_phi[kMaxWin], Qh_A[kMaxWin], Qh_g[kMaxWin];
  for (int i = 0; i < nm; ++i) {
    double N, Nd, C;
    bspline_eval((m0 + i) - hh / a, &N, &Nd, &C);
    Qh_phi[i] = -a * C;
    Qh_A[i] = -a * Nd;
    Qh_g[i] = hasP ? (Nd * cdot + zeta * N) / hh : 0.0;
  }
  // distance range of x to T, for the knot range
  double rmax = 0.0, cen[3];
  for (int q = 0; q < 3; ++q) cen[q] = (v[q] + v[3 + q] + v[6 + q]) / 3.0;
  double rad = 0.0;
  for (int k = 0; k < 3; ++k) {
    double dx = v[3 * k] - x[0], dy = v[3 * k + 1] - x[1], dz = v[3 * k + 2] - x[2];
    rmax = fmax(rmax, sqrt(dx * dx + dy * dy + dz * dz));
    double ex = v[3 * k] - cen[0], ey = v[3 * k + 1] - cen[1], ez = v[3 * k + 2] - cen[2];
    rad = fmax(rad, sqrt(ex * ex + ey * ey + ez * ez));
  }
  double dcx = x[0] - cen[0], dcy = x[1] - cen[1], dcz = x[2] - cen[2];
  double rlow = sqrt(dcx * dcx + dcy * dcy + dcz * dcz) - rad;
  int jlo = (int)floor(fmax(rlow, 0.0) / a);
  if (jlo < 1) jlo = 1;
  int jhi = (int)floor(rmax / a) + 1;
  if (jhi - jlo + 1 > kMaxWin) return false;

  for (int k = 0; k < 3; ++k) {
    const double* va = v + 3 * k;
    const double* vb = v + 3 * ((k + 1) % 3);
    double tv[3] = {vb[0] - va[0], vb[1] - va[1], vb[2] - va[2]};
    double L = sqrt(tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2]);
    tv[0] /= L; tv[1] /= L; tv[2] /= L;
    double nu[3] = {tv[1] * nT[2] - tv[2] * nT[1], tv[2] * nT[0] - tv[0] * nT[2], tv[0] * nT[1] - tv[1] * nT[0]};
    double wa[3] = {va[0] - p[0], va[1] - p[1], va[2] - p[2]};
    double wb[3] = {vb[0] - p[0], vb[1] - p[1], vb[2] - p[2]};
    double d = wa[0] * nu[0] + wa[1] * nu[1] + wa[2] * nu[2];
    double sm = wa[0] * tv[0] + wa[1] * tv[1] + wa[2] * tv[2];
    double sp = wb[0] * tv[0] + wb[1] * tv[1] + wb[2] * tv[2];
    double R0sq = h * h + d * d;
    bool ang = fabs(d) > 1e-14 * L;
    // break points at the light-cone circles, sorted
    double br[2 * kMaxWin + 2];
    int nb = 0;
    br[nb++] = sm;
    for (int j = jlo; j <= jhi; ++j) {
      double R = j * a;
      double q = R * R - R0sq;
      if (q > 0.0) {
        double sq = sqrt(q);
        if (-sq > sm && -sq < sp) br[nb++] = -sq;
        if (sq > sm && sq < sp) br[nb++] = sq;
      }
    }
    br[nb++] = sp;
    for (int i = 1; i < nb; ++i) {  // insertion sort
      double t = br[i];
      int jj = i - 1;
      while (jj >= 0 && br[jj] > t) {
        br[jj + 1] = br[jj];
        --jj;
      }
      br[jj + 1] = t;
    }
    double psi_side = ang ? (atan(sp / d) - atan(sm / d)) : 0.0;
    // the -Q(|h|) part of the angular integrand, once per side
    if (ang) {
      for (int i = 0; i < nm; ++i) {
        o.phi[i] -= Qh_phi[i] * psi_side;
        o.A0[i] -= Qh_A[i] * psi_side;
        if (hasP) o.Sn[i] -= Qh_g[i] * psi_side;
      }
    }
    double Ea[5], Aa[5];
    side_primitives(br[0], d, hh, R0sq, ang, hasP, Ea, Aa);
    for (int pc = 0; pc + 1 < nb; ++pc) {
      double sa = br[pc], sb = br[pc + 1];
      double Eb[5], Ab[5];
      side_primitives(sb, d, hh, R0sq, ang, hasP, Eb, Ab);
      if (sb > sa) {
        double dE[5], dA[5];
        for (int n = 0; n < 5; ++n) {
          dE[n] = Eb[n] - Ea[n];
          dA[n] = Ab[n] - Aa[n];
        }
        double dpsi = ang ? (atan(sb / d) - atan(sa / d)) : 0.0;
        double sm2 = 0.5 * (sa + sb);
        double rmid = sqrt(R0sq + sm2 * sm2);
        int j = (int)floor(rmid / a);
        for (int i = 0; i < nm; ++i) {
          int m = m0 + i;
          int kap = m - j - 1;  // spline piece on this side piece: tau in (kap, kap+1)
          if (kap < 0) continue;
          if (kap > 2) {  // tau > 3: C = 1 (Q_phi = -a constant), Ndot = N = 0
            o.phi[i] += -a * dpsi;
            continue;
          }
          double Np[3], Ndp[3], Cp[4];
          bspline_piece_coeffs(kap, Np, Ndp, Cp);
          double u0 = (double)(m - kap), beta = -1.0 / a;
          // Q_phi = -a C,  Q_A = -a Ndot,  G = cdot Ndot + zeta N  (g = G/r)
          double qC[4], qNd[2], qG[3], Gu[3];
          for (int n = 0; n < 3; ++n) Gu[n] = Ndp[n] * cdot + zeta * Np[n];
          poly_u_to_r<3>(Cp, u0, beta, qC);
          poly_u_to_r<1>(Ndp, u0, beta, qNd);
          poly_u_to_r<2>(Gu, u0, beta, qG);
          double uh = u0 + beta * hh;  // local variable at r = |h| on this piece's polynomial
          double Cph = Cp[0] + uh * (Cp[1] + uh * (Cp[2] + uh * Cp[3]));
          double Ndph = Ndp[0] + uh * Ndp[1];
          double Gph = Gu[0] + uh * (Gu[1] + uh * Gu[2]);
          // angular parts: sum_n q_n dAt_n + Q_piece(|h|) dpsi
          double angC = qC[0] * dA[1] + qC[1] * dA[2] + qC[2] * dA[3] + qC[3] * dA[4];
          double angNd = qNd[0] * dA[1] + qNd[1] * dA[2];
          o.phi[i] += -a * (angC + Cph * dpsi);
          o.A0[i] += -a * (angNd + Ndph * dpsi);
          double sideNd = qNd[0] * dE[1] + qNd[1] * dE[2];
          for (int q = 0; q < 3; ++q) o.EA[i][q] += nu[q] * (-a * sideNd);
          if (hasP) {
            double angG = qG[0] * dA[0] + qG[1] * dA[1] + qG[2] * dA[2];
            o.Sn[i] += angG + (Gph / hh) * dpsi;
            double sideG = qG[0] * dE[0] + qG[1] * dE[1] + qG[2] * dE[2];
            for (int q = 0; q < 3; ++q) o.EP[i][q] += nu[q] * sideG;
          }
        }
      }
      for (int n = 0; n < 5; ++n) {
        Ea[n] = Eb[n];
        Aa[n] = Ab[n];
      }
    }
  }
  return true;
}

}  // namespace tdbem
