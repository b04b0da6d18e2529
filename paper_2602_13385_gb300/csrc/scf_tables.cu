// Host generation of the recurrence and normalisation tables used by the SCF
// kernels (double precision; float copies for the mixed-precision kernels).
#include <cmath>
#include <cstring>

#include "scf_device.cuh"
#include "scf_internal.h"

static const double kPi = 3.14159265358979323846;

// Gegenbauer index of degree l in the Zhao (1996) family of exponent alpha
// (Eq. 4): lambda_l = (2l + 1) alpha + 1/2 (2l + 3/2 for Hernquist-Ostriker).
static double zhao_lambda(int l, double alpha) { return (2.0 * l + 1.0) * alpha + 0.5; }

void scf_make_const(ScfConst* t, double alpha) {
  std::memset(t, 0, sizeof(*t));
  for (int l = 0; l <= SCF_LMAX_CAP; ++l) {
    const double al = zhao_lambda(l, alpha);
    for (int fam = 0; fam < 2; ++fam) {
      const double a = al + fam;  // lambda_l (values) and lambda_l + 1 (derivative family)
      double* A = fam ? t->hA[l] : t->gA[l];
      double* B = fam ? t->hB[l] : t->gB[l];
      A[1] = 2.0 * a;
      B[1] = 0.0;
      for (int n = 2; n <= SCF_NMAX_CAP; ++n) {
        A[n] = 2.0 * (n + a - 1.0) / n;
        B[n] = (n + 2.0 * a - 2.0) / n;
      }
    }
    double scale = 1.0, hs = 1.0;
    for (int n = 0; n <= SCF_NMAX_CAP; ++n) {
      if (n >= 1) {
        scale *= t->gA[l][n];
        hs *= t->hA[l][n];
      }
      t->gscale[l][n] = scale;
      t->hscale[l][n] = hs;
      t->gbeta[l][n] = n >= 2 ? t->gB[l][n] / (t->gA[l][n] * t->gA[l][n - 1]) : 0.0;
      t->hbeta[l][n] = n >= 2 ? t->hB[l][n] / (t->hA[l][n] * t->hA[l][n - 1]) : 0.0;
      t->gscalef[l][n] = (float)scale;
      t->hscalef[l][n] = (float)hs;
      t->gbetaf[l][n] = (float)t->gbeta[l][n];
      t->hratiof[l][n] = n >= 1 ? (float)(t->hscale[l][n - 1] / t->gscale[l][n]) : 0.f;
      t->hbetaf[l][n] = (float)t->hbeta[l][n];
      t->gAf[l][n] = (float)t->gA[l][n];
      t->gBf[l][n] = (float)t->gB[l][n];
      t->hAf[l][n] = (float)t->hA[l][n];
      t->hBf[l][n] = (float)t->hB[l][n];
    }
  }
  // Normalised associated Legendre functions without the sin^m factor.
  t->ldiag[0] = 1.0 / std::sqrt(4.0 * kPi);
  for (int l = 1; l <= SCF_LMAX_CAP; ++l) {
    t->ldiag[l] = -std::sqrt((2.0 * l + 1.0) / (2.0 * l)) * t->ldiag[l - 1];
    t->lsub[l] = std::sqrt(2.0 * l + 1.0);
  }
  for (int l = 0; l <= SCF_LMAX_CAP; ++l) {
    for (int m = 0; m <= l; ++m) {
      const int i = scf_lm(l, m);
      if (m <= l - 2) {
        const double l2 = (double)l * l, m2 = (double)m * m;
        t->la[i] = std::sqrt((4.0 * l2 - 1.0) / (l2 - m2));
        t->lb[i] = std::sqrt(((l - 1.0) * (l - 1.0) - m2) * (2.0 * l + 1.0) / ((2.0 * l - 3.0) * (l2 - m2)));
      }
      t->lk[i] = std::sqrt((double)(l - m) * (l + m + 1.0));
      // 1/N_lm = sqrt(4 pi (l+m)! / ((2l+1) (l-m)!))
      double ratio = 1.0;
      for (int k = l - m + 1; k <= l + m; ++k) ratio *= (double)k;
      t->inv_nlm[i] = std::sqrt(4.0 * kPi * ratio / (2.0 * l + 1.0));
      t->laf[i] = (float)t->la[i];
      t->lbf[i] = (float)t->lb[i];
      t->lkf[i] = (float)t->lk[i];
    }
    t->lsubf[l] = (float)t->lsub[l];
    t->ldiagf[l] = (float)t->ldiag[l];
  }
}

// S = -(2 - delta_m0) N_lm / I_nl(b) * (1/b) * Sh, and b I_nl(b) = I_nl(1), so
// the factor is independent of b:  -(2 - delta_m0) N_lm / I_nl(1).  The radial
// self-energy of pair (n, l) of the Zhao family, with a = (2l+1) alpha and
// lambda = a + 1/2, follows from the Gegenbauer norm after t = s^(1/alpha),
// xi = (t-1)/(t+1):
//   I_nl(1) = -(n+a)(n+a+1)/alpha Gamma(n+2 lambda) / (2^(4a+3) n! (n+lambda) Gamma(lambda)^2)
// (alpha = 1: -K_nl Gamma(n+4l+3) / (2^(8l+6) n! (n+2l+3/2) Gamma(2l+3/2)^2),
// K_nl = n(n+4l+3)/2 + (l+1)(2l+1)).
void scf_make_norm(int nmax, int lmax, double* norm /* 2*NC */, double alpha) {
  const int nlm = (lmax + 1) * (lmax + 2) / 2, nc = (nmax + 1) * nlm;
  for (int n = 0; n <= nmax; ++n)
    for (int l = 0; l <= lmax; ++l) {
      const double a = (2.0 * l + 1.0) * alpha, lam = zhao_lambda(l, alpha);
      const double lg = std::lgamma(n + 2.0 * lam) - (4.0 * a + 3.0) * std::log(2.0) - std::lgamma(n + 1.0) -
                        std::log(n + lam) - 2.0 * std::lgamma(lam);
      const double inl = -(n + a) * (n + a + 1.0) / alpha * std::exp(lg);
      for (int m = 0; m <= l; ++m) {
        double ratio = 1.0;
        for (int k = l - m + 1; k <= l + m; ++k) ratio /= (double)k;
        const double nlm_norm = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * ratio);
        const int i = n * nlm + scf_lm(l, m);
        const double f = -(m == 0 ? 1.0 : 2.0) * nlm_norm / inl;
        norm[i] = f;
        norm[nc + i] = (m == 0) ? 0.0 : f;
      }
    }
}

void scf_make_kscale(int nmax, int lmax, double* kscale, double alpha) {
  ScfConst* t = new ScfConst;
  scf_make_const(t, alpha);
  const int nlm = (lmax + 1) * (lmax + 2) / 2;
  for (int n = 0; n <= nmax; ++n)
    for (int l = 0; l <= lmax; ++l)
      for (int m = 0; m <= l; ++m) {
        const int i = n * nlm + scf_lm(l, m);
        kscale[2 * i] = t->gscale[l][n];
        kscale[2 * i + 1] = n >= 1 ? t->hscale[l][n - 1] : 0.0;
      }
  delete t;
}
