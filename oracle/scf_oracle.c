/*
 * Plain FP64 CPU oracle for the self-consistent-field (SCF) gravity step of
 * the basis-expansion N-body method (KRIOS II, arXiv:2602.13385).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition the CUDA path is checked against.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * What it computes, and where the paper defines it:
 *   - Eq. 1a/1b: potential and density as sums of a_nlm times basis functions.
 *   - Eq. 2:     separable basis psi_nlm = U_n^l(r) Y_l^m(theta, phi).
 *   - Eq. 3a/3b: coefficients from a mass-weighted particle sum,
 *                a_nlm = -sum_k m_k psi*_nlm(r_k).
 *   - Eq. 4:     Zhao (1996) radial family of exponent alpha; alpha = 1 is the
 *                Hernquist-Ostriker (1992) Gegenbauer basis, alpha = 1/2 the
 *                Clutton-Brock (1973) one.
 *   - Sec. 2 ("N individual, embarrassingly parallel integrations"): every
 *                particle is moved in -grad psi_SCF.
 *   - Sec. 2.1:  accelerating, non-rotating cluster frame whose origin follows
 *                a centre-of-mass test particle in the host potential.
 *   - App. A:    Hernquist, NFW and Miyamoto-Nagai host components, and the
 *                power-law bulge with an exponential cut-off of
 *                MWPotential2014 (lower incomplete gamma function).
 *
 * Conventions (the paper's normalisation is a bi-orthonormal basis with a
 * leading minus in Eq. 3a; the reading below is the same expansion written
 * with the normalisation I_nl of each potential-density pair):
 *   s = r/b, t = s^(1/alpha), xi = (t-1)/(t+1), a_l = (2l+1) alpha,
 *   lambda_l = a_l + 1/2 (Gegenbauer index; 2l + 3/2 at alpha = 1)
 *   Phi_nl(r) = -(1/b) s^l (1+t)^-a_l C_n^(lambda_l)(xi)            (G = 1)
 *   rho_nl(r) = K_nl/(4 pi b^3) s^(l-2+1/alpha) (1+t)^-(a_l+2) C_n^(lambda_l)(xi)
 *   K_nl      = (n + a_l)(n + a_l + 1) / alpha^2
 *               (at alpha = 1: twice n(n+4l+3)/2 + (l+1)(2l+1), the
 *               Hernquist-Ostriker constant with its 1/(2 pi) prefactor)
 *   I_nl      = int r^2 rho_nl Phi_nl dr
 * U_00 = -(1/b)(1 + s^(1/alpha))^-alpha is the form Eq. 4 prints.
 *   Real form of the coefficients (S = cosine part, T = sine part):
 *   S_nlm = (2-delta_m0)/I_nl N_lm^2 sum_k w_k m_k Phi_nl(r_k) P_l^m(cos th_k) cos(m ph_k)
 *   T_nlm = (2-delta_m0)/I_nl N_lm^2 sum_k w_k m_k Phi_nl(r_k) P_l^m(cos th_k) sin(m ph_k)
 *   N_lm^2 = (2l+1)/(4 pi) (l-m)!/(l+m)!, P_l^m with the Condon-Shortley phase.
 *   psi(x) = G sum_nl Phi_nl(r) sum_m P_l^m(cos th) [S_nlm cos(m ph) + T_nlm sin(m ph)]
 *
 * Coefficient storage: A = [S | T], each (nmax+1) * (lmax+1)(lmax+2)/2 doubles,
 * index (n, l, m) -> n * N_lm + l(l+1)/2 + m; T_nl0 is stored as 0.
 * Particle storage: 4 doubles per particle, (x, y, z, m) for positions,
 * (vx, vy, vz, unused) for velocities, (ax, ay, az, potential) for accelerations.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Special functions (textbook recurrences)                                 */
/* ------------------------------------------------------------------------ */

/* Gegenbauer polynomial C_n^alpha(xi) by the three-term recurrence
 * n C_n = 2 (n + alpha - 1) xi C_{n-1} - (n + 2 alpha - 2) C_{n-2}. */
double or_gegenbauer(int n, double alpha, double xi) {
  if (n < 0) return 0.0;
  double c_prev = 1.0;
  if (n == 0) return c_prev;
  double c = 2.0 * alpha * xi;
  for (int k = 2; k <= n; ++k) {
    double c_next = (2.0 * (k + alpha - 1.0) * xi * c - (k + 2.0 * alpha - 2.0) * c_prev) / k;
    c_prev = c;
    c = c_next;
  }
  return c;
}

/* Associated Legendre function P_l^m(cos th), 0 <= m <= l, including the
 * Condon-Shortley phase (-1)^m, from c = cos th and s = sin th >= 0:
 *   P_m^m = (-1)^m (2m-1)!! s^m,  P_{m+1}^m = c (2m+1) P_m^m,
 *   (l-m) P_l^m = c (2l-1) P_{l-1}^m - (l+m-1) P_{l-2}^m.
 * Taking s separately (rather than sqrt(1 - c^2)) keeps full accuracy next to
 * the z axis. */
static double plm_cs(int l, int m, double c, double s) {
  if (m < 0 || m > l) return 0.0;
  double pmm = 1.0;
  for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1.0) * s;
  if (l == m) return pmm;
  double pmmp1 = c * (2.0 * m + 1.0) * pmm;
  if (l == m + 1) return pmmp1;
  double pll = 0.0;
  for (int ll = m + 2; ll <= l; ++ll) {
    pll = (c * (2.0 * ll - 1.0) * pmmp1 - (ll + m - 1.0) * pmm) / (ll - m);
    pmm = pmmp1;
    pmmp1 = pll;
  }
  return pll;
}

static double sin_from_cos(double x) { return sqrt(fmax(0.0, (1.0 - x) * (1.0 + x))); }

double or_plm(int l, int m, double x) { return plm_cs(l, m, x, sin_from_cos(x)); }

/* dP_l^m(cos th)/d th, from the identity
 *   dP_l^m/dth = (P_l^{m+1} - (l+m)(l-m+1) P_l^{m-1}) / 2   (m >= 1),
 *   dP_l^0/dth = P_l^1,
 * which involves no division by sin(th) and so holds on the z axis. */
static double dplm_dtheta_cs(int l, int m, double c, double s) {
  if (m == 0) return plm_cs(l, 1, c, s);
  return 0.5 * (plm_cs(l, m + 1, c, s) - (double)(l + m) * (l - m + 1) * plm_cs(l, m - 1, c, s));
}

/* m P_l^m(cos th) / sin(th) for m >= 1, from the identity
 *   m P_l^m / sin th = -(P_{l+1}^{m+1} + (l-m+1)(l-m+2) P_{l+1}^{m-1}) / 2,
 * finite on the z axis. */
static double mplm_over_sin_cs(int l, int m, double c, double s) {
  if (m == 0) return 0.0;
  return -0.5 * (plm_cs(l + 1, m + 1, c, s) + (double)(l - m + 1) * (l - m + 2) * plm_cs(l + 1, m - 1, c, s));
}

double or_dplm_dtheta(int l, int m, double costh) { return dplm_dtheta_cs(l, m, costh, sin_from_cos(costh)); }
double or_mplm_over_sin(int l, int m, double costh) { return mplm_over_sin_cs(l, m, costh, sin_from_cos(costh)); }

/* N_lm^2 = (2l+1)/(4 pi) (l-m)!/(l+m)! */
double or_nlm2(int l, int m) {
  double ratio = 1.0;
  for (int k = l - m + 1; k <= l + m; ++k) ratio /= (double)k;
  return (2.0 * l + 1.0) / (4.0 * OR_PI) * ratio;
}

/* ------------------------------------------------------------------------ */
/* Zhao (1996) radial basis (Eq. 4), exponent alpha > 0                     */
/* ------------------------------------------------------------------------ */

double or_knl(int n, int l, double alpha) {
  const double a = (2.0 * l + 1.0) * alpha;
  return (n + a) * (n + a + 1.0) / (alpha * alpha);
}

/* Closed form of I_nl = int_0^inf r^2 rho_nl Phi_nl dr.  With t = s^(1/alpha)
 * the integrand becomes -(K_nl alpha / 4 pi b) t^a (1+t)^-(2a+2) C_n^2 dt, and
 * xi = (t-1)/(t+1) turns it into the Gegenbauer weight (1 - xi^2)^(lambda-1/2)
 * / 2^(2a+1) dxi, whose integral of C_n^2 is
 * pi 2^(1-2 lambda) Gamma(n+2 lambda) / (n! (n+lambda) Gamma(lambda)^2):
 *   I_nl = -K_nl alpha Gamma(n+2 lambda) / (2^(4a+3) n! (n+lambda) Gamma(lambda)^2) / b
 * (alpha = 1: -K_nl Gamma(n+4l+3) / (2^(8l+7) n! (n+2l+3/2) Gamma(2l+3/2)^2) / b). */
double or_inl(int n, int l, double b, double alpha) {
  const double a = (2.0 * l + 1.0) * alpha, lam = a + 0.5;
  double lg = lgamma(n + 2.0 * lam) - (4.0 * a + 3.0) * log(2.0) - lgamma(n + 1.0) - log(n + lam) -
              2.0 * lgamma(lam);
  return -or_knl(n, l, alpha) * alpha * exp(lg) / b;
}

/* s, t = s^(1/alpha) and xi = (t-1)/(t+1) of a radius. */
static void zhao_coords(double r, double b, double alpha, double* s, double* t, double* xi) {
  *s = r / b;
  *t = (alpha == 1.0) ? *s : pow(*s, 1.0 / alpha);
  *xi = (*t - 1.0) / (*t + 1.0);
}

double or_phi_nl(int n, int l, double b, double alpha, double r) {
  double s, t, xi;
  zhao_coords(r, b, alpha, &s, &t, &xi);
  const double a = (2.0 * l + 1.0) * alpha;
  return -(1.0 / b) * pow(s, l) * pow(1.0 + t, -a) * or_gegenbauer(n, a + 0.5, xi);
}

/* Phi_nl(r) / r for l >= 1 (finite at r = 0). */
double or_phi_nl_over_r(int n, int l, double b, double alpha, double r) {
  double s, t, xi;
  zhao_coords(r, b, alpha, &s, &t, &xi);
  const double a = (2.0 * l + 1.0) * alpha;
  return -(1.0 / (b * b)) * pow(s, l - 1) * pow(1.0 + t, -a) * or_gegenbauer(n, a + 0.5, xi);
}

/* dPhi_nl/dr.  With q = 1/(1+t) and dt/ds = t/(alpha s):
 *   d/ds [s^l q^a] = s^(l-1) q^a l - (2l+1) s^l q^a w,    w = q t / s,
 *   dC_n^lam/dxi = 2 lam C_{n-1}^(lam+1),  dxi/ds = 2 q w / alpha
 * (alpha = 1: w = q, dxi/ds = 2 q^2).  w = q s^(1/alpha - 1) is 0 at s = 0 for
 * alpha < 1 and unbounded for alpha > 1; there it is set to 0: the terms it
 * multiplies carry s^l, and the l = 0 radial term at r = 0, which has no
 * direction, is dropped by the caller. */
double or_dphi_nl_dr(int n, int l, double b, double alpha, double r) {
  double s, t, xi;
  zhao_coords(r, b, alpha, &s, &t, &xi);
  const double a = (2.0 * l + 1.0) * alpha, lam = a + 0.5;
  double cn = or_gegenbauer(n, lam, xi);
  double dcn = 2.0 * lam * or_gegenbauer(n - 1, lam + 1.0, xi);
  double q = 1.0 / (1.0 + t);
  double w = (alpha == 1.0) ? q : (s > 0.0 ? q * pow(s, 1.0 / alpha - 1.0) : 0.0);
  double sl = pow(s, l), qpow = pow(q, a);
  double t1 = (l > 0) ? l * pow(s, l - 1) * qpow * cn : 0.0;
  double t2 = -(2.0 * l + 1.0) * sl * qpow * w * cn;
  double t3 = sl * qpow * dcn * 2.0 * q * w / alpha;
  return -(1.0 / (b * b)) * (t1 + t2 + t3);
}

double or_rho_nl(int n, int l, double b, double alpha, double r) {
  double s, t, xi;
  zhao_coords(r, b, alpha, &s, &t, &xi);
  const double a = (2.0 * l + 1.0) * alpha;
  return or_knl(n, l, alpha) / (4.0 * OR_PI * b * b * b) * pow(s, l - 2.0 + 1.0 / alpha) * pow(1.0 + t, -(a + 2.0)) *
         or_gegenbauer(n, a + 0.5, xi);
}

/* ------------------------------------------------------------------------ */
/* Coefficients (Eq. 3b, real form)                                         */
/* ------------------------------------------------------------------------ */

static int nlm_count(int lmax) { return (lmax + 1) * (lmax + 2) / 2; }
static int lm_index(int l, int m) { return l * (l + 1) / 2 + m; }

/* Neumaier compensated accumulation. */
static void neu_add(double* sum, double* comp, double v) {
  double t = *sum + v;
  if (fabs(*sum) >= fabs(v)) *comp += (*sum - t) + v;
  else *comp += (v - t) + *sum;
  *sum = t;
}

/* Spherical angles of a point; at r = 0 the point is given theta = 0, phi = 0
 * (only l = 0 terms are non-zero there, so the choice does not matter).
 * sin(theta) comes from the cylindrical radius, not from cos(theta). */
static void sph(double x, double y, double z, double* r, double* costh, double* sinth, double* phi) {
  *r = sqrt(x * x + y * y + z * z);
  *costh = (*r > 0.0) ? z / *r : 1.0;
  *sinth = (*r > 0.0) ? sqrt(x * x + y * y) / *r : 0.0;
  if (*costh > 1.0) *costh = 1.0;
  if (*costh < -1.0) *costh = -1.0;
  if (*sinth > 1.0) *sinth = 1.0;
  *phi = atan2(y, x);
}

#define OR_CHUNKS 64

/* A = [S | T] for the particles with mask[k] != 0 (mask NULL: all). */
void or_coeffs(int64_t n_part, const double* pos, const uint8_t* mask, int nmax, int lmax, double b, double alpha,
               double* A) {
  const int nn = nmax + 1, nlm = nlm_count(lmax), nc = nn * nlm;
  /* Fixed particle chunks summed in chunk order: the result does not depend
   * on the number of threads. */
  double* part = (double*)calloc((size_t)OR_CHUNKS * 4 * nc, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
  for (int ch = 0; ch < OR_CHUNKS; ++ch) {
    int64_t k0 = n_part * ch / OR_CHUNKS, k1 = n_part * (ch + 1) / OR_CHUNKS;
    double* ssum = part + (size_t)ch * 4 * nc;
    double* scmp = ssum + nc;
    double* tsum = ssum + 2 * nc;
    double* tcmp = ssum + 3 * nc;
    double* phinl = (double*)malloc(sizeof(double) * nn * (lmax + 1));
    double* plm = (double*)malloc(sizeof(double) * nlm);
    for (int64_t k = k0; k < k1; ++k) {
      if (mask && !mask[k]) continue;
      const double* p = pos + 4 * k;
      double r, costh, sinth, phi;
      sph(p[0], p[1], p[2], &r, &costh, &sinth, &phi);
      for (int n = 0; n <= nmax; ++n)
        for (int l = 0; l <= lmax; ++l) phinl[n * (lmax + 1) + l] = or_phi_nl(n, l, b, alpha, r);
      for (int l = 0; l <= lmax; ++l)
        for (int m = 0; m <= l; ++m) plm[lm_index(l, m)] = plm_cs(l, m, costh, sinth);
      for (int n = 0; n <= nmax; ++n)
        for (int l = 0; l <= lmax; ++l)
          for (int m = 0; m <= l; ++m) {
            double w = p[3] * phinl[n * (lmax + 1) + l] * plm[lm_index(l, m)];
            int i = n * nlm + lm_index(l, m);
            neu_add(&ssum[i], &scmp[i], w * cos(m * phi));
            if (m > 0) neu_add(&tsum[i], &tcmp[i], w * sin(m * phi));
          }
    }
    free(phinl);
    free(plm);
  }
  for (int i = 0; i < nc; ++i) {
    double s = 0.0, sc = 0.0, t = 0.0, tc = 0.0;
    for (int ch = 0; ch < OR_CHUNKS; ++ch) {
      const double* q = part + (size_t)ch * 4 * nc;
      neu_add(&s, &sc, q[i] + q[nc + i]);
      neu_add(&t, &tc, q[2 * nc + i] + q[3 * nc + i]);
    }
    A[i] = s + sc;
    A[nc + i] = t + tc;
  }
  free(part);
  for (int n = 0; n <= nmax; ++n)
    for (int l = 0; l <= lmax; ++l) {
      double inl = or_inl(n, l, b, alpha);
      for (int m = 0; m <= l; ++m) {
        double f = (m == 0 ? 1.0 : 2.0) / inl * or_nlm2(l, m);
        int i = n * nlm + lm_index(l, m);
        A[i] *= f;
        A[nc + i] = (m == 0) ? 0.0 : A[nc + i] * f;
      }
    }
}

/* ------------------------------------------------------------------------ */
/* Potential and acceleration of the expansion (Eq. 1a; a = -grad psi)      */
/* ------------------------------------------------------------------------ */

/* Spherical components of -grad psi:
 *   a_r  = -sum dPhi_nl/dr  sum_m P_l^m        [S cos + T sin]
 *   a_th = -sum Phi_nl/r    sum_m dP_l^m/dth   [S cos + T sin]
 *   a_ph = -sum Phi_nl/r    sum_m m P_l^m/sin  [-S sin + T cos]
 * On the z axis phi = 0 is used (the field is smooth there and the formulas
 * above are finite).  At r = 0 the l = 0 radial term has no direction and is
 * dropped (its limit depends on the direction of approach); the l = 1 terms
 * give the finite gradient there and l >= 2 terms vanish. */
static void field_one(const double* x3, const double* A, int nmax, int lmax, double b, double alpha, double G,
                      double* out4) {
  const int nlm = nlm_count(lmax), nc = (nmax + 1) * nlm;
  double r, costh, sinth, phi;
  sph(x3[0], x3[1], x3[2], &r, &costh, &sinth, &phi);
  double pot = 0.0, ar = 0.0, ath = 0.0, aph = 0.0;
  for (int l = 0; l <= lmax; ++l) {
    for (int n = 0; n <= nmax; ++n) {
      double phi_nl = or_phi_nl(n, l, b, alpha, r);
      double dphi = (r == 0.0 && l == 0) ? 0.0 : or_dphi_nl_dr(n, l, b, alpha, r);
      double phi_r = (l >= 1) ? or_phi_nl_over_r(n, l, b, alpha, r) : 0.0;
      for (int m = 0; m <= l; ++m) {
        int i = n * nlm + lm_index(l, m);
        double S = A[i], T = A[nc + i];
        double cm = cos(m * phi), sm = sin(m * phi);
        double ang = S * cm + T * sm;
        double plm = plm_cs(l, m, costh, sinth);
        pot += phi_nl * plm * ang;
        if (!(r == 0.0 && l == 0)) ar -= dphi * plm * ang;
        if (l >= 1) {
          ath -= phi_r * dplm_dtheta_cs(l, m, costh, sinth) * ang;
          aph -= phi_r * mplm_over_sin_cs(l, m, costh, sinth) * (-S * sm + T * cm);
        }
      }
    }
  }
  double cph = cos(phi), sph_ = sin(phi);
  out4[0] = G * (ar * sinth * cph + ath * costh * cph - aph * sph_);
  out4[1] = G * (ar * sinth * sph_ + ath * costh * sph_ + aph * cph);
  out4[2] = G * (ar * costh - ath * sinth);
  out4[3] = G * pot;
}

void or_field(int64_t n_part, const double* pos, const double* A, int nmax, int lmax, double b, double alpha, double G,
              double* acc) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n_part; ++k) field_one(pos + 4 * k, A, nmax, lmax, b, alpha, G, acc + 4 * k);
}

/* Density of the expansion (Eq. 1b) at each point:
 *   rho(x) = sum_nl rho_nl(r) sum_m P_l^m(cos th) [S_nlm cos(m ph) + T_nlm sin(m ph)]
 * (mass density: no G).  Infinite at r = 0 where rho_00 has a cusp (alpha > 1/2). */
void or_density(int64_t n_part, const double* pos, const double* A, int nmax, int lmax, double b, double alpha,
                double* rho) {
  const int nlm = nlm_count(lmax), nc = (nmax + 1) * nlm;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n_part; ++k) {
    double r, costh, sinth, phi;
    sph(pos[4 * k], pos[4 * k + 1], pos[4 * k + 2], &r, &costh, &sinth, &phi);
    double sum = 0.0;
    for (int l = 0; l <= lmax; ++l)
      for (int n = 0; n <= nmax; ++n) {
        const double rnl = or_rho_nl(n, l, b, alpha, r);
        for (int m = 0; m <= l; ++m) {
          const int i = n * nlm + lm_index(l, m);
          sum += rnl * plm_cs(l, m, costh, sinth) * (A[i] * cos(m * phi) + A[nc + i] * sin(m * phi));
        }
      }
    rho[k] = sum;
  }
}

/* ------------------------------------------------------------------------ */
/* Host potential (App. A): Hernquist, NFW, Miyamoto-Nagai, cut-off bulge    */
/* ------------------------------------------------------------------------ */

enum { OR_HOST_HERNQUIST = 1, OR_HOST_NFW = 2, OR_HOST_MN = 3, OR_HOST_POWCUT = 4 };

typedef struct {
  int kind;
  double M; /* Hernquist: total mass; NFW: scale mass M_NFW; MN: disk mass; bulge: total mass M_b */
  double a; /* Hernquist: scale radius; NFW: r_s; MN: scale length a; bulge: cut-off radius r_c */
  double b; /* MN: scale height b; bulge: power-law index alpha (rho ~ r^-alpha); unused otherwise */
} or_host_comp;

/* Lower incomplete gamma function gamma(a, x) = int_0^x t^(a-1) e^-t dt,
 * a > 0, x >= 0, in long double.  For x < a + 1 the power series
 *   gamma(a, x) = x^a e^-x sum_{n>=0} x^n / (a (a+1) ... (a+n))
 * (Abramowitz & Stegun 6.5.4 with 6.5.29); otherwise gamma = Gamma(a) - Gamma(a, x)
 * with the upper function from Legendre's continued fraction
 *   Gamma(a, x) = x^a e^-x / (x + 1 - a - 1(1-a)/(x + 3 - a - 2(2-a)/(x + 5 - a - ...)))
 * (A&S 6.5.31), evaluated forwards by the modified Lentz method. */
static long double lower_gamma_l(long double a, long double x) {
  if (!(x > 0)) return 0;
  const long double eps = 4 * LDBL_EPSILON, tiny = 1e-300L;
  const long double pref = expl(a * logl(x) - x);
  if (x < a + 1) {
    long double term = 1 / a, sum = term, ap = a;
    for (int n = 1; n < 10000; ++n) {
      ap += 1;
      term *= x / ap;
      sum += term;
      if (fabsl(term) < fabsl(sum) * eps) break;
    }
    return pref * sum;
  }
  /* b_k = x + 2k + 1 - a, a_k = -k (k - a); f = b_0 + a_1/(b_1 + a_2/(b_2 + ...)) */
  long double b = x + 1 - a, c = 1 / tiny, d = 1 / b, f = d;
  for (int k = 1; k < 10000; ++k) {
    const long double an = -k * (k - a);
    b += 2;
    d = an * d + b;
    if (fabsl(d) < tiny) d = tiny;
    c = b + an / c;
    if (fabsl(c) < tiny) c = tiny;
    d = 1 / d;
    const long double delta = d * c;
    f *= delta;
    if (fabsl(delta - 1) < eps) break;
  }
  return tgammal(a) - pref * f;
}

double or_lower_gamma(double a, double x) { return (double)lower_gamma_l(a, x); }

/* Power-law bulge with an exponential cut-off (App. A, MWPotential2014):
 *   rho = rho0 (r_c/r)^alpha exp(-(r/r_c)^2),  s = (3 - alpha)/2,  x = (r/r_c)^2,
 *   M_enc = M_b gamma(s, x)/Gamma(s),  f_r = -G M_enc/r^2,
 *   psi = G M_b/Gamma(s) (gamma(1 - alpha/2, x)/r_c - gamma(s, x)/r),
 *   d f_r/dr = 2 G M_b (gamma(s, x) - x^s e^-x)/(Gamma(s) r^3). */
static void powcut_eval_l(long double GM, long double rc, long double alpha, long double r, long double* fr,
                          long double* dfr, long double* psi) {
  const long double s = 0.5L * (3 - alpha), x = (r / rc) * (r / rc), gs = tgammal(s);
  const long double lg = lower_gamma_l(s, x);
  if (psi) *psi = GM / gs * (lower_gamma_l(1 - 0.5L * alpha, x) / rc - (r > 0 ? lg / r : 0));
  if (r > 0) {
    if (fr) *fr = -GM * lg / (gs * r * r);
    if (dfr) *dfr = 2 * GM * (lg - expl(s * logl(x) - x)) / (gs * r * r * r);
  } else {
    if (fr) *fr = 0;
    if (dfr) *dfr = 0;
  }
}

typedef struct {
  int n;
  double G;
  or_host_comp c[8];
} or_host;

/* Potential and acceleration of the host at x (long double throughout). */
static void host_eval_l(const or_host* h, const long double* x, long double* a, long double* pot) {
  long double ax = 0, ay = 0, az = 0, ps = 0;
  long double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  long double r = sqrtl(r2);
  for (int i = 0; i < h->n; ++i) {
    const or_host_comp* c = &h->c[i];
    long double GM = (long double)h->G * c->M;
    if (c->kind == OR_HOST_HERNQUIST) {
      /* psi = -GM/(r+a); f_r = -G M_enc/r^2 = -GM/(r+a)^2 */
      long double A = c->a;
      ps += -GM / (r + A);
      if (r > 0) {
        long double fr = -GM / ((r + A) * (r + A));
        ax += fr * x[0] / r; ay += fr * x[1] / r; az += fr * x[2] / r;
      }
    } else if (c->kind == OR_HOST_NFW) {
      /* psi = -GM ln(1+r/rs)/r; M_enc = M g(r/rs), g(u) = ln(1+u) - u/(1+u) */
      long double rs = c->a;
      if (r > 0) {
        long double u = r / rs;
        ps += -GM * log1pl(u) / r;
        long double g = log1pl(u) - u / (1 + u);
        long double fr = -GM * g / r2;
        ax += fr * x[0] / r; ay += fr * x[1] / r; az += fr * x[2] / r;
      } else {
        ps += -GM / rs;
      }
    } else if (c->kind == OR_HOST_MN) {
      /* psi = -GM / sqrt(R^2 + z_ab^2), z_ab = sqrt(z^2+b^2) + a */
      long double A = c->a, B = c->b;
      long double zb = sqrtl(x[2] * x[2] + B * B);
      long double zab = zb + A;
      long double D2 = x[0] * x[0] + x[1] * x[1] + zab * zab;
      long double D = sqrtl(D2);
      long double D3 = D2 * D;
      ps += -GM / D;
      ax += -GM * x[0] / D3;
      ay += -GM * x[1] / D3;
      az += -GM * x[2] * zab / (zb * D3);
    } else if (c->kind == OR_HOST_POWCUT) {
      long double fr, p;
      powcut_eval_l(GM, c->a, c->b, r, &fr, NULL, &p);
      ps += p;
      if (r > 0) {
        ax += fr * x[0] / r; ay += fr * x[1] / r; az += fr * x[2] / r;
      }
    }
  }
  a[0] = ax; a[1] = ay; a[2] = az;
  *pot = ps;
}

void or_host_accel(const or_host* h, const double* x, double* a, double* pot) {
  long double xl[3] = {x[0], x[1], x[2]}, al[3], pl;
  host_eval_l(h, xl, al, &pl);
  a[0] = (double)al[0]; a[1] = (double)al[1]; a[2] = (double)al[2];
  if (pot) *pot = (double)pl;
}

/* Tidal acceleration in the accelerating, non-rotating cluster frame
 * (Sec. 2.1): a_host(R + x) - a_host(R), evaluated and differenced in long
 * double so the cancellation between the two terms costs nothing. */
void or_tidal(const or_host* h, const double* R, const double* x, double* a) {
  long double p[3] = {(long double)R[0] + x[0], (long double)R[1] + x[1], (long double)R[2] + x[2]};
  long double q[3] = {R[0], R[1], R[2]};
  long double ap[3], aq[3], pp, pq;
  host_eval_l(h, p, ap, &pp);
  host_eval_l(h, q, aq, &pq);
  for (int i = 0; i < 3; ++i) a[i] = (double)(ap[i] - aq[i]);
}

/* Tidal tensor T_ij = d a_i / d x_j of the host at x (App. A), long double.
 * Spherical components (Hernquist, NFW): a = f_r(r) x/r, so
 *   T = (f_r/r) (I - n n^T) + (d f_r/dr) n n^T,
 * with, from App. A,
 *   Hernquist: f_r = -GM/(r+a)^2,            d f_r/dr = 2GM/(r+a)^3
 *              (the printed 2GM (r/a)^3 / (r^3 (1+r/a)^3) is the same),
 *   NFW:       f_r = -GM g(u)/r^2, u = r/r_s, d f_r/dr = (2GM g/r^3) (1 - u^2 / (2 g (1+u)^2)),
 *   bulge:     f_r = -G M_enc/r^2, d f_r/dr as printed in App. A (powcut_eval_l).
 * Miyamoto-Nagai (cylindrical R, z; z_ab = sqrt(z^2+b^2) + a, D^2 = R^2 + z_ab^2):
 *   f_R = -GM R/D^3,  f_z = -GM z z_ab/(sqrt(z^2+b^2) D^3),
 *   d f_R/dR = 3GM R^2/D^5 - GM/D^3,
 *   d f_R/dz = d f_z/dR = 3GM z R z_ab/(sqrt(z^2+b^2) D^5),
 *   d f_z/dz = 3GM z^2 z_ab^2/((z^2+b^2) D^5) - GM z^2/((z^2+b^2) D^3)
 *              + GM z^2 z_ab/((z^2+b^2)^(3/2) D^3) - GM z_ab/(sqrt(z^2+b^2) D^3),
 * and a_x = f_R x/R, a_y = f_R y/R, a_z = f_z give the Cartesian entries
 *   T_xx = f_R'' x^2/R^2 + (f_R/R) y^2/R^2   (f_R'' = d f_R/dR), T_xy = (f_R'' - f_R/R) x y/R^2,
 *   T_xz = (d f_R/dz) x/R, T_zz = d f_z/dz, and the symmetric counterparts,
 * where f_R/R = -GM/D^3 and (d f_R/dz)/R stay finite on the axis. */
static void tidal_tensor_l(const or_host* h, const long double* x, long double* T) {
  for (int i = 0; i < 9; ++i) T[i] = 0;
  const long double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  const long double r = sqrtl(r2);
  for (int i = 0; i < h->n; ++i) {
    const or_host_comp* c = &h->c[i];
    const long double GM = (long double)h->G * c->M;
    if (c->kind == OR_HOST_HERNQUIST || c->kind == OR_HOST_NFW || c->kind == OR_HOST_POWCUT) {
      if (!(r > 0)) continue;
      long double fr, dfr;
      if (c->kind == OR_HOST_HERNQUIST) {
        const long double ra = r + c->a;
        fr = -GM / (ra * ra);
        dfr = 2 * GM / (ra * ra * ra);
      } else if (c->kind == OR_HOST_POWCUT) {
        powcut_eval_l(GM, c->a, c->b, r, &fr, &dfr, NULL);
      } else {
        const long double u = r / c->a;
        const long double g = log1pl(u) - u / (1 + u);
        fr = -GM * g / r2;
        dfr = 2 * GM * g / (r2 * r) * (1 - u * u / (2 * g * (1 + u) * (1 + u)));
      }
      const long double n[3] = {x[0] / r, x[1] / r, x[2] / r};
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) T[3 * a + b] += (fr / r) * ((a == b) - n[a] * n[b]) + dfr * n[a] * n[b];
    } else if (c->kind == OR_HOST_MN) {
      const long double A = c->a, B = c->b;
      const long double R2 = x[0] * x[0] + x[1] * x[1];
      const long double z = x[2];
      const long double zb2 = z * z + B * B, zb = sqrtl(zb2);
      const long double zab = zb + A;
      const long double D2 = R2 + zab * zab, D = sqrtl(D2), D3 = D2 * D, D5 = D3 * D2;
      const long double fR_over_R = -GM / D3;
      const long double dfRdR = 3 * GM * R2 / D5 - GM / D3;
      const long double dfRdz_over_R = 3 * GM * z * zab / (zb * D5);
      const long double dfzdz = 3 * GM * z * z * zab * zab / (zb2 * D5) - GM * z * z / (zb2 * D3) +
                                GM * z * z * zab / (zb2 * zb * D3) - GM * zab / (zb * D3);
      /* T_xx = dfRdR x^2/R^2 + (f_R/R) y^2/R^2 etc.; on the axis (R = 0) the
       * horizontal block is (f_R/R) I, since dfRdR -> f_R/R there */
      long double cxx, cyy, cxy;
      if (R2 > 0) {
        cxx = (dfRdR * x[0] * x[0] + fR_over_R * x[1] * x[1]) / R2;
        cyy = (dfRdR * x[1] * x[1] + fR_over_R * x[0] * x[0]) / R2;
        cxy = (dfRdR - fR_over_R) * x[0] * x[1] / R2;
      } else {
        cxx = cyy = fR_over_R;
        cxy = 0;
      }
      T[0] += cxx;
      T[4] += cyy;
      T[1] += cxy;
      T[3] += cxy;
      T[2] += dfRdz_over_R * x[0];
      T[6] += dfRdz_over_R * x[0];
      T[5] += dfRdz_over_R * x[1];
      T[7] += dfRdz_over_R * x[1];
      T[8] += dfzdz;
    }
  }
}

/* Tidal tensors at n points P = [n][3] into T = [n][9] (row-major). */
void or_tidal_tensor(const or_host* h, int64_t n, const double* P, double* T) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k) {
    long double x[3] = {P[3 * k], P[3 * k + 1], P[3 * k + 2]}, t[9];
    tidal_tensor_l(h, x, t);
    for (int i = 0; i < 9; ++i) T[9 * k + i] = (double)t[i];
  }
}

/* Host acceleration at n points P = [n][3] into a = [n][3]. */
void or_host_accel_many(const or_host* h, int64_t n, const double* P, double* a) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k) or_host_accel(h, P + 3 * k, a + 3 * k, NULL);
}

/* Tidal accelerations a_host(R + x_k) - a_host(R) for particles pos = [n][4]. */
void or_tidal_many(const or_host* h, const double* R, int64_t n, const double* pos, double* a) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k) or_tidal(h, R, pos + 4 * k, a + 3 * k);
}

/* Energy of a cluster in its accelerating, non-rotating frame (Sec. 2.1),
 * for particles pos/vel and expansion coefficients A (Eq. 1a):
 *   out[0] = K = sum_k 1/2 m_k |v_k|^2
 *   out[1] = W = 1/2 sum_k m_k psi_SCF(x_k)   (self energy; the factor 1/2
 *            because psi_SCF is the particles' own field)
 *   out[2] = U = sum_k m_k phi_tid(x_k), phi_tid(x) = psi_host(R + x) - psi_host(R) + x . a_host(R),
 *            the potential of the frame's tidal acceleration a_host(R + x) - a_host(R)
 *            (0 without a host; evaluated in long double)
 *   out[3] = K + W + U.
 * Sums run in particle order in long double. */
void or_energy(int64_t n_part, const double* pos, const double* vel, const double* A, const double* com,
               const or_host* host, int nmax, int lmax, double b, double alpha, double G, double* out) {
  double* f = (double*)malloc(sizeof(double) * 4 * (n_part > 0 ? n_part : 1));
  or_field(n_part, pos, A, nmax, lmax, b, alpha, G, f);
  const int has_host = host && host->n > 0 && com;
  long double aR[3] = {0, 0, 0}, pR = 0;
  if (has_host) {
    long double R[3] = {com[0], com[1], com[2]};
    host_eval_l(host, R, aR, &pR);
  }
  long double K = 0, W = 0, U = 0;
  for (int64_t k = 0; k < n_part; ++k) {
    const double* x = pos + 4 * k;
    const double* v = vel + 4 * k;
    const long double m = x[3];
    K += 0.5L * m * ((long double)v[0] * v[0] + (long double)v[1] * v[1] + (long double)v[2] * v[2]);
    W += 0.5L * m * f[4 * k + 3];
    if (has_host) {
      long double P[3] = {(long double)com[0] + x[0], (long double)com[1] + x[1], (long double)com[2] + x[2]};
      long double aP[3], pP;
      host_eval_l(host, P, aP, &pP);
      U += m * (pP - pR + x[0] * aR[0] + x[1] * aR[1] + x[2] * aR[2]);
    }
  }
  free(f);
  out[0] = (double)K;
  out[1] = (double)W;
  out[2] = (double)U;
  out[3] = (double)(K + W + U);
}

/* acc = -grad psi_SCF (coefficients A) + tidal term (host may be NULL). */
void or_forces(int64_t n_part, const double* pos, const double* A, const double* com, const or_host* host, int nmax,
               int lmax, double b, double alpha, double G, double* acc) {
  or_field(n_part, pos, A, nmax, lmax, b, alpha, G, acc);
  if (host && host->n > 0) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n_part; ++k) {
      double t[3];
      or_tidal(host, com, pos + 4 * k, t);
      acc[4 * k + 0] += t[0];
      acc[4 * k + 1] += t[1];
      acc[4 * k + 2] += t[2];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Kick-drift-kick leapfrog with the centre-of-mass orbit in lock-step      */
/* ------------------------------------------------------------------------ */

/* Advances nsteps of size dt.  On entry acc holds the acceleration at pos
 * (e.g. from or_forces); on exit it holds the acceleration at the new pos.
 * com = (R, V) of the cluster frame in the host frame; it moves with the same
 * kick-drift-kick in the host field alone (Sec. 2.1).  The coefficients are
 * recomputed from the particles at every force evaluation unless A_frozen is
 * given, in which case the potential is static.  mask (nullable) is the
 * coefficient set: only particles with mask[k] != 0 enter Eq. 3b, every
 * particle moves in the field (Sec. 2.2).  A_out (nullable) receives the last
 * coefficients used. */
void or_step(int64_t n_part, double* pos, double* vel, double* acc, double* com, const or_host* host, int nmax,
             int lmax, double b, double alpha, double G, double dt, int nsteps, const double* A_frozen,
             const uint8_t* mask,
             double* A_out) {
  const int nc = (nmax + 1) * nlm_count(lmax);
  double* A = (double*)malloc(sizeof(double) * 2 * nc);
  int has_host = host && host->n > 0;
  double aR[3] = {0, 0, 0};
  if (has_host) or_host_accel(host, com, aR, NULL);
  for (int st = 0; st < nsteps; ++st) {
    for (int64_t k = 0; k < n_part; ++k) {
      double* p = pos + 4 * k;
      double* v = vel + 4 * k;
      const double* a = acc + 4 * k;
      for (int d = 0; d < 3; ++d) {
        v[d] += 0.5 * dt * a[d];
        p[d] += dt * v[d];
      }
    }
    if (has_host) {
      for (int d = 0; d < 3; ++d) {
        com[3 + d] += 0.5 * dt * aR[d];
        com[d] += dt * com[3 + d];
      }
    }
    if (A_frozen) memcpy(A, A_frozen, sizeof(double) * 2 * nc);
    else or_coeffs(n_part, pos, mask, nmax, lmax, b, alpha, A);
    or_forces(n_part, pos, A, com, host, nmax, lmax, b, alpha, G, acc);
    if (has_host) {
      or_host_accel(host, com, aR, NULL);
      for (int d = 0; d < 3; ++d) com[3 + d] += 0.5 * dt * aR[d];
    }
    for (int64_t k = 0; k < n_part; ++k) {
      double* v = vel + 4 * k;
      const double* a = acc + 4 * k;
      for (int d = 0; d < 3; ++d) v[d] += 0.5 * dt * a[d];
    }
  }
  if (A_out) memcpy(A_out, A, sizeof(double) * 2 * nc);
  free(A);
}

/* ------------------------------------------------------------------------ */
/* Direct summation (the comparison of Sec. 4.1 / Fig. 11)                  */
/* ------------------------------------------------------------------------ */

/* Newtonian potential and acceleration at n_tgt points from the n_src
 * particles (no softening; a source at the target's own position is skipped). */
void or_direct(int64_t n_src, const double* src, int64_t n_tgt, const double* tgt, double G, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_tgt; ++i) {
    double ax = 0, ay = 0, az = 0, ps = 0;
    for (int64_t j = 0; j < n_src; ++j) {
      double dx = src[4 * j] - tgt[4 * i], dy = src[4 * j + 1] - tgt[4 * i + 1], dz = src[4 * j + 2] - tgt[4 * i + 2];
      double d2 = dx * dx + dy * dy + dz * dz;
      if (d2 == 0.0) continue;
      double d = sqrt(d2);
      double w = G * src[4 * j + 3] / (d2 * d);
      ax += w * dx; ay += w * dy; az += w * dz;
      ps -= G * src[4 * j + 3] / d;
    }
    out[4 * i] = ax; out[4 * i + 1] = ay; out[4 * i + 2] = az; out[4 * i + 3] = ps;
  }
}

/* Power in each l of the expansion, E_l = sum_{n,m} |a_nlm|^2 (Sec. 4.2), with
 * a_nlm the coefficients of the bi-orthonormal basis of Eq. 3a.  In terms of
 * the real form: the orthonormal-harmonic coefficient is A_nl0 = S_nl0/N_l0
 * and, for m > 0, |A_nlm|^2 = |A_nl,-m|^2 = (S^2 + T^2)/(4 N_lm^2); the
 * bi-orthonormal basis rescales each by sqrt(|I_nl|). */
void or_power_l(const double* A, int nmax, int lmax, double b, double alpha, double* El) {
  const int nlm = nlm_count(lmax), nc = (nmax + 1) * nlm;
  for (int l = 0; l <= lmax; ++l) {
    double e = 0.0;
    for (int n = 0; n <= nmax; ++n) {
      double inl = fabs(or_inl(n, l, b, alpha));
      for (int m = 0; m <= l; ++m) {
        int i = n * nlm + lm_index(l, m);
        double n2 = or_nlm2(l, m);
        if (m == 0) e += inl * A[i] * A[i] / n2;
        else e += inl * 2.0 * (A[i] * A[i] + A[nc + i] * A[nc + i]) / (4.0 * n2);
      }
    }
    El[l] = e;
  }
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
