// Device-side building blocks of the SCF kernels (internal header).
//
// Formulation used on the GPU (the same expansion as the C ABI documents,
// arranged so that no division by r or sin(theta) appears anywhere):
//   n_hat = x/r (0 at r = 0), u = n_x, v = n_y, c = n_z,
//   W_m = (u + i v)^m = C_m + i S_m   (so W_m = sin^m(th) e^{i m ph}),
//   Pb_lm(c) = N_lm P_l^m(c) / sin^m(th): the normalised associated Legendre
//              function without its sin^m factor (a polynomial in c),
//   s = r/b, q = 1/(1+s), xi = (s-1)/(s+1) = 1 - 2q,
//   radial factor of degree l: s^l q^(2l+1) C_n^(2l+3/2)(xi)  (Eq. 4, alpha = 1);
//   for the Zhao family of exponent alpha, t = s^(1/alpha) replaces s in q and
//   xi, q^((2l+1) alpha) replaces q^(2l+1), and the index is (2l+1) alpha + 1/2.
// Coefficient pass (Eq. 3b):  Sh_nlm = sum_k m_k s^l q^(2l+1) C_n Pb_lm C_m(k), Th: S_m.
// Field (Eq. 1a):  psi = sum_lm Pb_lm [Gc_lm C_m + Gs_lm S_m],
//   G_lm(r) = s^l q^(2l+1) sum_n F_nlm C_n,  F = -G {S,T}_nlm / (b N_lm),
// and grad psi from dPb_lm/dc = -sqrt((l-m)(l+m+1)) Pb_l,m+1 and
//   r grad c = z_hat - c n_hat,  r grad W_m = m W_{m-1} (x_hat + i y_hat) - m W_m n_hat.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define SCF_NMAX_CAP 40
#define SCF_LMAX_CAP 12
#define SCF_NLM_CAP ((SCF_LMAX_CAP + 1) * (SCF_LMAX_CAP + 2) / 2)
#define SCF_HOST_CAP 8

// Recurrence and normalisation tables, generated on the host in double
// precision (scf_tables.cu) and uploaded to each translation unit's constant
// bank once per device.
struct ScfConst {
  // Gegenbauer recurrence C_n = gA[l][n] xi C_{n-1} - gB[l][n] C_{n-2}, C_0 = 1,
  // for alpha = 2l + 3/2 (g*) and alpha + 1 (h*); index n >= 1 (gB[l][1] = 0).
  double gA[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  double gB[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  double hA[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  double hB[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  float gAf[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  float gBf[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  float hAf[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  float hBf[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  // Normalised Legendre (without sin^m): Pb_lm = la c Pb_{l-1,m} - lb Pb_{l-2,m} (m <= l-2),
  // Pb_{l,l-1} = lsub[l] c Pb_{l-1,l-1}, Pb_ll = ldiag[l] (a constant).
  double la[SCF_NLM_CAP], lb[SCF_NLM_CAP], lk[SCF_NLM_CAP];
  double lsub[SCF_LMAX_CAP + 1], ldiag[SCF_LMAX_CAP + 1];
  float laf[SCF_NLM_CAP], lbf[SCF_NLM_CAP], lkf[SCF_NLM_CAP];
  float lsubf[SCF_LMAX_CAP + 1], ldiagf[SCF_LMAX_CAP + 1];
  double inv_nlm[SCF_NLM_CAP];  // 1 / N_lm
  // Scaled Gegenbauer polynomials for the register-tiled coefficient kernel:
  // Ch_n = C_n / gscale[l][n] with gscale[l][n] = gA[l][1] ... gA[l][n] obey
  // Ch_n = xi Ch_{n-1} - gbeta[l][n] Ch_{n-2}, Ch_0 = 1, Ch_1 = xi,
  // gbeta[l][n] = gB[l][n] / (gA[l][n] gA[l][n-1]) (one multiply and one FMA a step).
  float gbetaf[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  float gscalef[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  // The same scaling for both families in the field kernel: Ch (alpha) and
  // Dh (alpha + 1, scale hscale = hA[l][1] ... hA[l][n], step hbeta).
  double gbeta[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1], gscale[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  double hbeta[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1], hscale[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  float hbetaf[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1], hscalef[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
  // hscale[l][n-1] / gscale[l][n] (0 at n = 0): lets the single-precision field
  // kernel use one scaled coefficient F gscale_n for both families
  float hratiof[SCF_LMAX_CAP + 1][SCF_NMAX_CAP + 1];
};

// Host-side generation of the tables (scf_tables.cu) for the radial family of
// exponent alpha (1: Hernquist-Ostriker, the tables of the constant banks).
void scf_make_const(ScfConst* t, double alpha = 1.0);

// Host potential parameters passed by value to the kernels.
struct ScfHostParams {
  int n;
  int kind[SCF_HOST_CAP];
  double GM[SCF_HOST_CAP], a[SCF_HOST_CAP], b[SCF_HOST_CAP];
};

// Forward-mode dual number (value, derivative) in double precision: the
// adjoint kernels evaluate the same formulas on duals to get exact
// directional derivatives (Hessian-vector products) of the expansion and of
// the host potential.
struct Dual {
  double v, d;
  __host__ __device__ Dual() : v(0.0), d(0.0) {}
  __host__ __device__ Dual(double x) : v(x), d(0.0) {}
  __host__ __device__ Dual(double x, double dx) : v(x), d(dx) {}
};
__host__ __device__ inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__host__ __device__ inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__host__ __device__ inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__host__ __device__ inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__host__ __device__ inline Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__host__ __device__ inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
__host__ __device__ inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
__host__ __device__ inline Dual& operator+=(Dual& a, Dual b) { return a = a + b; }
__host__ __device__ inline Dual& operator-=(Dual& a, Dual b) { return a = a - b; }
__host__ __device__ inline Dual& operator*=(Dual& a, Dual b) { return a = a * b; }
__host__ __device__ inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
__host__ __device__ inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
__device__ inline Dual sqrt(Dual a) {
  const double s = ::sqrt(a.v);
  return Dual(s, s > 0.0 ? 0.5 * a.d / s : 0.0);
}
__device__ inline Dual log1p(Dual a) { return Dual(::log1p(a.v), a.d / (1.0 + a.v)); }
__device__ inline bool isfinite(Dual a) { return ::isfinite(a.v) && ::isfinite(a.d); }
__device__ inline double value_of(Dual a) { return a.v; }
__device__ inline double value_of(double a) { return a; }

// Four doubles with the 16-byte alignment the ABI promises for particle arrays.
struct __align__(16) ScfD4 {
  double x, y, z, w;
};

__host__ __device__ constexpr int scf_lm(int l, int m) { return l * (l + 1) / 2 + m; }

// Regularised lower incomplete gamma function P(a, x) = gamma(a, x) / Gamma(a)
// (a > 0, x >= 0) for the cut-off power-law bulge of MWPotential2014 (App. A).
// Kummer's series P = x^a e^-x / Gamma(a + 1) sum_k x^k / ((a+1)...(a+k)) for
// x < a + 1; otherwise P = 1 - Q with Q = x^a e^-x / Gamma(a) times Legendre's
// continued fraction 1/(x + 1 - a - 1(1 - a)/(x + 3 - a - 2(2 - a)/(x + 5 - a - ...))),
// evaluated forwards by the modified Lentz algorithm (Thompson & Barnett 1986).
template <typename F>
__device__ __forceinline__ F scf_gamma_p_t(F a, F x) {
  if (!(x > F(0))) return F(0);
  const F eps = sizeof(F) == 8 ? F(1e-16) : F(3e-8), tiny = sizeof(F) == 8 ? F(1e-300) : F(1e-30);
  const F lpre = a * log(x) - x - lgamma(a);
  if (x < a + F(1)) {
    F ap = a, term = F(1) / a, sum = term;
    for (int k = 0; k < 500; ++k) {
      ap += F(1);
      term *= x / ap;
      sum += term;
      if (fabs(term) < fabs(sum) * eps) break;
    }
    return sum * exp(lpre);
  }
  F b = x + F(1) - a, c = F(1) / tiny, d = F(1) / b, h = d;
  for (int k = 1; k < 500; ++k) {
    const F an = -F(k) * (F(k) - a);
    b += F(2);
    d = an * d + b;
    if (fabs(d) < tiny) d = tiny;
    c = b + an / c;
    if (fabs(c) < tiny) c = tiny;
    d = F(1) / d;
    const F del = d * c;
    h *= del;
    if (fabs(del - F(1)) < eps) break;
  }
  return F(1) - exp(lpre) * h;
}
__device__ __forceinline__ double scf_gamma_p(double a, double x) { return scf_gamma_p_t<double>(a, x); }
__device__ __forceinline__ float scf_gamma_pf(float a, float x) { return scf_gamma_p_t<float>(a, x); }
// Dual argument: dP/dx = x^(a-1) e^-x / Gamma(a).
__device__ __forceinline__ Dual scf_gamma_p(double a, Dual x) {
  const double v = scf_gamma_p(a, x.v);
  const double dens = x.v > 0.0 ? exp((a - 1.0) * log(x.v) - x.v - lgamma(a)) : 0.0;
  return Dual(v, x.d * dens);
}
// Acceleration of the analytic host (App. A) at (x, y, z), double precision.
//   Hernquist: f_r = -GM/(r+a)^2;  NFW: f_r = -GM [ln(1+u) - u/(1+u)]/r^2, u = r/r_s;
//   Miyamoto-Nagai: f_R = -GM R/D^3, f_z = -GM z z_ab/(sqrt(z^2+b^2) D^3),
//   z_ab = sqrt(z^2+b^2) + a, D^2 = R^2 + z_ab^2;
//   cut-off power-law bulge (a = r_c, b = alpha): f_r = -GM P(s, (r/r_c)^2)/r^2, s = (3 - alpha)/2.
// One host component's acceleration; N is double or Dual (for derivatives).
template <typename N>
__device__ __forceinline__ void scf_host_comp_accel(int kind, N GM, N A, N B, N x, N y, N z, N& ax, N& ay, N& az) {
  ax = N(0.0);
  ay = N(0.0);
  az = N(0.0);
  if (kind == 1 || kind == 2) {
    const N r2 = x * x + y * y + z * z;
    if (!(r2 > N(0.0))) return;
    const N r = sqrt(r2);
    const N rinv = N(1.0) / r;
    N f;
    if (kind == 1) {  // Hernquist
      const N ra = r + A;
      f = -GM / (ra * ra) * rinv;
    } else {  // NFW
      const N u = r / A;
      const N g = log1p(u) - u / (N(1.0) + u);
      f = -GM * g * rinv * rinv * rinv;
    }
    ax = f * x;
    ay = f * y;
    az = f * z;
  } else if (kind == 4) {  // cut-off power-law bulge (the index alpha is not a variable of N)
    const N r2 = x * x + y * y + z * z;
    if (!(r2 > N(0.0))) return;
    const double s = 0.5 * (3.0 - value_of(B));
    const N r = sqrt(r2);
    const N f = -GM * scf_gamma_p(s, r2 / (A * A)) / (r2 * r);
    ax = f * x;
    ay = f * y;
    az = f * z;
  } else if (kind == 3) {  // Miyamoto-Nagai
    const N zb = sqrt(z * z + B * B);
    const N zab = zb + A;
    const N D2 = x * x + y * y + zab * zab;
    const N D3 = D2 * sqrt(D2);
    const N f = -GM / D3;
    ax = f * x;
    ay = f * y;
    az = f * z * zab / zb;
  }
}

template <typename N>
__device__ __forceinline__ void scf_host_accel_t(const ScfHostParams& hp, N x, N y, N z, N& ax, N& ay, N& az) {
  ax = N(0.0);
  ay = N(0.0);
  az = N(0.0);
  for (int i = 0; i < hp.n; ++i) {
    N cx, cy, cz;
    scf_host_comp_accel<N>(hp.kind[i], N(hp.GM[i]), N(hp.a[i]), N(hp.b[i]), x, y, z, cx, cy, cz);
    ax += cx;
    ay += cy;
    az += cz;
  }
}

__device__ __forceinline__ void scf_host_accel(const ScfHostParams& hp, double x, double y, double z, double& ax,
                                               double& ay, double& az) {
  scf_host_accel_t<double>(hp, x, y, z, ax, ay, az);
}

// Potential of the analytic host (App. A) at (x, y, z), double precision:
//   Hernquist -GM/(r+a);  NFW -GM ln(1 + r/r_s)/r (-GM/r_s at r = 0);
//   Miyamoto-Nagai -GM/sqrt(R^2 + (sqrt(z^2+b^2) + a)^2);
//   cut-off bulge GM (P(1 - alpha/2, x) Gamma(1 - alpha/2)/(Gamma(s) r_c) - P(s, x)/r), x = (r/r_c)^2.
__device__ __forceinline__ double scf_host_pot(const ScfHostParams& hp, double x, double y, double z) {
  double psi = 0.0;
  const double r = sqrt(x * x + y * y + z * z);
  for (int i = 0; i < hp.n; ++i) {
    const double GM = hp.GM[i], A = hp.a[i];
    if (hp.kind[i] == 1) {
      psi -= GM / (r + A);
    } else if (hp.kind[i] == 2) {
      psi -= r > 0.0 ? GM * log1p(r / A) / r : GM / A;
    } else if (hp.kind[i] == 3) {
      const double zab = sqrt(z * z + hp.b[i] * hp.b[i]) + A;
      psi -= GM / sqrt(x * x + y * y + zab * zab);
    } else if (hp.kind[i] == 4) {
      const double s = 0.5 * (3.0 - hp.b[i]), s2 = 1.0 - 0.5 * hp.b[i], X = (r / A) * (r / A);
      psi += GM * (scf_gamma_p(s2, X) * exp(lgamma(s2) - lgamma(s)) / A - (r > 0.0 ? scf_gamma_p(s, X) / r : 0.0));
    }
  }
  return psi;
}

// Tidal acceleration a_host(R + x) - a_host(R) in single precision, written
// as divided differences so that no two large terms are subtracted: with
// P = R + x, r0 = |R|, r1 = |P| and dr = r1 - r0 = (2 R.x + |x|^2)/(r1 + r0),
//   spherical parts (a = -g(r) r_vec):  a(P) - a(R) = -[g(r1) x + (g(r1) - g(r0)) R],
//     Hernquist  g = GM / p(r), p = r (r+a)^2,  p1 - p0 = dr (r1^2 + r1 r0 + r0^2 + 2a(r1+r0) + a^2),
//     NFW        g = GM h(u)/r^3, u = r/r_s,   h1 - h0 = log1p(d) - d/(1+u1), d = (dr/r_s)/(1+u0),
//                1/r1^3 - 1/r0^3 = -dr (r0^2 + r0 r1 + r1^2)/(r0^3 r1^3);
//   Miyamoto-Nagai (D^2 = R_cyl^2 + (zb + a)^2, zb = sqrt(z^2 + b^2)):
//     D1^2 - D0^2 = 2(Rx x + Ry y) + x^2 + y^2 + (zb1 - zb0)(zab1 + zab0),
//     zb1 - zb0 = (2 Rz z + z^2)/(zb1 + zb0),  D1 - D0 = (D1^2 - D0^2)/(D1 + D0),
//     1/D1^3 - 1/D0^3 = -(D1 - D0)(D1^2 + D1 D0 + D0^2)/(D0^3 D1^3),
//     a_z = -GM z v/D^3 with v = 1 + a/zb, v1 - v0 = -a (zb1 - zb0)/(zb1 zb0).
//   cut-off power-law bulge (g = GM P(s, X)/r^3, X = (r/r_c)^2, s = (3 - alpha)/2):
//     g1 - g0 = GM [(P1 - P0)/r1^3 + P0 (1/r1^3 - 1/r0^3)], X1 - X0 = dr (r1 + r0)/r_c^2,
//     P1 - P0 = int_X0^X1 t^(s-1) e^-t dt / Gamma(s) by six-point Gauss-Legendre
//     quadrature when |X1 - X0| <= min(X0/2, 2) (the integrand is smooth there), else
//     the plain difference (no cancellation then).
// Relative error of the result a few float ulps for any |x|/|R| (checked
// against the long-double difference of the oracle).
//
// Every value that depends on R alone (r0, and per component p0; u0, h0;
// zb0, D0, 1/(D0^2 D0); X0, P0; ...) is the same for all the particles of a
// progenitor: scf_tidal_prep_f32 forms them once per block (component i in
// thread i, the same single-precision formulas), and the per-particle part
// reads them from shared memory.  Components with the same b (the three
// Miyamoto-Nagai disks of a disk fit) share zb1, 1/zb1 and zb1 - zb0.  The
// reciprocals are the hardware approximation (__fdividef, 2 ulp), the
// arguments lying far inside its range.
constexpr int SCF_TIDAL_W = 8;   // floats per component; [7] holds r0
__device__ __forceinline__ float scf_rcpf(float x) { return __fdividef(1.f, x); }

__device__ __forceinline__ void scf_tidal_prep_f32(const ScfHostParams& hp, int i, float Rx, float Ry, float Rz,
                                                   float* t) {
  const float r0 = sqrtf(Rx * Rx + Ry * Ry + Rz * Rz);
  const float A = (float)hp.a[i];
  for (int j = 0; j < SCF_TIDAL_W; ++j) t[j] = 0.f;
  t[7] = r0;
  if (hp.kind[i] == 1) {  // Hernquist: 1/p0
    t[0] = 1.f / (r0 * (r0 + A) * (r0 + A));
  } else if (hp.kind[i] == 2) {  // NFW: h0, 1/(1 + u0), 1/r0^3, 1/r_s
    const float u0 = r0 / A;
    t[0] = log1pf(u0) - u0 / (1.f + u0);
    t[1] = 1.f / (1.f + u0);
    t[2] = 1.f / (r0 * r0 * r0);
    t[3] = 1.f / A;
  } else if (hp.kind[i] == 3) {  // Miyamoto-Nagai: zb0, zab0, D0^2, D0, 1/(D0^2 D0), v0, 1/zb0
    const float B = (float)hp.b[i];
    const float zb0 = sqrtf(Rz * Rz + B * B), zab0 = zb0 + A;
    const float D2_0 = Rx * Rx + Ry * Ry + zab0 * zab0, D0 = sqrtf(D2_0);
    t[0] = zb0;
    t[1] = zab0;
    t[2] = D2_0;
    t[3] = D0;
    t[4] = 1.f / (D2_0 * D0);
    t[5] = 1.f + A / zb0;
    t[6] = 1.f / zb0;
  } else if (hp.kind[i] == 4) {  // cut-off power-law bulge: X0, P0, 1/r0^3, 1/r_c^2, lgamma(s)
    const float s = 0.5f * (3.f - (float)hp.b[i]);
    const float ia2 = 1.f / (A * A);
    t[0] = r0 * r0 * ia2;
    t[1] = scf_gamma_pf(s, t[0]);
    t[2] = 1.f / (r0 * r0 * r0);
    t[3] = ia2;
    t[4] = lgammaf(s);
  }
}

__device__ __forceinline__ void scf_tidal_f32(const ScfHostParams& hp, const float (*tr)[SCF_TIDAL_W], float Rx,
                                              float Ry, float Rz, float x, float y, float z, float& ax, float& ay,
                                              float& az) {
  ax = 0.f;
  ay = 0.f;
  az = 0.f;
  const float Px = Rx + x, Py = Ry + y, Pz = Rz + z;
  const float r0 = tr[0][7];
  const float r1 = sqrtf(Px * Px + Py * Py + Pz * Pz);
  const float xx = x * x + y * y + z * z;
  const float dr = (2.f * (Rx * x + Ry * y + Rz * z) + xx) * scf_rcpf(r1 + r0);
  float lastB = __int_as_float(0x7fffffff), zb1 = 0.f, izb1 = 0.f, dzb = 0.f;  // NaN: the first disk computes them
  for (int i = 0; i < hp.n; ++i) {
    const float GM = (float)hp.GM[i], A = (float)hp.a[i];
    const float* t = tr[i];
    if (hp.kind[i] == 1) {  // Hernquist
      const float p1 = r1 * (r1 + A) * (r1 + A);
      const float dp = dr * (r1 * r1 + r1 * r0 + r0 * r0 + 2.f * A * (r1 + r0) + A * A);
      const float ip1 = scf_rcpf(p1);
      const float g1 = GM * ip1;
      const float dg = -GM * dp * ip1 * t[0];
      ax -= g1 * x + dg * Rx;
      ay -= g1 * y + dg * Ry;
      az -= g1 * z + dg * Rz;
    } else if (hp.kind[i] == 2) {  // NFW
      const float u1 = r1 * t[3];
      const float iu1 = scf_rcpf(1.f + u1);
      const float h1 = log1pf(u1) - u1 * iu1;
      const float d = dr * t[3] * t[1];
      const float dh = log1pf(d) - d * iu1;
      const float i1 = scf_rcpf(r1 * r1 * r1);
      const float di = -dr * (r0 * r0 + r0 * r1 + r1 * r1) * t[2] * i1;
      const float g1 = GM * h1 * i1;
      const float dg = GM * (dh * i1 + t[0] * di);
      ax -= g1 * x + dg * Rx;
      ay -= g1 * y + dg * Ry;
      az -= g1 * z + dg * Rz;
    } else if (hp.kind[i] == 3) {  // Miyamoto-Nagai
      const float B = (float)hp.b[i];
      const float zb0 = t[0], zab0 = t[1], D2_0 = t[2], D0 = t[3];
      if (B != lastB) {
        zb1 = sqrtf(Pz * Pz + B * B);
        izb1 = scf_rcpf(zb1);
        dzb = (2.f * Rz * z + z * z) * scf_rcpf(zb1 + zb0);
        lastB = B;
      }
      const float zab1 = zb1 + A;
      const float D2_1 = Px * Px + Py * Py + zab1 * zab1;
      const float dD2 = 2.f * (Rx * x + Ry * y) + x * x + y * y + dzb * (zab1 + zab0);
      const float D1 = sqrtf(D2_1);
      const float dD = dD2 * scf_rcpf(D1 + D0);
      const float i1 = scf_rcpf(D2_1 * D1);
      const float di = -dD * (D2_1 + D1 * D0 + D2_0) * t[4] * i1;
      ax -= GM * (x * i1 + Rx * di);
      ay -= GM * (y * i1 + Ry * di);
      const float v1 = 1.f + A * izb1;
      const float dv = -A * dzb * izb1 * t[6];
      az -= GM * (z * v1 * i1 + Rz * (dv * i1 + t[5] * di));
    } else if (hp.kind[i] == 4) {  // cut-off power-law bulge
      const float s = 0.5f * (3.f - (float)hp.b[i]);
      const float X0 = t[0], P0 = t[1], ia2 = t[3];
      const float X1 = r1 * r1 * ia2;
      const float dX = dr * (r1 + r0) * ia2;
      const float P1 = scf_gamma_pf(s, X1);
      float dP;
      if (fabsf(dX) <= fminf(0.5f * X0, 2.f)) {
        // Gauss-Legendre nodes +-xi_j and weights w_j on [-1, 1] (6 points)
        const float gx[3] = {0.2386191860831969f, 0.6612093864662645f, 0.9324695142031521f};
        const float gw[3] = {0.4679139345726910f, 0.3607615730481386f, 0.1713244923791704f};
        const float lg = t[4], hw = 0.5f * dX, cm = X0 + hw;
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float t1 = cm + hw * gx[j], t2 = cm - hw * gx[j];
          acc += gw[j] * (expf((s - 1.f) * logf(t1) - t1 - lg) + expf((s - 1.f) * logf(t2) - t2 - lg));
        }
        dP = hw * acc;
      } else {
        dP = P1 - P0;
      }
      const float i1 = scf_rcpf(r1 * r1 * r1);
      const float di = -dr * (r0 * r0 + r0 * r1 + r1 * r1) * t[2] * i1;
      const float g1 = GM * P1 * i1;
      const float dg = GM * (dP * i1 + P0 * di);
      ax -= g1 * x + dg * Rx;
      ay -= g1 * y + dg * Ry;
      az -= g1 * z + dg * Rz;
    }
  }
}

template <typename T>
__device__ __forceinline__ bool scf_finite3(T x, T y, T z) {
  return isfinite(x) && isfinite(y) && isfinite(z);
}
