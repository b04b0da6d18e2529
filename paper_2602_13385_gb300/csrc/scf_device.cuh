// Device-side building blocks of the SCF kernels (internal header).
//
// Formulation used on the GPU (the same expansion as the C ABI documents,
// arranged so that no division by r or sin(theta) appears anywhere):
//   n_hat = x/r (0 at r = 0), u = n_x, v = n_y, c = n_z,
//   W_m = (u + i v)^m = C_m + i S_m   (so W_m = sin^m(th) e^{i m ph}),
//   Pb_lm(c) = N_lm P_l^m(c) / sin^m(th): the normalised associated Legendre
//              function without its sin^m factor (a polynomial in c),
//   s = r/b, q = 1/(1+s), xi = (s-1)/(s+1) = 1 - 2q,
//   radial factor of degree l: s^l q^(2l+1) C_n^(2l+3/2)(xi)  (Eq. 4, alpha = 1).
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
};

// Host-side generation of the tables (scf_tables.cu).
void scf_make_const(ScfConst* t);

// Host potential parameters passed by value to the kernels.
struct ScfHostParams {
  int n;
  int kind[SCF_HOST_CAP];
  double GM[SCF_HOST_CAP], a[SCF_HOST_CAP], b[SCF_HOST_CAP];
};

// Four doubles with the 16-byte alignment the ABI promises for particle arrays.
struct __align__(16) ScfD4 {
  double x, y, z, w;
};

__host__ __device__ constexpr int scf_lm(int l, int m) { return l * (l + 1) / 2 + m; }

// Acceleration of the analytic host (App. A) at (x, y, z), double precision.
//   Hernquist: f_r = -GM/(r+a)^2;  NFW: f_r = -GM [ln(1+u) - u/(1+u)]/r^2, u = r/r_s;
//   Miyamoto-Nagai: f_R = -GM R/D^3, f_z = -GM z z_ab/(sqrt(z^2+b^2) D^3),
//   z_ab = sqrt(z^2+b^2) + a, D^2 = R^2 + z_ab^2.
__device__ __forceinline__ void scf_host_accel(const ScfHostParams& hp, double x, double y, double z, double& ax,
                                               double& ay, double& az) {
  ax = 0.0;
  ay = 0.0;
  az = 0.0;
  const double r2 = x * x + y * y + z * z;
  const double r = sqrt(r2);
  const double rinv = r > 0.0 ? 1.0 / r : 0.0;
  for (int i = 0; i < hp.n; ++i) {
    const double GM = hp.GM[i], A = hp.a[i];
    if (hp.kind[i] == 1) {  // Hernquist
      const double ra = r + A;
      const double f = -GM / (ra * ra) * rinv;
      ax += f * x;
      ay += f * y;
      az += f * z;
    } else if (hp.kind[i] == 2) {  // NFW
      const double u = r / A;
      const double g = log1p(u) - u / (1.0 + u);
      const double f = -GM * g * rinv * rinv * rinv;
      ax += f * x;
      ay += f * y;
      az += f * z;
    } else if (hp.kind[i] == 3) {  // Miyamoto-Nagai
      const double B = hp.b[i];
      const double zb = sqrt(z * z + B * B);
      const double zab = zb + A;
      const double D2 = x * x + y * y + zab * zab;
      const double D3 = D2 * sqrt(D2);
      const double f = -GM / D3;
      ax += f * x;
      ay += f * y;
      az += f * z * zab / zb;
    }
  }
}

template <typename T>
__device__ __forceinline__ bool scf_finite3(T x, T y, T z) {
  return isfinite(x) && isfinite(y) && isfinite(z);
}
