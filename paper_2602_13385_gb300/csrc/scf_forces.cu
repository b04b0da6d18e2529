// Kernel 3: acceleration of the expansion (Eq. 1a, a = -grad psi) at every
// particle, plus the tidal acceleration of the accelerating, non-rotating
// cluster frame (Sec. 2.1), and in step mode the closing half kick.
//
// One thread per particle (two in double precision, see the degree split
// below).  The block's force coefficients
// F_nlm = -G {S,T}_nlm / (b N_lm) are staged in shared memory as 4-vectors
// (F gscale[l][n], F hscale[l][n-1]) of the cosine and sine parts; every
// thread then runs, for each l, the scaled Gegenbauer recurrences
//   Ch_n = xi Ch_{n-1} - gbeta[l][n] Ch_{n-2},  Dh_n = xi Dh_{n-1} - hbeta[l][n] Dh_{n-2}
// (Ch_n = C_n^alpha / gscale, Dh_n = C_n^{alpha+1} / hscale: one multiply and
// one FMA a step, see ScfConst) and accumulates, for m = 0..l,
//   Z0 = sum_n F_nlm C_n^alpha(xi),  Z1 = sum_n F_nlm C_{n-1}^{alpha+1}(xi)
// as sums of the scaled coefficients times Ch_n and Dh_{n-1}, from which
//   G_lm   = s^l q^(2l+1) Z0                               (potential),
//   G_lm/r = (1/b) s^(l-1) q^(2l+1) Z0                     (l >= 1),
//   G'_lm  = (1/b) [(l s^(l-1) q^(2l+1) - (2l+1) s^l q^(2l+2)) Z0 + 4 alpha s^l q^(2l+3) Z1]
// and the Cartesian gradient is assembled with the identities listed in
// scf_device.cuh.  No division by r or sin(theta) appears, so particles at
// the origin or on the z axis need no special case (at r = 0 the l = 0 term,
// whose direction is undefined there, contributes nothing).
#include "scf_device.cuh"
#include "scf_internal.h"

static __constant__ ScfConst c_tab;

cudaError_t scf_upload_const_forces(const ScfConst* t) { return cudaMemcpyToSymbol(c_tab, t, sizeof(ScfConst)); }

namespace {

template <typename T> struct Vec4;
template <> struct Vec4<double> { using type = ScfD4; };
template <> struct Vec4<float> { using type = float4; };
template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

template <typename T> __device__ __forceinline__ T tla(int i) { return sizeof(T) == 8 ? (T)c_tab.la[i] : (T)c_tab.laf[i]; }
template <typename T> __device__ __forceinline__ T tlb(int i) { return sizeof(T) == 8 ? (T)c_tab.lb[i] : (T)c_tab.lbf[i]; }
template <typename T> __device__ __forceinline__ T tlk(int i) { return sizeof(T) == 8 ? (T)c_tab.lk[i] : (T)c_tab.lkf[i]; }
template <typename T> __device__ __forceinline__ T tlsub(int l) { return sizeof(T) == 8 ? (T)c_tab.lsub[l] : (T)c_tab.lsubf[l]; }
template <typename T> __device__ __forceinline__ T tldiag(int l) { return sizeof(T) == 8 ? (T)c_tab.ldiag[l] : (T)c_tab.ldiagf[l]; }
template <typename T> __device__ __forceinline__ T tgbeta(int l, int n) { return sizeof(T) == 8 ? (T)c_tab.gbeta[l][n] : (T)c_tab.gbetaf[l][n]; }
template <typename T> __device__ __forceinline__ T thbeta(int l, int n) { return sizeof(T) == 8 ? (T)c_tab.hbeta[l][n] : (T)c_tab.hbetaf[l][n]; }

// Radial family of exponent alpha != 1 (GEN): recurrence steps from the
// handle's tables in device memory (read-only cache; warp-uniform addresses)
// instead of the constant bank.  (Staging them in shared memory per block
// measured slower: more registers, one block fewer per SM.)
template <typename T, bool GEN>
__device__ __forceinline__ T k3_gbeta(const K3Args& a, int l, int n) {
  if constexpr (GEN) return sizeof(T) == 8 ? (T)__ldg(&a.tab->gbeta[l][n]) : (T)__ldg(&a.tab->gbetaf[l][n]);
  else return tgbeta<T>(l, n);
}
template <typename T, bool GEN>
__device__ __forceinline__ T k3_hbeta(const K3Args& a, int l, int n) {
  if constexpr (GEN) return sizeof(T) == 8 ? (T)__ldg(&a.tab->hbeta[l][n]) : (T)__ldg(&a.tab->hbetaf[l][n]);
  else return thbeta<T>(l, n);
}
__device__ __forceinline__ double k3_pow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float k3_pow(float x, float y) { return powf(x, y); }

// NNF > 0: the shape (nmax, lmax) = (NNF - 1, LMAX) fixed at compile time
// (single precision): every coefficient offset is an immediate
// and the radial loop is unrolled by 4 (or 5, or 2) without a remainder.
constexpr int k3_unroll(int nnf) { return (nnf - 1) % 4 == 0 ? 4 : (nnf - 1) % 5 == 0 ? 5 : 2; }
template <typename T, int LMAX, int K3_TB, bool GEN, int NNF>
__device__ __forceinline__ void k3_body(const K3Args& a) {
  using V4 = typename Vec4<T>::type;
  using V2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // [NC] scaled (cosine, sine) force coefficients of this block's progenitor,
  // one shared-memory load for the four FMAs of an (n, l, m).  Double:
  // (Fc gscale_n, Fs gscale_n, Fc hscale_{n-1}, Fs hscale_{n-1}).  Single:
  // (Fc gscale_n, Fs gscale_n) only, the alpha + 1 family taking the
  // per-(l, n) ratio hratio = hscale_{n-1} / gscale_n on its recurrence value
  // instead (8 instead of 16 bytes per load).
  constexpr bool kF2 = sizeof(T) == 4;
  V4* F = reinterpret_cast<V4*>(smem_raw);
  V2* F2 = reinterpret_cast<V2*>(smem_raw);
  // single precision: the per-(l, n) recurrence constants (gbeta, hbeta,
  // hratio) staged beside the coefficients from the handle's table (coalesced
  // 16-byte loads), one broadcast shared load per radial step instead of
  // three constant-bank loads with runtime indices
  float4* CS = reinterpret_cast<float4*>(smem_raw + ((sizeof(V2) * (size_t)a.nc + 15) & ~size_t(15)));
  __shared__ double s_R[3], s_aR[3];
  const int tid = threadIdx.x;
  const int prog = a.blk_prog[blockIdx.x];
  const double b = a.b_prog[prog];
  if constexpr (kF2)
    for (int i = tid; i < (a.lmax + 1) * (a.nmax + 1); i += K3_TB) CS[i] = a.cs[i];
  {
    const V2* Fg = reinterpret_cast<const V2*>(a.F) + (size_t)prog * a.nc;
    const V2* Sg = reinterpret_cast<const V2*>(a.kscale);
    for (int i = tid; i < a.nc; i += K3_TB) {
      if constexpr (kF2) {
        F2[i] = Fg[i];  // kernel 2 wrote them times gscale
      } else {
        const V2 f = Fg[i], sc = Sg[i];
        V4 q;
        q.x = f.x * sc.x;
        q.y = f.y * sc.x;
        q.z = f.x * sc.y;
        q.w = f.y * sc.y;
        F[i] = q;
      }
    }
  }
  const bool has_host = a.host.n > 0 && a.com != nullptr;
  if (tid < 3) {
    s_R[tid] = has_host ? a.com[6 * prog + tid] : 0.0;
    s_aR[tid] = has_host ? a.aR[4 * prog + tid] : 0.0;
  }
  // single precision: the values of the tidal differences that depend on R
  // alone, formed by kernel 2 (or the force-coefficient set-up) for this R
  __shared__ float s_tid[kF2 ? SCF_HOST_CAP : 1][SCF_TIDAL_W];
  if constexpr (kF2) {
    if (has_host && tid < a.host.n * SCF_TIDAL_W)
      (&s_tid[0][0])[tid] = a.tid[(size_t)prog * SCF_HOST_CAP * SCF_TIDAL_W + tid];
  }
  __syncthreads();

  // Double precision splits each particle's degrees between two warps: warps
  // of the first half take l >= Ls (and finish the particle), warps of the
  // second half l < Ls, with Ls chosen so that both halves have about the
  // same sum of (l + 1) (the work of a degree).  Twice as many, half as long
  // warp tasks fill the 2 FP64 units per SM more evenly at the end of the
  // grid.  The branch on a degree's owner is uniform across a warp.
  constexpr int SPLIT = sizeof(T) == 8 ? 2 : 1;
  constexpr int PPB = K3_TB / SPLIT;  // particles per block
  const int half = tid / PPB;
  const int pidx = tid - half * PPB;
  const int64_t k = a.blk_begin[blockIdx.x] + pidx;
  const bool live = k < a.blk_end[blockIdx.x];
  if (SPLIT == 1 && !live) return;
  int Ls = 0;
  if constexpr (SPLIT == 2) {
    const int tot = (a.lmax + 1) * (a.lmax + 2) / 2;
    int best = tot;
    for (int c = 0; c <= a.lmax + 1; ++c) {
      const int d = abs(c * (c + 1) - tot);
      if (d < best) {
        best = d;
        Ls = c;
      }
    }
  }
  V4 p;
  if (live) {
    p = reinterpret_cast<const V4*>(a.pos)[k];
  } else {
    p.x = p.y = p.z = p.w = (T)0;
  }
  const bool finite = scf_finite3(p.x, p.y, p.z);
  if (!finite && half == 0) atomicOr(a.status, 1u);
  const T x = finite ? p.x : (T)0, y = finite ? p.y : (T)0, z = finite ? p.z : (T)0;

  const T binv = (T)(1.0 / b);
  const T r = sqrt(x * x + y * y + z * z);
  const T rinv = r > (T)0 ? (T)1 / r : (T)0;
  const T u = x * rinv, v = y * rinv, c = z * rinv;
  const T s = r * binv;
  // alpha = 1: q = 1/(1+s), prefactor s^l q^(2l+1).  alpha != 1: with
  // t = s^(1/alpha), q = 1/(1+t), the prefactor is s^l q^((2l+1) alpha) and
  // the radial derivative carries w = q t / s (= q at alpha = 1), set to 0 at
  // s = 0 where the terms it multiplies vanish (l >= 1) or have no direction
  const T t = GEN ? k3_pow(s, (T)a.inv_alpha) : s;
  const T q = (T)1 / ((T)1 + t);
  const T xi = (T)1 - (T)2 * q;
  const T qa = GEN ? k3_pow(q, (T)a.alpha) : q;
  const T w = GEN ? (s > (T)0 ? q * k3_pow(s, (T)(a.inv_alpha - 1.0)) : (T)0) : q;
  const T sq2 = s * qa * qa;

  T Wc[LMAX + 1], Ws[LMAX + 1];
  Wc[0] = 1;
  Ws[0] = 0;
#pragma unroll
  for (int m = 1; m <= LMAX; ++m) {
    Wc[m] = Wc[m - 1] * u - Ws[m - 1] * v;
    Ws[m] = Wc[m - 1] * v + Ws[m - 1] * u;
  }
  T P[LMAX + 1], P1[LMAX + 1], P2[LMAX + 1];
  T An = 0, Ax = 0, Ay = 0, Az = 0, pot = 0;
  T slq = qa;              // s^l q^((2l+1) alpha)
  T sl1q = qa * qa * qa;    // s^(l-1) q^((2l+1) alpha) for l >= 1 (set at l = 1)
  const int NN = NNF > 0 ? NNF : a.nmax + 1;
  const int NLM = NNF > 0 ? (LMAX + 1) * (LMAX + 2) / 2 : a.nlm;

#pragma unroll
  for (int l = 0; l <= LMAX; ++l) {
    if (NNF == 0 && l > a.lmax) break;
    if (SPLIT == 2 && half == 1 && l >= Ls) break;
#pragma unroll
    for (int m = 0; m + 2 <= l; ++m) P[m] = tla<T>(scf_lm(l, m)) * c * P1[m] - tlb<T>(scf_lm(l, m)) * P2[m];
    if (l >= 1) P[l - 1] = tlsub<T>(l) * c * P1[l - 1];
    P[l] = tldiag<T>(l);

    if (SPLIT == 1 || (half == 0) == (l >= Ls)) {
    // the (cosine, sine) sums over n of the Ch_n terms (Z0) and of the
    // Dh_{n-1} terms (Z1): scalars in double precision, packed pairs in single
    T Z0c[LMAX + 1], Z0s[LMAX + 1], Z1c[LMAX + 1], Z1s[LMAX + 1];
    V2 Z0[LMAX + 1], Z1[LMAX + 1];
    const int lm0 = scf_lm(l, 0);
#pragma unroll
    for (int m = 0; m <= l; ++m) {  // n = 0: Ch_0 = 1, no Dh_{-1} term
      if constexpr (kF2) {
        Z0[m] = F2[lm0 + m];
        Z1[m].x = 0;
        Z1[m].y = 0;
      } else {
        const V4 f0 = F[lm0 + m];
        Z0c[m] = f0.x;
        Z0s[m] = f0.y;
        Z1c[m] = 0;
        Z1s[m] = 0;
      }
    }
    {
      T cm1 = 0, c0 = 1;  // Ch_{n-2}, Ch_{n-1}
      T dm1 = 0, d0 = 1;  // Dh_{n-2}, Dh_{n-1}
      // The single-precision alpha = 1 kernel of the (20,10)-class degree bucket
      // runs the radial loop unrolled by two (measured 3% faster there); every
      // other instantiation keeps the compiler's choice (unrolling measured
      // slower at lmax 8 and for alpha != 1).
      const float4* CSl = CS + l * NN;
      auto radial_step = [&](int n) {
        T gbn, hbn;
        float hrn = 0.f;
        if constexpr (kF2) {
          const float4 cst = CSl[n];
          gbn = cst.x;
          hbn = cst.y;
          hrn = cst.z;
        } else {
          gbn = k3_gbeta<T, GEN>(a, l, n);
          hbn = k3_hbeta<T, GEN>(a, l, n);
        }
        const T cn = xi * c0 - gbn * cm1;
        const int o = n * NLM + lm0;
        if constexpr (kF2) {
          // one packed FMA per (cosine, sine) pair: each lane rounds as the
          // scalar fmaf, in the same order over n
          const float2 cc = make_float2(cn, cn), dv = make_float2(d0 * hrn, d0 * hrn);
#pragma unroll
          for (int m = 0; m <= l; ++m) {
            const float2 fv = F2[o + m];
            Z0[m] = __ffma2_rn(fv, cc, Z0[m]);
            Z1[m] = __ffma2_rn(fv, dv, Z1[m]);
          }
        } else {
#pragma unroll
          for (int m = 0; m <= l; ++m) {
            const V4 fv = F[o + m];
            Z0c[m] += fv.x * cn;
            Z0s[m] += fv.y * cn;
            Z1c[m] += fv.z * d0;
            Z1s[m] += fv.w * d0;
          }
        }
        const T dn = xi * d0 - hbn * dm1;
        cm1 = c0;
        c0 = cn;
        dm1 = d0;
        d0 = dn;
      };
      if constexpr (NNF > 0) {
        constexpr int U = k3_unroll(NNF);
        static_assert((NNF - 1) % U == 0, "the radial loop has no remainder");
#pragma unroll U
        for (int n = 1; n < NNF; ++n) radial_step(n);
      } else if constexpr (kF2 && !GEN && LMAX == 10) {
#pragma unroll 2
        for (int n = 1; n < NN; ++n) radial_step(n);
      } else {
        for (int n = 1; n < NN; ++n) radial_step(n);
      }
    }
    // radial prefactors; al4 = 4 lambda_l / alpha (4 (2l + 3/2) at alpha = 1)
    const T al4 = GEN ? (T)(4.0 * (2 * l + 1) + 2.0 * a.inv_alpha) : (T)(4.0 * (2.0 * l + 1.5));
    const T k1 = (l >= 1) ? binv * sl1q : (T)0;                                  // G/r per Z0
    const T k2a = binv * ((l >= 1 ? (T)l * sl1q : (T)0) - (T)(2 * l + 1) * slq * w);  // G' per Z0
    const T k2b = binv * al4 * slq * q * w;                                       // G' per Z1
    // The radial factors of degree l (slq, k1, k2a, k2b) multiply whole sums
    // over m, so the sums over m are formed first:
    //   Q0 = Z0c W_c + Z0s W_s, Q1 = Z1c W_c + Z1s W_s (W = W_m), and
    //   psi += slq sum Pl Q0,  A_n += k2a sum Pl Q0 + k2b sum Pl Q1 - k1 sum (c Pd + m Pl) Q0,
    //   A_z += k1 sum Pd Q0,  A_x += k1 sum m Pl (Z0c W_c,m-1 + Z0s W_s,m-1),
    //   A_y -= k1 sum m Pl (Z0c W_s,m-1 - Z0s W_c,m-1).
    T sP0 = 0, sP1 = 0, sE = 0, sZ = 0, sX = 0, sY = 0;
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      const T z0c = kF2 ? Z0[m].x : Z0c[m], z0s = kF2 ? Z0[m].y : Z0s[m];
      const T Q0 = z0c * Wc[m] + z0s * Ws[m];
      const T Q1 = kF2 ? Z1[m].x * Wc[m] + Z1[m].y * Ws[m] : Z1c[m] * Wc[m] + Z1s[m] * Ws[m];
      const T Pl = P[m];
      const T Pd = (m < l) ? -tlk<T>(scf_lm(l, m)) * P[m + 1] : (T)0;
      sP0 += Pl * Q0;
      sP1 += Pl * Q1;
      sZ += Pd * Q0;
      if (m >= 1) {
        const T mPl = (T)m * Pl;
        sE += (c * Pd + mPl) * Q0;
        sX += mPl * (z0c * Wc[m - 1] + z0s * Ws[m - 1]);
        sY += mPl * (z0c * Ws[m - 1] - z0s * Wc[m - 1]);
      } else {
        sE += c * Pd * Q0;
      }
    }
    pot += slq * sP0;
    An += k2a * sP0 + k2b * sP1 - k1 * sE;
    Az += k1 * sZ;
    Ax += k1 * sX;
    Ay -= k1 * sY;
    }  // degree owned by this half
    slq *= sq2;
    if (l >= 1) sl1q *= sq2;
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      P2[m] = P1[m];
      P1[m] = P[m];
    }
  }
  if constexpr (SPLIT == 2) {  // the first half adds the second half's sums
    __shared__ T s_part[5][PPB];
    if (half == 1) {
      s_part[0][pidx] = An;
      s_part[1][pidx] = Ax;
      s_part[2][pidx] = Ay;
      s_part[3][pidx] = Az;
      s_part[4][pidx] = pot;
    }
    __syncthreads();
    if (half == 1 || !live) return;
    An += s_part[0][pidx];
    Ax += s_part[1][pidx];
    Ay += s_part[2][pidx];
    Az += s_part[3][pidx];
    pot += s_part[4][pidx];
  }
  // a = -grad psi (G and the sign of the basis are folded into F)
  V4 out;
  if constexpr (sizeof(T) == 8) {
    double gx = -(An * u + Ax), gy = -(An * v + Ay), gz = -(An * c + Az);
    if (has_host) {
      // a_host(R + x) - a_host(R) in double precision
      double hx, hy, hz;
      scf_host_accel(a.host, s_R[0] + (double)p.x, s_R[1] + (double)p.y, s_R[2] + (double)p.z, hx, hy, hz);
      gx += hx - s_aR[0];
      gy += hy - s_aR[1];
      gz += hz - s_aR[2];
    }
    out.x = gx;
    out.y = gy;
    out.z = gz;
  } else {
    float gx = -(An * u + Ax), gy = -(An * v + Ay), gz = -(An * c + Az);
    if (has_host) {
      // the same difference in single precision without cancellation
      float tx, ty, tz;
      scf_tidal_f32(a.host, s_tid, (float)s_R[0], (float)s_R[1], (float)s_R[2], p.x, p.y, p.z, tx, ty, tz);
      gx += tx;
      gy += ty;
      gz += tz;
    }
    out.x = gx;
    out.y = gy;
    out.z = gz;
  }
  out.w = pot;
  if (!(isfinite(out.x) && isfinite(out.y) && isfinite(out.z))) atomicOr(a.status, 2u);
  if constexpr (sizeof(T) == 8) {
    if (a.mode == SCF_MODE_ADJ_J) {
      // adjoint through the coefficients: F holds the field of A^J, so
      // xbar_k += m_k f(x_k; A^J); then the drift x_t = x_{t-1} + dt v is undone
      ScfD4* xb = reinterpret_cast<ScfD4*>(a.adj.xbar) + k;
      ScfD4 X = *xb;
      X.x += p.w * out.x;
      X.y += p.w * out.y;
      X.z += p.w * out.z;
      *xb = X;
      if (a.adj.drift) {
        ScfD4* vb = reinterpret_cast<ScfD4*>(a.adj.vbar) + k;
        ScfD4 V = *vb;
        V.x += a.dt * X.x;
        V.y += a.dt * X.y;
        V.z += a.dt * X.z;
        *vb = V;
      }
      return;
    }
  }
  reinterpret_cast<V4*>(a.acc)[k] = out;
  if (a.mode == SCF_MODE_STEP) {
    V4* vel4 = reinterpret_cast<V4*>(a.vel);
    V4 vv = a.vel_in ? reinterpret_cast<const V4*>(a.vel_in)[k] : vel4[k];
    const T h = (T)(0.5 * a.dt);
    vv.x += h * out.x;
    vv.y += h * out.y;
    vv.z += h * out.z;
    vel4[k] = vv;
  }
}

template <typename T, int LMAX, int K3_TB, bool GEN = false, int NNF = 0>
__global__ void __launch_bounds__(K3_TB) k3_forces(K3Args a) {
  k3_body<T, LMAX, K3_TB, GEN, NNF>(a);
}

// Single precision in 320-thread blocks, held to two blocks per SM (at most
// 96 registers): 20 resident warps per SM against 16 with 256-thread blocks
// at 111 registers, which measured 3% faster at (nmax, lmax) = (20, 10).
template <typename T, int LMAX, bool GEN = false, int NNF = 0>
__global__ void __launch_bounds__(320, 2) k3_forces_w(K3Args a) {
  k3_body<T, LMAX, 320, GEN, NNF>(a);
}

template <typename T, int TB, int LMAX, bool GEN = false, int NNF = 0>
struct K3At {
  static constexpr bool kW = sizeof(T) == 4 && TB == 320;
  static void* fn() {
    if constexpr (kW) return (void*)k3_forces_w<T, LMAX, GEN, NNF>;
    else return (void*)k3_forces<T, LMAX, TB, GEN, NNF>;
  }
  static cudaError_t launch(const K3Args& a, int blocks, size_t smem, cudaStream_t s) {
    if constexpr (kW) k3_forces_w<T, LMAX, GEN, NNF><<<blocks, TB, smem, s>>>(a);
    else k3_forces<T, LMAX, TB, GEN, NNF><<<blocks, TB, smem, s>>>(a);
    return cudaGetLastError();
  }
};

int lmax_bucket(int lmax) {
  if (lmax <= 2) return 2;
  if (lmax <= 4) return 4;
  if (lmax <= 6) return 6;
  if (lmax <= 8) return 8;
  if (lmax <= 10) return 10;
  return 12;
}

// (nmax, lmax) = (20, 10) and (10, 5) (the paper's stream model) in single
// precision run the compile-time shape (any alpha).
template <typename T, int TB, typename Fn, bool GEN = false>
auto dispatch_lmax(int lmax, Fn&& f, int nmax = -1) {
  if constexpr (sizeof(T) == 4) {
    if (lmax == 10 && nmax == 20) return f(K3At<T, TB, 10, GEN, 21>());
    if (lmax == 5 && nmax == 10) return f(K3At<T, TB, 5, GEN, 11>());
  }
  switch (lmax_bucket(lmax)) {
    case 2: return f(K3At<T, TB, 2, GEN>());
    case 4: return f(K3At<T, TB, 4, GEN>());
    case 6: return f(K3At<T, TB, 6, GEN>());
    case 8: return f(K3At<T, TB, 8, GEN>());
    case 10: return f(K3At<T, TB, 10, GEN>());
    default: return f(K3At<T, TB, 12, GEN>());
  }
}

// Kernel 3 instantiations: blocks of 64, 128 or 256 threads, and 320 in single
// precision (the autotuner's choices).
template <typename T, typename Fn>
auto dispatch_k3(int tb, int lmax, int nmax, Fn&& f) {
  switch (tb) {
    case 64: return dispatch_lmax<T, 64>(lmax, f, nmax);
    case 256: return dispatch_lmax<T, 256>(lmax, f, nmax);
    case 320:
      if constexpr (sizeof(T) == 4) return dispatch_lmax<T, 320>(lmax, f, nmax);
      [[fallthrough]];
    default: return dispatch_lmax<T, 128>(lmax, f, nmax);
  }
}

template <typename T, bool GEN = false>
cudaError_t prepare_t(int lmax, int nmax, int tb, ScfLaunchInfo* info, int* blocks_per_sm) {
  const int nlm = (lmax + 1) * (lmax + 2) / 2, nc = (nmax + 1) * nlm;
  if (tb != 64 && tb != 128 && tb != 256 && !(tb == 320 && sizeof(T) == 4)) return cudaErrorInvalidValue;
  if (GEN && tb != 128) return cudaErrorInvalidValue;
  auto body = [&](auto k) -> cudaError_t {
    using KK = decltype(k);
    info->threads = tb;
    info->tile = sizeof(T) == 8 ? tb / 2 : tb;  // double: two warps share a particle (split degrees)
    info->variant = GEN ? 3 : 0;
    // scaled (cosine, sine) per coefficient; double also the alpha + 1 family's;
    // single also the per-(l, n) recurrence constants (a float4 each)
    info->smem = sizeof(T) == 4 ? ((sizeof(float) * 2 * (size_t)nc + 15) & ~size_t(15)) +
                                      sizeof(float4) * (size_t)(lmax + 1) * (nmax + 1)
                                : sizeof(T) * 4 * (size_t)nc;
    cudaError_t e = cudaFuncSetAttribute(KK::fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)info->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, KK::fn(), info->threads, info->smem);
  };
  if constexpr (GEN) return dispatch_lmax<T, 128, decltype(body)&, true>(lmax, body, nmax);
  else return dispatch_k3<T>(tb, lmax, nmax, body);
}

}  // namespace

cudaError_t scf_k3_prepare(int precision, int lmax, int nmax, int tb, ScfLaunchInfo* info, int* blocks_per_sm) {
  if (precision == 1) return prepare_t<float>(lmax, nmax, tb, info, blocks_per_sm);
  return prepare_t<double>(lmax, nmax, tb, info, blocks_per_sm);
}

cudaError_t scf_k3_gen_prepare(int precision, int lmax, int nmax, ScfLaunchInfo* info, int* blocks_per_sm) {
  if (precision == 1) return prepare_t<float, true>(lmax, nmax, 128, info, blocks_per_sm);
  return prepare_t<double, true>(lmax, nmax, 128, info, blocks_per_sm);
}

cudaError_t scf_k3_launch(int precision, const K3Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s) {
  cudaError_t err = cudaSuccess;
  auto go = [&](auto k) -> int {
    err = decltype(k)::launch(a, blocks, info.smem, s);
    return 0;
  };
  if (info.variant == 3) {  // radial family of exponent alpha != 1, 128-thread blocks
    if (precision == 1) dispatch_lmax<float, 128, decltype(go)&, true>(a.lmax, go, a.nmax);
    else dispatch_lmax<double, 128, decltype(go)&, true>(a.lmax, go);
  } else if (precision == 1) {
    dispatch_k3<float>(info.threads, a.lmax, a.nmax, go);
  } else {
    dispatch_k3<double>(info.threads, a.lmax, a.nmax, go);
  }
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}
