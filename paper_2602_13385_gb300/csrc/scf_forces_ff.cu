// Kernel 3 for double-precision particles in float-float arithmetic: the
// same field (Eq. 1a, a = -grad psi), tidal term (Sec. 2.1) and closing half
// kick as k3_forces<double>, with every step of the expansion -- the scaled
// Gegenbauer recurrences, the sums over n, the normalised Legendre
// recurrence, (u + iv)^m and the Cartesian assembly -- carried as float-float
// values (scf_ff.cuh) on the single-precision pipe, which GB300 runs 64 times
// faster than the double one.  Only the per-particle set-up (r, the unit
// vector, s, q, xi), the host's tidal difference and the final sum of the
// acceleration run in double.  Relative accuracy about 1e-13.
//
// Layout and split as k3_forces<double>: two threads per particle (degrees
// l >= Ls and l < Ls, combined through shared memory in a fixed order), the
// same block map, so either kernel serves a handle.  The force coefficients
// times their recurrence scales are staged as float-float pairs
// ((Fc gscale, Fs gscale), (Fc hscale, Fs hscale): 32 bytes a coefficient,
// as the double kernel), with the recurrence and Legendre constants.
#include "scf_device.cuh"
#include "scf_ff.cuh"
#include "scf_internal.h"

static __constant__ ScfConst c_tab;

cudaError_t scf_upload_const_forces_ff(const ScfConst* t) { return cudaMemcpyToSymbol(c_tab, t, sizeof(ScfConst)); }

namespace {

__device__ __forceinline__ FF ffz() { return {0.f, 0.f}; }

template <int LMAX, int K3_TB>
__global__ void __launch_bounds__(K3_TB) k3_forces_ff(K3Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nc = a.nc, nlm = a.nlm, NN = a.nmax + 1, L = a.lmax;
  float4* F = reinterpret_cast<float4*>(smem_raw);  // [nc][2]
  FF* GB = reinterpret_cast<FF*>(F + 2 * nc);       // [(L + 1) NN]
  FF* HB = GB + (L + 1) * NN;
  FF* LA = HB + (L + 1) * NN;                       // [nlm]
  FF* LB = LA + nlm;
  FF* LK = LB + nlm;
  FF* LS = LK + nlm;                                // [L + 1]
  FF* LD = LS + (L + 1);
  __shared__ double s_R[3], s_aR[3];
  const int tid = threadIdx.x;
  const int prog = a.blk_prog[blockIdx.x];
  const double b = a.b_prog[prog];
  {
    const double2* Fg = reinterpret_cast<const double2*>(a.F) + (size_t)prog * nc;
    const double2* Sg = reinterpret_cast<const double2*>(a.kscale);
    for (int i = tid; i < nc; i += K3_TB) {
      const double2 f = Fg[i], sc = Sg[i];
      const FF a0 = ff_from(f.x * sc.x), a1 = ff_from(f.y * sc.x), a2 = ff_from(f.x * sc.y), a3 = ff_from(f.y * sc.y);
      F[2 * i] = make_float4(a0.h, a0.l, a1.h, a1.l);
      F[2 * i + 1] = make_float4(a2.h, a2.l, a3.h, a3.l);
    }
    for (int i = tid; i < (L + 1) * NN; i += K3_TB) {
      const int l = i / NN, n = i - l * NN;
      GB[i] = ff_from(c_tab.gbeta[l][n]);
      HB[i] = ff_from(c_tab.hbeta[l][n]);
    }
    for (int i = tid; i < nlm; i += K3_TB) {
      LA[i] = ff_from(c_tab.la[i]);
      LB[i] = ff_from(c_tab.lb[i]);
      LK[i] = ff_from(c_tab.lk[i]);
    }
    for (int i = tid; i <= L; i += K3_TB) {
      LS[i] = ff_from(c_tab.lsub[i]);
      LD[i] = ff_from(c_tab.ldiag[i]);
    }
  }
  const bool has_host = a.host.n > 0 && a.com != nullptr;
  if (tid < 3) {
    s_R[tid] = has_host ? a.com[6 * prog + tid] : 0.0;
    s_aR[tid] = has_host ? a.aR[4 * prog + tid] : 0.0;
  }
  __syncthreads();

  constexpr int PPB = K3_TB / 2;  // particles per block: two threads each
  const int half = tid / PPB;
  const int pidx = tid - half * PPB;
  const int64_t k = a.blk_begin[blockIdx.x] + pidx;
  const bool live = k < a.blk_end[blockIdx.x];
  int Ls = 0;
  {
    const int tot = (L + 1) * (L + 2) / 2;
    int best = tot;
    for (int cc = 0; cc <= L + 1; ++cc) {
      const int d = abs(cc * (cc + 1) - tot);
      if (d < best) {
        best = d;
        Ls = cc;
      }
    }
  }
  ScfD4 p;
  if (live) {
    p = reinterpret_cast<const ScfD4*>(a.pos)[k];
  } else {
    p.x = p.y = p.z = p.w = 0.0;
  }
  const bool finite = scf_finite3(p.x, p.y, p.z);
  if (!finite && half == 0) atomicOr(a.status, 1u);
  const double x = finite ? p.x : 0.0, y = finite ? p.y : 0.0, z = finite ? p.z : 0.0;

  // per-particle set-up in double precision
  const double binv_d = 1.0 / b;
  const double r = sqrt(x * x + y * y + z * z);
  const double rinv = r > 0.0 ? 1.0 / r : 0.0;
  const double u_d = x * rinv, v_d = y * rinv, c_d = z * rinv;
  const double s_d = r * binv_d;
  const double q_d = 1.0 / (1.0 + s_d);
  const FF u = ff_from(u_d), v = ff_from(v_d), c = ff_from(c_d);
  const FF q = ff_from(q_d);
  const FF xi = ff_from(1.0 - 2.0 * q_d);
  const FF sq2 = ff_from(s_d * q_d * q_d);
  const FF binv = ff_from(binv_d);

  FF Wc[LMAX + 1], Ws[LMAX + 1];
  Wc[0] = ff_from(1.f);
  Ws[0] = ffz();
#pragma unroll
  for (int m = 1; m <= LMAX; ++m) {
    Wc[m] = ff_sub(ff_mul(Wc[m - 1], u), ff_mul(Ws[m - 1], v));
    Ws[m] = ff_add(ff_mul(Wc[m - 1], v), ff_mul(Ws[m - 1], u));
  }
  FF P[LMAX + 1], P1[LMAX + 1], P2[LMAX + 1];
#pragma unroll
  for (int m = 0; m <= LMAX; ++m) P1[m] = P2[m] = ffz();
  FF An = ffz(), Ax = ffz(), Ay = ffz(), Az = ffz(), pot = ffz();
  FF slq = q;                          // s^l q^(2l+1)
  FF sl1q = ff_mul(ff_mul(q, q), q);   // s^(l-1) q^(2l+1) for l >= 1

#pragma unroll
  for (int l = 0; l <= LMAX; ++l) {
    if (l > L) break;
    if (half == 1 && l >= Ls) break;
#pragma unroll
    for (int m = 0; m + 2 <= l; ++m)
      P[m] = ff_sub(ff_mul(ff_mul(LA[scf_lm(l, m)], c), P1[m]), ff_mul(LB[scf_lm(l, m)], P2[m]));
    if (l >= 1) P[l - 1] = ff_mul(ff_mul(LS[l], c), P1[l - 1]);
    P[l] = LD[l];

    if ((half == 0) == (l >= Ls)) {
      FF Z0c[LMAX + 1], Z0s[LMAX + 1], Z1c[LMAX + 1], Z1s[LMAX + 1];
      const int lm0 = scf_lm(l, 0);
#pragma unroll
      for (int m = 0; m <= l; ++m) {  // n = 0: Ch_0 = 1, no Dh_{-1} term
        const float4 f0 = F[2 * (lm0 + m)];
        Z0c[m] = {f0.x, f0.y};
        Z0s[m] = {f0.z, f0.w};
        Z1c[m] = ffz();
        Z1s[m] = ffz();
      }
      FF cm1 = ffz(), c0 = ff_from(1.f), dm1 = ffz(), d0 = ff_from(1.f);
      for (int n = 1; n < NN; ++n) {
        const FF cn = ff_sub(ff_mul(xi, c0), ff_mul(GB[l * NN + n], cm1));
        const int o = n * nlm + lm0;
#pragma unroll
        for (int m = 0; m <= l; ++m) {
          const float4 fg = F[2 * (o + m)], fh = F[2 * (o + m) + 1];
          ff_acc_prod(Z0c[m], FF{fg.x, fg.y}, cn);
          ff_acc_prod(Z0s[m], FF{fg.z, fg.w}, cn);
          ff_acc_prod(Z1c[m], FF{fh.x, fh.y}, d0);
          ff_acc_prod(Z1s[m], FF{fh.z, fh.w}, d0);
        }
        const FF dn = ff_sub(ff_mul(xi, d0), ff_mul(HB[l * NN + n], dm1));
        cm1 = c0;
        c0 = cn;
        dm1 = d0;
        d0 = dn;
      }
      // radial prefactors
      const float al4 = 4.f * (2.f * l + 1.5f);
      const FF k1 = l >= 1 ? ff_mul(binv, sl1q) : ffz();
      const FF k2a = ff_mul(binv, ff_sub(l >= 1 ? ff_mul(sl1q, (float)l) : ffz(), ff_mul(ff_mul(slq, q), (float)(2 * l + 1))));
      const FF k2b = ff_mul(ff_mul(ff_mul(binv, slq), ff_mul(q, q)), al4);
#pragma unroll
      for (int m = 0; m <= l; ++m) {
        const FF z0c = ff_acc_done(Z0c[m]), z0s = ff_acc_done(Z0s[m]);
        const FF z1c = ff_acc_done(Z1c[m]), z1s = ff_acc_done(Z1s[m]);
        const FF g0c = ff_mul(slq, z0c), g0s = ff_mul(slq, z0s);
        const FF g1c = ff_mul(k1, z0c), g1s = ff_mul(k1, z0s);
        const FF g2c = ff_add(ff_mul(k2a, z0c), ff_mul(k2b, z1c));
        const FF g2s = ff_add(ff_mul(k2a, z0s), ff_mul(k2b, z1s));
        const FF E = ff_add(ff_mul(g1c, Wc[m]), ff_mul(g1s, Ws[m]));
        const FF D = ff_add(ff_mul(g2c, Wc[m]), ff_mul(g2s, Ws[m]));
        const FF Pl = P[m];
        const FF Pd = (m < l) ? ff_neg(ff_mul(LK[scf_lm(l, m)], P[m + 1])) : ffz();
        pot = ff_add(pot, ff_mul(Pl, ff_add(ff_mul(g0c, Wc[m]), ff_mul(g0s, Ws[m]))));
        An = ff_add(An, ff_sub(ff_mul(Pl, D), ff_mul(ff_add(ff_mul(c, Pd), ff_mul(Pl, (float)m)), E)));
        Az = ff_add(Az, ff_mul(Pd, E));
        if (m >= 1) {
          const FF mP = ff_mul(Pl, (float)m);
          Ax = ff_add(Ax, ff_mul(mP, ff_add(ff_mul(g1c, Wc[m - 1]), ff_mul(g1s, Ws[m - 1]))));
          Ay = ff_sub(Ay, ff_mul(mP, ff_sub(ff_mul(g1c, Ws[m - 1]), ff_mul(g1s, Wc[m - 1]))));
        }
      }
    }  // degree owned by this half
    slq = ff_mul(slq, sq2);
    if (l >= 1) sl1q = ff_mul(sl1q, sq2);
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      P2[m] = P1[m];
      P1[m] = P[m];
    }
  }
  // the first half adds the second half's sums
  __shared__ FF s_part[5][PPB];
  if (half == 1) {
    s_part[0][pidx] = An;
    s_part[1][pidx] = Ax;
    s_part[2][pidx] = Ay;
    s_part[3][pidx] = Az;
    s_part[4][pidx] = pot;
  }
  __syncthreads();
  if (half == 1 || !live) return;
  An = ff_add(An, s_part[0][pidx]);
  Ax = ff_add(Ax, s_part[1][pidx]);
  Ay = ff_add(Ay, s_part[2][pidx]);
  Az = ff_add(Az, s_part[3][pidx]);
  pot = ff_add(pot, s_part[4][pidx]);
  // a = -grad psi (G and the sign of the basis are folded into F), in double
  const double an = ff_to_double(An);
  double gx = -(an * u_d + ff_to_double(Ax)), gy = -(an * v_d + ff_to_double(Ay)), gz = -(an * c_d + ff_to_double(Az));
  if (has_host) {
    double hx, hy, hz;
    scf_host_accel(a.host, s_R[0] + p.x, s_R[1] + p.y, s_R[2] + p.z, hx, hy, hz);
    gx += hx - s_aR[0];
    gy += hy - s_aR[1];
    gz += hz - s_aR[2];
  }
  ScfD4 out;
  out.x = gx;
  out.y = gy;
  out.z = gz;
  out.w = ff_to_double(pot);
  if (!(isfinite(out.x) && isfinite(out.y) && isfinite(out.z))) atomicOr(a.status, 2u);
  reinterpret_cast<ScfD4*>(a.acc)[k] = out;
  if (a.mode == SCF_MODE_STEP) {
    ScfD4* vel4 = reinterpret_cast<ScfD4*>(a.vel);
    ScfD4 vv = vel4[k];
    const double h = 0.5 * a.dt;
    vv.x += h * out.x;
    vv.y += h * out.y;
    vv.z += h * out.z;
    vel4[k] = vv;
  }
}

template <int TB, int LMAX>
struct K3ff {
  static void* fn() { return (void*)k3_forces_ff<LMAX, TB>; }
  static void launch(const K3Args& a, int blocks, size_t smem, cudaStream_t s) {
    k3_forces_ff<LMAX, TB><<<blocks, TB, smem, s>>>(a);
  }
};

template <int TB, typename Fn>
auto dispatch_lmax_ff(int lmax, Fn&& f) {
  if (lmax <= 2) return f(K3ff<TB, 2>());
  if (lmax <= 4) return f(K3ff<TB, 4>());
  if (lmax <= 6) return f(K3ff<TB, 6>());
  if (lmax <= 8) return f(K3ff<TB, 8>());
  if (lmax <= 10) return f(K3ff<TB, 10>());
  return f(K3ff<TB, 12>());
}

// One block size (128 threads, 64 particles) keeps the build short; the
// autotuner's other block sizes report the variant as unsupported.
constexpr int kFFThreads = 128;

template <typename Fn>
auto dispatch_ff(int lmax, Fn&& f) {
  return dispatch_lmax_ff<kFFThreads>(lmax, f);
}

}  // namespace

size_t scf_k3_ff_smem(int lmax, int nmax) {
  const int nlm = (lmax + 1) * (lmax + 2) / 2, nc = (nmax + 1) * nlm;
  return 32 * (size_t)nc + sizeof(FF) * (2 * (size_t)(lmax + 1) * (nmax + 1) + 3 * (size_t)nlm + 2 * (size_t)(lmax + 1));
}

cudaError_t scf_k3_ff_prepare(int lmax, int nmax, int tb, ScfLaunchInfo* info, int* blocks_per_sm) {
  if (tb != kFFThreads) return cudaErrorInvalidValue;
  return dispatch_ff(lmax, [&](auto k) -> cudaError_t {
    using KK = decltype(k);
    info->threads = tb;
    info->tile = tb / 2;  // two threads a particle, as the double kernel
    info->variant = 2;
    info->smem = scf_k3_ff_smem(lmax, nmax);
    cudaError_t e = cudaFuncSetAttribute(KK::fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)info->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, KK::fn(), info->threads, info->smem);
  });
}

cudaError_t scf_k3_ff_launch(const K3Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s) {
  dispatch_ff(a.lmax, [&](auto k) -> int {
    decltype(k)::launch(a, blocks, info.smem, s);
    return 0;
  });
  return cudaGetLastError();
}
