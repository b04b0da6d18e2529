// Kernel 1 for double-precision particles in float-float arithmetic: the
// same half kick + drift and per-block coefficient partials (Eq. 3b) as
// k1_partials<double>, with the basis -- (u + iv)^m, the normalised Legendre
// and scaled Gegenbauer recurrences, the angular factors m s^l q^(2l+1) -- and
// the contraction over the tile's particles carried as float-float values
// (scf_ff.cuh) on the single-precision pipe.  The geometry of a particle
// (r, the unit vector, s, q, xi), the kick and drift, the running block sums
// (one double addition per output and tile) and the partial rows stay in
// double, so kernel 2 is unchanged.  Relative accuracy about 1e-13.
//
// Layout as k1_partials<double>: one thread per particle computes its basis
// rows for a degree, staged in shared memory ([TP][NN] radial, [TP][2l+1]
// angular, float-float pairs); thread j then contracts output (n, mm) over the
// tile's TP particles with a float-float accumulator.
#include "scf_device.cuh"
#include "scf_ff.cuh"
#include "scf_internal.h"

static __constant__ ScfConst c_tab;

cudaError_t scf_upload_const_coeffs_ff(const ScfConst* t) { return cudaMemcpyToSymbol(c_tab, t, sizeof(ScfConst)); }

namespace {

constexpr int kFFTile = 128;  // particles per tile = threads per block

__device__ __forceinline__ FF ffz() { return {0.f, 0.f}; }

template <int LMAX>
__global__ void __launch_bounds__(kFFTile) k1_partials_ff(K1Args a) {
  constexpr int TP = kFFTile;
  constexpr int YS = 2 * LMAX + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NN = a.nmax + 1, L = a.lmax, nlm = a.nlm, nc = a.nc;
  double* acc = reinterpret_cast<double*>(smem_raw);       // [2 NC] running block sums
  FF* R = reinterpret_cast<FF*>(acc + 2 * nc);             // [TP][NN]
  FF* Y = R + TP * NN;                                     // [TP][YS]
  FF* GB = Y + TP * YS;                                    // [(L + 1) NN]
  FF* LA = GB + (L + 1) * NN;                              // [nlm]
  FF* LB = LA + nlm;
  FF* LS = LB + nlm;                                       // [L + 1]
  FF* LD = LS + (L + 1);
  const int tid = threadIdx.x;
  for (int i = tid; i < 2 * nc; i += TP) acc[i] = 0.0;
  for (int i = tid; i < (L + 1) * NN; i += TP) {
    const int l = i / NN, n = i - l * NN;
    GB[i] = ff_from(c_tab.gbeta[l][n]);
  }
  for (int i = tid; i < nlm; i += TP) {
    LA[i] = ff_from(c_tab.la[i]);
    LB[i] = ff_from(c_tab.lb[i]);
  }
  for (int i = tid; i <= L; i += TP) {
    LS[i] = ff_from(c_tab.lsub[i]);
    LD[i] = ff_from(c_tab.ldiag[i]);
  }
  __syncthreads();  // the tables above are read by every thread's basis

  const int prog = a.blk_prog[blockIdx.x];
  const double binv = 1.0 / a.b_prog[prog];
  const int64_t k_begin = a.blk_begin[blockIdx.x], k_end = a.blk_end[blockIdx.x];
  ScfD4* pos4 = reinterpret_cast<ScfD4*>(a.pos);

  for (int64_t base = k_begin; base < k_end; base += TP) {
    const int64_t k = base + tid;
    double x = 0, y = 0, z = 0, mass = 0;
    if (k < k_end) {
      ScfD4 p = pos4[k];
      if (a.mode == SCF_MODE_STEP) {
        ScfD4* vel4 = reinterpret_cast<ScfD4*>(a.vel);
        const ScfD4* acc4 = reinterpret_cast<const ScfD4*>(a.acc);
        ScfD4 v = vel4[k];
        const ScfD4 g = acc4[k];
        const double h = 0.5 * a.dt, dt = a.dt;
        v.x += h * g.x;
        v.y += h * g.y;
        v.z += h * g.z;
        p.x += dt * v.x;
        p.y += dt * v.y;
        p.z += dt * v.z;
        vel4[k] = v;
        pos4[k] = p;
      }
      if (scf_finite3(p.x, p.y, p.z) && isfinite(p.w)) {
        x = p.x;
        y = p.y;
        z = p.z;
        mass = (a.mask == nullptr || a.mask[k]) ? p.w : 0.0;
      } else {
        atomicOr(a.status, 1u);
      }
    }
    // geometry in double precision
    const double r = sqrt(x * x + y * y + z * z);
    const double rinv = r > 0.0 ? 1.0 / r : 0.0;
    const double s_d = r * binv;
    const double q_d = 1.0 / (1.0 + s_d);
    const FF u = ff_from(x * rinv), v = ff_from(y * rinv), c = ff_from(z * rinv);
    const FF xi = ff_from(1.0 - 2.0 * q_d);
    const FF sq2 = ff_from(s_d * q_d * q_d);
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
    FF pre = ff_from(mass * q_d);  // m_k s^l q^(2l+1) at l = 0

#pragma unroll
    for (int l = 0; l <= LMAX; ++l) {
      if (l > L) break;
#pragma unroll
      for (int m = 0; m + 2 <= l; ++m)
        P[m] = ff_sub(ff_mul(ff_mul(LA[scf_lm(l, m)], c), P1[m]), ff_mul(LB[scf_lm(l, m)], P2[m]));
      if (l >= 1) P[l - 1] = ff_mul(ff_mul(LS[l], c), P1[l - 1]);
      P[l] = LD[l];
      {  // radial rows: scaled Gegenbauer values Ch_n = C_n / gscale[l][n]
        FF cm1 = ffz(), c0 = ff_from(1.f);
        FF* Rt = R + tid * NN;
        Rt[0] = c0;
        for (int n = 1; n < NN; ++n) {
          const FF cn = ff_sub(ff_mul(xi, c0), ff_mul(GB[l * NN + n], cm1));
          cm1 = c0;
          c0 = cn;
          Rt[n] = cn;
        }
      }
      {  // angular rows with the radial prefactor
        FF* Yt = Y + tid * YS;
#pragma unroll
        for (int m = 0; m <= l; ++m) {
          const FF pp = ff_mul(pre, P[m]);
          Yt[m] = ff_mul(pp, Wc[m]);
          if (m >= 1) Yt[l + m] = ff_mul(pp, Ws[m]);
        }
      }
      __syncthreads();
      // contraction over the tile's particles
      const int nout = NN * (2 * l + 1);
      for (int j = tid; j < nout; j += TP) {
        const int mm = j / NN, n = j - mm * NN;
        FF sum = ffz();
#pragma unroll 4
        for (int t = 0; t < TP; ++t) ff_acc_prod(sum, R[t * NN + n], Y[t * YS + mm]);
        const int idx = (mm <= l) ? n * nlm + scf_lm(l, mm) : nc + n * nlm + scf_lm(l, mm - l);
        acc[idx] += ff_to_double(ff_acc_done(sum));
      }
      __syncthreads();
      pre = ff_mul(pre, sq2);
#pragma unroll
      for (int m = 0; m <= l; ++m) {
        P2[m] = P1[m];
        P1[m] = P[m];
      }
    }
  }
  __syncthreads();
  double* out = a.partials + (size_t)blockIdx.x * 2 * nc;
  for (int i = tid; i < 2 * nc; i += TP) {
    const int ii = i < nc ? i : i - nc;
    const int n = ii / nlm, lm = ii - n * nlm;
    int l = 0;
    while ((l + 1) * (l + 2) / 2 <= lm) ++l;
    out[i] = acc[i] * c_tab.gscale[l][n];  // undo the scaling of the staged C_n
  }
}

template <int LMAX>
struct K1ff {
  static void* fn() { return (void*)k1_partials_ff<LMAX>; }
  static void launch(const K1Args& a, int blocks, size_t smem, cudaStream_t s) {
    k1_partials_ff<LMAX><<<blocks, kFFTile, smem, s>>>(a);
  }
};

template <typename Fn>
auto dispatch_k1_ff(int lmax, Fn&& f) {
  if (lmax <= 2) return f(K1ff<2>());
  if (lmax <= 4) return f(K1ff<4>());
  if (lmax <= 6) return f(K1ff<6>());
  if (lmax <= 8) return f(K1ff<8>());
  if (lmax <= 10) return f(K1ff<10>());
  return f(K1ff<12>());
}

int lmax_bucket(int lmax) { return lmax <= 2 ? 2 : lmax <= 4 ? 4 : lmax <= 6 ? 6 : lmax <= 8 ? 8 : lmax <= 10 ? 10 : 12; }

}  // namespace

cudaError_t scf_k1_ff_prepare(int lmax, int nmax, int tp, ScfLaunchInfo* info, int* blocks_per_sm) {
  if (tp != kFFTile) return cudaErrorInvalidValue;
  const int nlm = (lmax + 1) * (lmax + 2) / 2, nc = (nmax + 1) * nlm, NN = nmax + 1, LB = lmax_bucket(lmax);
  info->threads = kFFTile;
  info->tile = kFFTile;
  info->variant = 2;
  info->smem = sizeof(double) * 2 * (size_t)nc +
               sizeof(FF) * ((size_t)kFFTile * (NN + 2 * LB + 1) + (size_t)(lmax + 1) * NN + 2 * (size_t)nlm +
                             2 * (size_t)(lmax + 1));
  if (info->smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  return dispatch_k1_ff(lmax, [&](auto k) -> cudaError_t {
    using KK = decltype(k);
    cudaError_t e = cudaFuncSetAttribute(KK::fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)info->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, KK::fn(), info->threads, info->smem);
  });
}

cudaError_t scf_k1_ff_launch(const K1Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s) {
  dispatch_k1_ff(a.lmax, [&](auto k) -> int {
    decltype(k)::launch(a, blocks, info.smem, s);
    return 0;
  });
  return cudaGetLastError();
}
