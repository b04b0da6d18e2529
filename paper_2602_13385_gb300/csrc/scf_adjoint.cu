// Adjoint (reverse mode) of the SCF force and of the leapfrog, double precision.
//
// The forward step (kick-drift-kick, Sec. 2.1, with a(x, R) = f(x; A(x)) +
// a_host(R + x) - a_host(R) and the centre orbit R, V stepped in the host
// alone) is reversed level by level.  At level t the accelerations a(x_t, R_t)
// are pulled back along d_k = w vbar_k; w = dt/2 at the first and last level,
// dt in between, since a(x_t) feeds both the closing kick of step t and the
// opening kick of step t+1.  The pull-back of the self-gravity has two parts:
//
//   xbar_k += (da_k/dx_k) d_k                        own-position term (Hessian of psi, symmetric),
//   xbar_k += m_k f(x_k; A^J),  A^J = sum_i d_i . grad B(x_i)   through the coefficients,
//
// where B is the normalised basis vector of Eq. 3b.  The second form holds
// because the expansion is symmetric: psi(x) = sum_c kappa_c beta_c(x) sum_j
// m_j beta_c(x_j) for the raw basis beta_c of kernel 1, so the field of the
// coefficient vector A^J is exactly the required contraction.  Kernel 3 in
// dual numbers gives the first term (the derivative part of a(x + eps d)),
// kernel 1 in dual numbers with unit weights gives A^J (the derivative part of
// sum_i beta(x_i + eps d_i)), and kernel 2 and kernel 3 in their ordinary
// double form (mode ADJ_J) apply it.  The tidal term contributes T(R + x_k) d_k
// to xbar_k and, summed per block, the partials the centre-orbit adjoint needs.
#include "scf_device.cuh"
#include "scf_internal.h"

static __constant__ ScfConst c_tab;

cudaError_t scf_upload_const_adjoint(const ScfConst* t) { return cudaMemcpyToSymbol(c_tab, t, sizeof(ScfConst)); }

namespace {

constexpr int kK1DualTile = 64;
constexpr int kK3DualThreads = 128;

__device__ __forceinline__ Dual dual_pos(double x, double d) { return Dual(x, d); }

// Geometry of one particle in dual numbers: n_hat = (u, v, c), q = 1/(1+s),
// xi = 1 - 2q, sq2 = s q^2, and W_m = (u + i v)^m.
template <int LMAX>
struct DualGeom {
  Dual u, v, c, q, xi, sq2;
  Dual Wc[LMAX + 1], Ws[LMAX + 1];
  __device__ __forceinline__ DualGeom(Dual x, Dual y, Dual z, double binv) {
    const Dual r = sqrt(x * x + y * y + z * z);
    const Dual rinv = r.v > 0.0 ? Dual(1.0) / r : Dual(0.0);
    u = x * rinv;
    v = y * rinv;
    c = z * rinv;
    const Dual s = r * binv;
    q = Dual(1.0) / (Dual(1.0) + s);
    xi = Dual(1.0) - 2.0 * q;
    sq2 = s * q * q;
    Wc[0] = Dual(1.0);
    Ws[0] = Dual(0.0);
#pragma unroll
    for (int m = 1; m <= LMAX; ++m) {
      Wc[m] = Wc[m - 1] * u - Ws[m - 1] * v;
      Ws[m] = Wc[m - 1] * v + Ws[m - 1] * u;
    }
  }
};

// Legendre row l (without sin^m) from rows l-1 and l-2.
template <int LMAX>
__device__ __forceinline__ void dual_legendre_row(int l, Dual c, Dual* P, const Dual* P1, const Dual* P2) {
#pragma unroll
  for (int m = 0; m + 2 <= LMAX; ++m)
    if (m + 2 <= l) P[m] = c_tab.la[scf_lm(l, m)] * c * P1[m] - c_tab.lb[scf_lm(l, m)] * P2[m];
  if (l >= 1) P[l - 1] = c_tab.lsub[l] * c * P1[l - 1];
  P[l] = Dual(c_tab.ldiag[l]);
}

// ---------------------------------------------------------------------------
// Kernel 1 in dual numbers: per-block partials of
//   sum_k d/deps beta_nlm(x_k + eps d_k)   (unit weights).
// Same tile structure as kernel 1; the staged factors carry their value and
// derivative parts, and the contraction adds Rv Yd + Rd Yv.
// ---------------------------------------------------------------------------
template <int LMAX, int TP>
__global__ void __launch_bounds__(TP) k1_dual(K1Args a) {
  constexpr int YS = 2 * LMAX + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NN = a.nmax + 1;
  double* acc = reinterpret_cast<double*>(smem_raw);  // [2*NC]
  double* Rv = acc + 2 * a.nc;                         // [TP][NN]
  double* Rd = Rv + TP * NN;
  double* Yv = Rd + TP * NN;                           // [TP][YS]
  double* Yd = Yv + TP * YS;
  const int tid = threadIdx.x;
  for (int i = tid; i < 2 * a.nc; i += TP) acc[i] = 0.0;

  const int prog = a.blk_prog[blockIdx.x];
  const double binv = 1.0 / a.b_prog[prog];
  const int64_t k_begin = a.blk_begin[blockIdx.x], k_end = a.blk_end[blockIdx.x];
  const ScfD4* pos4 = reinterpret_cast<const ScfD4*>(a.pos);
  const ScfD4* vb4 = reinterpret_cast<const ScfD4*>(a.adj.vbar);

  for (int64_t base = k_begin; base < k_end; base += TP) {
    const int64_t k = base + tid;
    Dual x(0.0), y(0.0), z(0.0);
    if (k < k_end) {
      const ScfD4 p = pos4[k], vb = vb4[k];
      if (scf_finite3(p.x, p.y, p.z) && scf_finite3(vb.x, vb.y, vb.z)) {
        const double w = a.adj.weight;
        x = dual_pos(p.x, w * vb.x);
        y = dual_pos(p.y, w * vb.y);
        z = dual_pos(p.z, w * vb.z);
      } else {
        atomicOr(a.status, 1u);
      }
    }
    DualGeom<LMAX> g(x, y, z, binv);
    Dual P[LMAX + 1], P1[LMAX + 1], P2[LMAX + 1];
    Dual pre = g.q;  // s^l q^(2l+1) at l = 0
#pragma unroll
    for (int l = 0; l <= LMAX; ++l) {
      if (l > a.lmax) break;
      dual_legendre_row<LMAX>(l, g.c, P, P1, P2);
      {
        Dual cm1(0.0), c0(1.0);
        double* rv = Rv + tid * NN;
        double* rd = Rd + tid * NN;
        rv[0] = pre.v;
        rd[0] = pre.d;
        for (int n = 1; n < NN; ++n) {
          const Dual cn = c_tab.gA[l][n] * g.xi * c0 - c_tab.gB[l][n] * cm1;
          cm1 = c0;
          c0 = cn;
          const Dual f = pre * cn;
          rv[n] = f.v;
          rd[n] = f.d;
        }
      }
      {
        double* yv = Yv + tid * YS;
        double* yd = Yd + tid * YS;
#pragma unroll
        for (int m = 0; m <= l; ++m) {
          const Dual f = P[m] * g.Wc[m];
          yv[m] = f.v;
          yd[m] = f.d;
        }
#pragma unroll
        for (int m = 1; m <= l; ++m) {
          const Dual f = P[m] * g.Ws[m];
          yv[l + m] = f.v;
          yd[l + m] = f.d;
        }
      }
      __syncthreads();
      const int nout = NN * (2 * l + 1);
      for (int j = tid; j < nout; j += TP) {
        const int mm = j / NN, n = j - mm * NN;
        double sum = 0.0;
#pragma unroll 4
        for (int t = 0; t < TP; ++t)
          sum += Rv[t * NN + n] * Yd[t * YS + mm] + Rd[t * NN + n] * Yv[t * YS + mm];
        const int idx = (mm <= l) ? n * a.nlm + scf_lm(l, mm) : a.nc + n * a.nlm + scf_lm(l, mm - l);
        acc[idx] += sum;
      }
      __syncthreads();
      pre *= g.sq2;
#pragma unroll
      for (int m = 0; m <= l; ++m) {
        P2[m] = P1[m];
        P1[m] = P[m];
      }
    }
  }
  __syncthreads();
  double* out = a.partials + (size_t)blockIdx.x * 2 * a.nc;
  for (int i = tid; i < 2 * a.nc; i += TP) out[i] = acc[i];
}

// ---------------------------------------------------------------------------
// Kernel 3 in dual numbers: xbar_k += d/deps a(x_k + eps d_k) with the
// coefficients held fixed (the self-gravity Hessian term plus T(R + x_k) d_k),
// and the block's tidal partials.
// ---------------------------------------------------------------------------

// Directional derivative of the expansion's acceleration at (x, y, z) along
// the dual parts; F = [NC] (cosine, sine) force-coefficient pairs.
template <int LMAX>
__device__ __forceinline__ void dual_field(const double2* F, int lmax, int nmax, int nlm, double binv, Dual x, Dual y,
                                           Dual z, double& ax, double& ay, double& az) {
  DualGeom<LMAX> g(x, y, z, binv);
  Dual P[LMAX + 1], P1[LMAX + 1], P2[LMAX + 1];
  Dual An(0.0), Ax(0.0), Ay(0.0), Az(0.0);
  Dual slq = g.q;                // s^l q^(2l+1)
  Dual sl1q = g.q * g.q * g.q;   // s^(l-1) q^(2l+1), l >= 1
  const int NN = nmax + 1;
#pragma unroll
  for (int l = 0; l <= LMAX; ++l) {
    if (l > lmax) break;
    dual_legendre_row<LMAX>(l, g.c, P, P1, P2);
    Dual Z0c[LMAX + 1], Z0s[LMAX + 1], Z1c[LMAX + 1], Z1s[LMAX + 1];
    const int lm0 = scf_lm(l, 0);
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      const double2 f0 = F[lm0 + m];
      Z0c[m] = Dual(f0.x);
      Z0s[m] = Dual(f0.y);
      Z1c[m] = Dual(0.0);
      Z1s[m] = Dual(0.0);
    }
    {
      Dual cm1(0.0), c0(1.0), dm1(0.0), d0(1.0);
      for (int n = 1; n < NN; ++n) {
        const Dual cn = c_tab.gA[l][n] * g.xi * c0 - c_tab.gB[l][n] * cm1;
        const int o = n * nlm + lm0;
#pragma unroll
        for (int m = 0; m <= l; ++m) {
          const double2 fv = F[o + m];
          Z0c[m] += fv.x * cn;
          Z0s[m] += fv.y * cn;
          Z1c[m] += fv.x * d0;
          Z1s[m] += fv.y * d0;
        }
        const Dual dn = c_tab.hA[l][n] * g.xi * d0 - c_tab.hB[l][n] * dm1;
        cm1 = c0;
        c0 = cn;
        dm1 = d0;
        d0 = dn;
      }
    }
    const double al4 = 4.0 * (2.0 * l + 1.5);
    const Dual k1 = (l >= 1) ? binv * sl1q : Dual(0.0);
    const Dual k2a = binv * ((l >= 1 ? (double)l * sl1q : Dual(0.0)) - (double)(2 * l + 1) * slq * g.q);
    const Dual k2b = (binv * al4) * slq * g.q * g.q;
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      const Dual g1c = k1 * Z0c[m], g1s = k1 * Z0s[m];
      const Dual g2c = k2a * Z0c[m] + k2b * Z1c[m], g2s = k2a * Z0s[m] + k2b * Z1s[m];
      const Dual E = g1c * g.Wc[m] + g1s * g.Ws[m];
      const Dual D = g2c * g.Wc[m] + g2s * g.Ws[m];
      const Dual Pl = P[m];
      const Dual Pd = (m < l) ? -c_tab.lk[scf_lm(l, m)] * P[m + 1] : Dual(0.0);
      An += Pl * D - (g.c * Pd + (double)m * Pl) * E;
      Az += Pd * E;
      if (m >= 1) {
        Ax += (double)m * Pl * (g1c * g.Wc[m - 1] + g1s * g.Ws[m - 1]);
        Ay -= (double)m * Pl * (g1c * g.Ws[m - 1] - g1s * g.Wc[m - 1]);
      }
    }
    slq *= g.sq2;
    if (l >= 1) sl1q *= g.sq2;
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      P2[m] = P1[m];
      P1[m] = P[m];
    }
  }
  ax = -(An * g.u + Ax).d;
  ay = -(An * g.v + Ay).d;
  az = -(An * g.c + Az).d;
}

template <int LMAX>
__global__ void __launch_bounds__(kK3DualThreads) k3_dual(K3Args a) {
  constexpr int NW = kK3DualThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* F = reinterpret_cast<double2*>(smem_raw);
  __shared__ double s_R[3];
  __shared__ double s_red[NW][SCF_ADJ_Q];
  const int tid = threadIdx.x;
  const int prog = a.blk_prog[blockIdx.x];
  const double binv = 1.0 / a.b_prog[prog];
  {
    const double2* Fg = reinterpret_cast<const double2*>(a.F) + (size_t)prog * a.nc;
    for (int i = tid; i < a.nc; i += kK3DualThreads) F[i] = Fg[i];
  }
  const bool has_host = a.host.n > 0 && a.com != nullptr;
  if (tid < 3) s_R[tid] = has_host ? a.com[6 * prog + tid] : 0.0;
  __syncthreads();

  double acc[SCF_ADJ_Q];
#pragma unroll
  for (int i = 0; i < SCF_ADJ_Q; ++i) acc[i] = 0.0;
  const ScfD4* pos4 = reinterpret_cast<const ScfD4*>(a.pos);
  const ScfD4* vb4 = reinterpret_cast<const ScfD4*>(a.adj.vbar);
  ScfD4* xb4 = reinterpret_cast<ScfD4*>(a.adj.xbar);
  const int64_t k_end = a.blk_end[blockIdx.x];
  for (int64_t k = a.blk_begin[blockIdx.x] + tid; k < k_end; k += kK3DualThreads) {
    const ScfD4 p = pos4[k], vb = vb4[k];
    if (!(scf_finite3(p.x, p.y, p.z) && scf_finite3(vb.x, vb.y, vb.z))) {
      atomicOr(a.status, 1u);
      continue;
    }
    const double w = a.adj.weight;
    const double dx = w * vb.x, dy = w * vb.y, dz = w * vb.z;
    double gx, gy, gz;
    dual_field<LMAX>(F, a.lmax, a.nmax, a.nlm, binv, dual_pos(p.x, dx), dual_pos(p.y, dy), dual_pos(p.z, dz), gx,
                     gy, gz);
    if (has_host) {
      const double Px = s_R[0] + p.x, Py = s_R[1] + p.y, Pz = s_R[2] + p.z;
      Dual hx, hy, hz;
      scf_host_accel_t<Dual>(a.host, Dual(Px, dx), Dual(Py, dy), Dual(Pz, dz), hx, hy, hz);
      gx += hx.d;
      gy += hy.d;
      gz += hz.d;
      acc[0] += dx;
      acc[1] += dy;
      acc[2] += dz;
      acc[3] += hx.d;
      acc[4] += hy.d;
      acc[5] += hz.d;
#pragma unroll
      for (int c = 0; c < SCF_HOST_CAP; ++c) {
        if (c >= a.host.n) break;
        double ux, uy, uz;  // a_c / GM_c
        scf_host_comp_accel<double>(a.host.kind[c], 1.0, a.host.a[c], a.host.b[c], Px, Py, Pz, ux, uy, uz);
        Dual sx, sy, sz;    // derivative in the scale length a_c
        scf_host_comp_accel<Dual>(a.host.kind[c], Dual(a.host.GM[c]), Dual(a.host.a[c], 1.0), Dual(a.host.b[c]),
                                  Dual(Px), Dual(Py), Dual(Pz), sx, sy, sz);
        acc[6 + 2 * c] += dx * ux + dy * uy + dz * uz;
        acc[7 + 2 * c] += dx * sx.d + dy * sy.d + dz * sz.d;
      }
    }
    if (!(isfinite(gx) && isfinite(gy) && isfinite(gz))) atomicOr(a.status, 2u);
    ScfD4 X = xb4[k];
    X.x += gx;
    X.y += gy;
    X.z += gz;
    xb4[k] = X;
  }
  // block partials in a fixed order: shuffle tree in each warp, then warps in order
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int i = 0; i < SCF_ADJ_Q; ++i) {
    double v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp][i] = v;
  }
  __syncthreads();
  if (tid < SCF_ADJ_Q) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) v += s_red[w][tid];
    a.adj.part[(size_t)blockIdx.x * SCF_ADJ_Q + tid] = v;
  }
}

// ---------------------------------------------------------------------------
// Centre-orbit adjoint at one level, one warp per progenitor.  With S the
// progenitor's summed partials and u = w Vbar - sum d:
//   Rbar += sum T(P_k) d_k + T(R) u
//   GMbar_c += sum d_k . a_c(P_k)/GM_c + a_c(R)/GM_c . u
//   abar_c  += sum d_k . da_c(P_k)/da_c + da_c(R)/da_c . u
// (the -a_host(R) of the tidal term and the centre's own kicks at this
// level), then, unless this is the last level of the sweep, the drift is
// undone: Vbar += dt Rbar.
// ---------------------------------------------------------------------------
__global__ void k_com_adj(ComAdjArgs a) {
  const int p = blockIdx.x;
  const int lane = threadIdx.x;
  const int nq = 6 + 2 * a.host.n;
  double S[SCF_ADJ_Q];
#pragma unroll
  for (int i = 0; i < SCF_ADJ_Q; ++i) S[i] = 0.0;
  for (int b = lane; b < a.n_blocks; b += 32) {
    if (a.blk3_prog[b] != p) continue;
    const double* src = a.part + (size_t)b * SCF_ADJ_Q;
#pragma unroll
    for (int i = 0; i < SCF_ADJ_Q; ++i)
      if (i < nq) S[i] += src[i];
  }
#pragma unroll
  for (int i = 0; i < SCF_ADJ_Q; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) S[i] += __shfl_xor_sync(0xffffffffu, S[i], o);
  if (lane != 0) return;
  const double* R = a.com + 6 * p;
  double* cb = a.combar + 6 * p;
  const double ux = a.weight * cb[3] - S[0], uy = a.weight * cb[4] - S[1], uz = a.weight * cb[5] - S[2];
  Dual tx, ty, tz;
  scf_host_accel_t<Dual>(a.host, Dual(R[0], ux), Dual(R[1], uy), Dual(R[2], uz), tx, ty, tz);
  cb[0] += S[3] + tx.d;
  cb[1] += S[4] + ty.d;
  cb[2] += S[5] + tz.d;
  double* th = a.thetabar + (size_t)p * 2 * a.host.n;
  for (int c = 0; c < a.host.n; ++c) {
    double gx, gy, gz;
    scf_host_comp_accel<double>(a.host.kind[c], 1.0, a.host.a[c], a.host.b[c], R[0], R[1], R[2], gx, gy, gz);
    Dual sx, sy, sz;
    scf_host_comp_accel<Dual>(a.host.kind[c], Dual(a.host.GM[c]), Dual(a.host.a[c], 1.0), Dual(a.host.b[c]),
                              Dual(R[0]), Dual(R[1]), Dual(R[2]), sx, sy, sz);
    th[2 * c] += S[6 + 2 * c] + gx * ux + gy * uy + gz * uz;
    th[2 * c + 1] += S[7 + 2 * c] + sx.d * ux + sy.d * uy + sz.d * uz;
  }
  if (a.drift) {
    cb[3] += a.dt * cb[0];
    cb[4] += a.dt * cb[1];
    cb[5] += a.dt * cb[2];
  }
}

int lmax_bucket(int lmax) {
  if (lmax <= 4) return 4;
  if (lmax <= 8) return 8;
  return 12;
}

template <int LMAX>
struct AdjAt {
  static void* k1() { return (void*)k1_dual<LMAX, kK1DualTile>; }
  static void* k3() { return (void*)k3_dual<LMAX>; }
  static size_t k1_smem(int nmax, int nc) {
    return sizeof(double) * (2 * (size_t)nc + 2 * (size_t)kK1DualTile * ((nmax + 1) + (2 * LMAX + 1)));
  }
  static void launch1(const K1Args& a, int blocks, size_t smem, cudaStream_t s) {
    k1_dual<LMAX, kK1DualTile><<<blocks, kK1DualTile, smem, s>>>(a);
  }
  static void launch3(const K3Args& a, int blocks, size_t smem, cudaStream_t s) {
    k3_dual<LMAX><<<blocks, kK3DualThreads, smem, s>>>(a);
  }
};

template <typename Fn>
auto dispatch_adj(int lmax, Fn&& f) {
  switch (lmax_bucket(lmax)) {
    case 4: return f(AdjAt<4>());
    case 8: return f(AdjAt<8>());
    default: return f(AdjAt<12>());
  }
}

}  // namespace

cudaError_t scf_k1_dual_prepare(int lmax, int nmax, ScfLaunchInfo* info, int* blocks_per_sm) {
  const int nc = (nmax + 1) * (lmax + 1) * (lmax + 2) / 2;
  return dispatch_adj(lmax, [&](auto k) -> cudaError_t {
    using KK = decltype(k);
    info->threads = kK1DualTile;
    info->tile = kK1DualTile;
    info->variant = 0;
    info->smem = KK::k1_smem(nmax, nc);
    if (info->smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(KK::k1(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)info->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, KK::k1(), info->threads, info->smem);
  });
}

cudaError_t scf_k3_dual_prepare(int lmax, int nmax, ScfLaunchInfo* info, int* blocks_per_sm) {
  const int nc = (nmax + 1) * (lmax + 1) * (lmax + 2) / 2;
  return dispatch_adj(lmax, [&](auto k) -> cudaError_t {
    using KK = decltype(k);
    info->threads = kK3DualThreads;
    info->tile = kK3DualThreads;
    info->variant = 0;
    info->smem = sizeof(double2) * (size_t)nc;
    cudaError_t e = cudaFuncSetAttribute(KK::k3(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)info->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, KK::k3(), info->threads, info->smem);
  });
}

cudaError_t scf_k1_dual_launch(const K1Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s) {
  dispatch_adj(a.lmax, [&](auto k) -> int {
    decltype(k)::launch1(a, blocks, info.smem, s);
    return 0;
  });
  return cudaGetLastError();
}

cudaError_t scf_k3_dual_launch(const K3Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s) {
  dispatch_adj(a.lmax, [&](auto k) -> int {
    decltype(k)::launch3(a, blocks, info.smem, s);
    return 0;
  });
  return cudaGetLastError();
}

cudaError_t scf_com_adj_launch(const ComAdjArgs& a, cudaStream_t s) {
  k_com_adj<<<a.n_prog, 32, 0, s>>>(a);
  return cudaGetLastError();
}
