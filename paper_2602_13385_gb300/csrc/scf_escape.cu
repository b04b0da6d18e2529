// Escape physics of the cluster (Sec. 2.2; Sec. 3.1 footnote on r_t):
//
// * boundedness: particle i is bound when kin |v_i|^2 - sum_{j != i} G m_j / r_ij < 0
//   in the cluster frame, the sum an unsoftened direct summation over every
//   particle of its progenitor;
// * the energy-based Lagrange radius r_x: the k-th smallest cluster-frame radius
//   among the bound particles, k = ceil(frac n_bound); the coefficient set of
//   Eq. 3b is r <= r_x;
// * tidal scales at the centre R: T_ij = -d^2 psi_host/dx_i dx_j, its eigenvalues,
//   the tidal radius r_t = (G M_c / (l1 - (l2 + l3)/2))^(1/3) and the
//   integration timestep dt_int = sqrt(eta) (|T|_F^2 / 6)^(-1/4).
//
// Kernels:
//   k_bound_pairs  O(N^2) pair sums.  Grid (i-chunk, progenitor, j-segment):
//                  each block stages its j-segment through shared memory in
//                  tiles and keeps four (float) or two (double) i-particles
//                  per thread in registers.  Single precision sums blocks of
//                  64 pair terms in float and adds them in double; double
//                  precision evaluates the pair terms in float-float
//                  arithmetic (k_bound_pairs_ff) and adds blocks of 64 of
//                  them in double.  Each block writes one double per
//                  particle and segment.
//   k_bound_finish one thread per particle: adds the segments in order, forms
//                  E_i and the bound flag, and the radius key (bits of r^2).
//   k_select       one block per progenitor: bound count and mass, radix
//                  selection of the k-th smallest key (8 passes of 8 bits over
//                  shared-memory histograms of integer counts), the mask.
//   k_tidal        one thread per progenitor.
// Every sum has a fixed order, so results are bitwise reproducible.
#include <cmath>
#include <cstdint>
#include <math_constants.h>

#include "scf_device.cuh"

#include "scf_escape.h"

namespace {

constexpr int kPairThreads = 128;
constexpr int kPairSub = 64;      // pair terms summed in the element type before the double add
constexpr int kSelectThreads = 1024;

template <typename V4>
struct Elem;
template <>
struct Elem<float4> {
  using T = float;
  static constexpr int I = 4;     // i-particles per thread
};
template <>
struct Elem<ScfD4> {
  using T = double;
  static constexpr int I = 2;
};

// 1/sqrt(r2) of a single-precision pair by the hardware approximation
// (rsqrt.approx.ftz.f32, a few ulp); 0 for a pair that adds nothing: r2 zero,
// below the smallest normal float (which the approximation flushes to zero)
// or not finite.
__device__ __forceinline__ float pair_inv_r(float r2) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
  return r2 >= 1.17549435e-38f ? y : 0.f;  // r2 = inf gives y = 0
}
template <typename V4>
__global__ void __launch_bounds__(kPairThreads) k_bound_pairs(BoundArgs a) {
  using T = typename Elem<V4>::T;
  constexpr int kPairI = Elem<V4>::I;
  __shared__ V4 s_j[kPairThreads];
  const V4* pos = reinterpret_cast<const V4*>(a.pos);
  for (int p = blockIdx.y; p < a.n_prog; p += gridDim.y) {
    const int64_t o0 = a.prog_off[p], o1 = a.prog_off[p + 1];
    const int64_t ib = o0 + (int64_t)blockIdx.x * (kPairThreads * kPairI);
    if (ib >= o1) continue;  // the same for every thread of the block
    const int64_t seg = (o1 - o0 + a.split - 1) / a.split;
    const int64_t j0 = min(o1, o0 + (int64_t)blockIdx.z * seg), j1 = min(o1, j0 + seg);
    T xi[kPairI], yi[kPairI], zi[kPairI];
    double acc[kPairI];
#pragma unroll
    for (int q = 0; q < kPairI; ++q) {
      const int64_t i = ib + threadIdx.x + q * kPairThreads;
      const V4 pi = i < o1 ? pos[i] : V4{};
      xi[q] = pi.x;
      yi[q] = pi.y;
      zi[q] = pi.z;
      acc[q] = 0.0;
    }
    for (int64_t jb = j0; jb < j1; jb += kPairThreads) {
      const int cnt = (int)min((int64_t)kPairThreads, j1 - jb);
      __syncthreads();
      if ((int)threadIdx.x < cnt) s_j[threadIdx.x] = pos[jb + threadIdx.x];
      __syncthreads();
      for (int s = 0; s < cnt; s += kPairSub) {
        const int e = min(cnt, s + kPairSub);
        T part[kPairI];
#pragma unroll
        for (int q = 0; q < kPairI; ++q) part[q] = T(0);
#pragma unroll 4
        for (int jj = s; jj < e; ++jj) {
          const V4 pj = s_j[jj];
#pragma unroll
          for (int q = 0; q < kPairI; ++q) {
            const T dx = pj.x - xi[q], dy = pj.y - yi[q], dz = pj.z - zi[q];
            const T r2 = dx * dx + dy * dy + dz * dz;
            // the self pair (and any coincident pair, and non-finite r2) adds nothing
            const T ri = pair_inv_r(r2);
            part[q] += pj.w * ri;
          }
        }
#pragma unroll
        for (int q = 0; q < kPairI; ++q) acc[q] += (double)part[q];
      }
    }
#pragma unroll
    for (int q = 0; q < kPairI; ++q) {
      const int64_t i = ib + threadIdx.x + q * kPairThreads;
      if (i < o1) a.part[(size_t)blockIdx.z * (size_t)a.n_total + (size_t)i] = acc[q];
    }
  }
}

// Double-precision pair sums in float-float arithmetic ("double-single"):
// GB300 retires 64 single-precision FMAs for each double one, and a pair term
// carried as unevaluated sums of two floats (Dekker 1971; Knuth's TwoSum and
// the FMA-based exact product) costs about 80 single-precision operations
// against 11 double ones, so it runs several times faster at a relative error
// near 1e-13.  Positions and masses are split once into hi + lo floats when
// they are staged (48 of a double's 53 bits: a pair term's relative error
// grows like 2^-48 |x| / r_ij for pairs far closer together than their
// distance from the centre); separations are exact differences of the hi
// parts plus the difference of the lo parts; r^2 keeps each square's
// rounding error; 1/r is
// the hardware estimate refined by one Newton step whose residual 1 - r^2 y^2
// is formed in float-float; m / r is added to a float-float sum, folded into
// a double every 64 pairs.
struct FF {
  float h, l;
};

// The error-free transformations are written with the _rn intrinsics, which
// the compiler never contracts into FMAs (a contraction would break them).
__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ FF split_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(kPairThreads) k_bound_pairs_ff(BoundArgs a) {
  constexpr int kPairI = Elem<ScfD4>::I;
  __shared__ float4 s_hi[kPairThreads], s_lo[kPairThreads];
  const ScfD4* pos = reinterpret_cast<const ScfD4*>(a.pos);
  for (int p = blockIdx.y; p < a.n_prog; p += gridDim.y) {
    const int64_t o0 = a.prog_off[p], o1 = a.prog_off[p + 1];
    const int64_t ib = o0 + (int64_t)blockIdx.x * (kPairThreads * kPairI);
    if (ib >= o1) continue;  // the same for every thread of the block
    const int64_t seg = (o1 - o0 + a.split - 1) / a.split;
    const int64_t j0 = min(o1, o0 + (int64_t)blockIdx.z * seg), j1 = min(o1, j0 + seg);
    FF xi[kPairI], yi[kPairI], zi[kPairI];
    double acc[kPairI];
#pragma unroll
    for (int q = 0; q < kPairI; ++q) {
      const int64_t i = ib + threadIdx.x + q * kPairThreads;
      const ScfD4 pi = i < o1 ? pos[i] : ScfD4{};
      xi[q] = split_double(pi.x);
      yi[q] = split_double(pi.y);
      zi[q] = split_double(pi.z);
      acc[q] = 0.0;
    }
    for (int64_t jb = j0; jb < j1; jb += kPairThreads) {
      const int cnt = (int)min((int64_t)kPairThreads, j1 - jb);
      __syncthreads();
      if ((int)threadIdx.x < cnt) {
        const ScfD4 pj = pos[jb + threadIdx.x];
        const FF x = split_double(pj.x), y = split_double(pj.y), z = split_double(pj.z), m = split_double(pj.w);
        s_hi[threadIdx.x] = make_float4(x.h, y.h, z.h, m.h);
        s_lo[threadIdx.x] = make_float4(x.l, y.l, z.l, m.l);
      }
      __syncthreads();
      for (int s = 0; s < cnt; s += kPairSub) {
        const int e = min(cnt, s + kPairSub);
        FF sum[kPairI];
#pragma unroll
        for (int q = 0; q < kPairI; ++q) sum[q] = {0.f, 0.f};
#pragma unroll 2
        for (int jj = s; jj < e; ++jj) {
          const float4 hj = s_hi[jj], lj = s_lo[jj];
#pragma unroll
          for (int q = 0; q < kPairI; ++q) {
            // separation: exact difference of the hi parts + difference of the lo parts
            const FF dx = two_sum(hj.x, -xi[q].h), dy = two_sum(hj.y, -yi[q].h), dz = two_sum(hj.z, -zi[q].h);
            const float lx = __fadd_rn(dx.l, __fsub_rn(lj.x, xi[q].l));
            const float ly = __fadd_rn(dy.l, __fsub_rn(lj.y, yi[q].l));
            const float lz = __fadd_rn(dz.l, __fsub_rn(lj.z, zi[q].l));
            // r^2 = sum (h + l)^2 = sum h^2 + (2h + l) l, with the exact rounding
            // error of each h^2, renormalised (all of r^2 may sit in the l parts)
            const float px = __fmul_rn(dx.h, dx.h), py = __fmul_rn(dy.h, dy.h), pz = __fmul_rn(dz.h, dz.h);
            const float cx = fmaf(__fadd_rn(__fadd_rn(dx.h, dx.h), lx), lx, fmaf(dx.h, dx.h, -px));
            const float cy = fmaf(__fadd_rn(__fadd_rn(dy.h, dy.h), ly), ly, fmaf(dy.h, dy.h, -py));
            const float cz = fmaf(__fadd_rn(__fadd_rn(dz.h, dz.h), lz), lz, fmaf(dz.h, dz.h, -pz));
            const FF s1 = two_sum(px, py);
            const FF s2 = two_sum(s1.h, pz);
            const FF r2 = two_sum(s2.h, __fadd_rn(__fadd_rn(s1.l, s2.l), __fadd_rn(__fadd_rn(cx, cy), cz)));
            const float r2h = r2.h, r2l = r2.l;
            // 1/r: one Newton step y0 (1 + d/2), d = 1 - r^2 y0^2 in float-float
            const float y0 = rsqrt_approx(r2h);
            const float t = __fmul_rn(y0, y0), te = fmaf(y0, y0, -t);
            const float u = __fmul_rn(r2h, t);
            const float ue = fmaf(r2l, t, fmaf(r2h, te, fmaf(r2h, t, -u)));
            const float d = __fsub_rn(__fsub_rn(1.f, u), ue);
            const float corr = __fmul_rn(__fmul_rn(0.5f, y0), d);
            const float yh = __fadd_rn(y0, corr), yl = __fsub_rn(corr, __fsub_rn(yh, y0));
            // m / r into the float-float sum; pairs outside the normal range add nothing
            const bool ok = r2h >= 1.17549435e-38f && r2h <= 3.40282347e38f;
            const float ph = ok ? __fmul_rn(hj.w, yh) : 0.f;
            const float pe = ok ? fmaf(hj.w, yl, fmaf(lj.w, yh, fmaf(hj.w, yh, -ph))) : 0.f;
            const FF ns = two_sum(sum[q].h, ph);
            sum[q] = {ns.h, __fadd_rn(sum[q].l, __fadd_rn(ns.l, pe))};
          }
        }
#pragma unroll
        for (int q = 0; q < kPairI; ++q) acc[q] += (double)sum[q].h + (double)sum[q].l;
      }
    }
#pragma unroll
    for (int q = 0; q < kPairI; ++q) {
      const int64_t i = ib + threadIdx.x + q * kPairThreads;
      if (i < o1) a.part[(size_t)blockIdx.z * (size_t)a.n_total + (size_t)i] = acc[q];
    }
  }
}

template <typename V4>
__global__ void k_bound_finish(BoundArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_total) return;
  double pot = 0.0;
  for (int s = 0; s < a.split; ++s) pot += a.part[(size_t)s * (size_t)a.n_total + (size_t)i];
  const V4 v = reinterpret_cast<const V4*>(a.vel)[i];
  const V4 p = reinterpret_cast<const V4*>(a.pos)[i];
  const double vx = v.x, vy = v.y, vz = v.z;
  const double E = a.kin * (vx * vx + vy * vy + vz * vz) - a.G * pot;
  if (a.E_out) a.E_out[i] = E;
  a.bound[i] = E < 0.0 ? 1 : 0;
  // r^2 = (x x + y y) + z z without contraction, the same rounding as a plain
  // evaluation of that expression; for r^2 >= 0 its bits order like its value
  const double x = p.x, y = p.y, z = p.z;
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
  a.key[i] = (unsigned long long)__double_as_longlong(r2);
}

template <typename V4>
__global__ void __launch_bounds__(kSelectThreads) k_select(BoundArgs a) {
  constexpr int NW = kSelectThreads / 32;
  __shared__ unsigned s_hist[256];
  __shared__ double s_m[NW];
  __shared__ unsigned long long s_c[NW];
  __shared__ unsigned long long s_prefix, s_krem, s_nb;
  __shared__ double s_mb;
  const int p = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t o0 = a.prog_off[p], o1 = a.prog_off[p + 1];
  const V4* pos = reinterpret_cast<const V4*>(a.pos);
  const uint8_t* bound = a.bound;
  const unsigned long long* key = a.key;

  // bound count and bound mass (fixed order: thread strides, shuffle tree, warps in order)
  unsigned long long c = 0;
  double m = 0.0;
  for (int64_t k = o0 + tid; k < o1; k += kSelectThreads)
    if (bound[k]) {
      ++c;
      m += (double)pos[k].w;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    m += __shfl_xor_sync(0xffffffffu, m, o);
  }
  if (lane == 0) {
    s_c[warp] = c;
    s_m[warp] = m;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long nb = 0;
    double mb = 0.0;
    for (int w = 0; w < NW; ++w) {
      nb += s_c[w];
      mb += s_m[w];
    }
    unsigned long long k = 0;
    if (nb > 0) {
      const double kk = ceil(a.frac * (double)nb);
      k = kk < 1.0 ? 1ull : (unsigned long long)kk;
      if (k > nb) k = nb;
    }
    s_nb = nb;
    s_mb = mb;
    s_krem = k;
    s_prefix = 0ull;
  }
  __syncthreads();
  const unsigned long long nb = s_nb;

  // radix selection of the k-th smallest key among the bound particles
  if (nb > 0) {
    for (int pass = 0; pass < 8; ++pass) {
      const int shift = 56 - 8 * pass;
      const unsigned long long hi = pass == 0 ? 0ull : (~0ull << (shift + 8));
      for (int d = tid; d < 256; d += kSelectThreads) s_hist[d] = 0u;
      __syncthreads();
      const unsigned long long prefix = s_prefix;
      for (int64_t k = o0 + tid; k < o1; k += kSelectThreads) {
        if (!bound[k]) continue;
        const unsigned long long kk = key[k];
        if ((kk & hi) == prefix) atomicAdd(&s_hist[(kk >> shift) & 255ull], 1u);
      }
      __syncthreads();
      if (tid == 0) {
        const unsigned long long krem = s_krem;
        unsigned long long cum = 0;
        for (int d = 0; d < 256; ++d) {
          const unsigned long long hd = s_hist[d];
          if (cum + hd >= krem) {
            s_prefix = prefix | ((unsigned long long)d << shift);
            s_krem = krem - cum;
            break;
          }
          cum += hd;
        }
      }
      __syncthreads();
    }
  }
  // key of r_x^2 (0 = the bits of +0.0 when nothing is bound)
  const unsigned long long kx = nb > 0 ? s_prefix : 0ull;

  // the coefficient set r <= r_x, and its size
  unsigned long long cm = 0;
  for (int64_t k = o0 + tid; k < o1; k += kSelectThreads) {
    const bool in = key[k] <= kx;
    if (a.mask) a.mask[k] = in ? 1 : 0;
    cm += in ? 1ull : 0ull;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cm += __shfl_xor_sync(0xffffffffu, cm, o);
  __syncthreads();
  if (lane == 0) s_c[warp] = cm;
  __syncthreads();
  if (tid == 0) {
    unsigned long long n_in = 0;
    for (int w = 0; w < NW; ++w) n_in += s_c[w];
    double* st = a.stats + 4 * (size_t)p;
    st[0] = (double)nb;
    st[1] = s_mb;
    st[2] = sqrt(__longlong_as_double((long long)kx));
    st[3] = (double)n_in;
  }
}

// Eigenvalues l1 >= l2 >= l3 of a symmetric 3x3 matrix S (row-major) by the
// trigonometric solution of its characteristic cubic (Smith, Comm. ACM 4, 168,
// 1961): with q = tr S / 3 and p = sqrt(tr((S - qI)^2) / 6), the eigenvalues
// are q + 2p cos(phi + 2 pi j / 3), phi = acos(det((S - qI)/p) / 2) / 3.
__device__ void sym3_eigen(const double* S, double* lam) {
  const double p1 = S[1] * S[1] + S[2] * S[2] + S[5] * S[5];
  const double q = (S[0] + S[4] + S[8]) / 3.0;
  if (p1 == 0.0) {
    double d0 = S[0], d1 = S[4], d2 = S[8], t;
    if (d0 < d1) { t = d0; d0 = d1; d1 = t; }
    if (d1 < d2) { t = d1; d1 = d2; d2 = t; }
    if (d0 < d1) { t = d0; d0 = d1; d1 = t; }
    lam[0] = d0;
    lam[1] = d1;
    lam[2] = d2;
    return;
  }
  const double a0 = S[0] - q, a4 = S[4] - q, a8 = S[8] - q;
  const double p2 = a0 * a0 + a4 * a4 + a8 * a8 + 2.0 * p1;
  const double p = sqrt(p2 / 6.0);
  const double b0 = a0 / p, b4 = a4 / p, b8 = a8 / p, b1 = S[1] / p, b2 = S[2] / p, b5 = S[5] / p;
  const double det = b0 * (b4 * b8 - b5 * b5) - b1 * (b1 * b8 - b5 * b2) + b2 * (b1 * b5 - b4 * b2);
  double r = 0.5 * det;
  r = r < -1.0 ? -1.0 : (r > 1.0 ? 1.0 : r);
  const double phi = acos(r) / 3.0;
  const double two_pi_3 = 2.0943951023931954923;  // 2 pi / 3
  lam[0] = q + 2.0 * p * cos(phi);
  lam[2] = q + 2.0 * p * cos(phi + two_pi_3);
  lam[1] = 3.0 * q - lam[0] - lam[2];
}

__global__ void k_tidal(TidalArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n_prog) return;
  double R[3] = {0.0, 0.0, 0.0};
  if (a.com)
    for (int i = 0; i < 3; ++i) R[i] = a.com[6 * (size_t)p + i];
  double T[9];
  for (int j = 0; j < 3; ++j) {  // column j: derivative of a_host along x_j (dual numbers)
    Dual x(R[0], j == 0 ? 1.0 : 0.0), y(R[1], j == 1 ? 1.0 : 0.0), z(R[2], j == 2 ? 1.0 : 0.0);
    Dual ax, ay, az;
    scf_host_accel_t<Dual>(a.host, x, y, z, ax, ay, az);
    T[0 + j] = ax.d;
    T[3 + j] = ay.d;
    T[6 + j] = az.d;
  }
  double S[9], lam[3], fro2 = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      S[3 * i + j] = 0.5 * (T[3 * i + j] + T[3 * j + i]);
      fro2 += T[3 * i + j] * T[3 * i + j];
    }
  sym3_eigen(S, lam);
  const double fro = sqrt(fro2);
  const double l1e = lam[0] - 0.5 * (lam[1] + lam[2]);
  const double Mc = a.M_c ? a.M_c[(size_t)p * a.M_stride] : 0.0;
  double* o = a.out + 16 * (size_t)p;
  for (int i = 0; i < 9; ++i) o[i] = T[i];
  o[9] = lam[0];
  o[10] = lam[1];
  o[11] = lam[2];
  o[12] = fro;
  o[13] = l1e;
  o[14] = l1e > 0.0 ? cbrt(a.G * Mc / l1e) : CUDART_INF;
  o[15] = fro > 0.0 ? sqrt(a.eta) / sqrt(fro / sqrt(6.0)) : CUDART_INF;
}

}  // namespace

int scf_bound_split(int64_t i_chunks, int n_sm) {
  if (i_chunks <= 0) return 1;
  const int64_t s = (4 * (int64_t)n_sm + i_chunks - 1) / i_chunks;
  return (int)(s < 1 ? 1 : (s > kBoundMaxSplit ? kBoundMaxSplit : s));
}

int64_t scf_bound_chunk(int f32) { return kPairThreads * (f32 ? Elem<float4>::I : Elem<ScfD4>::I); }

cudaError_t scf_bound_launch(const BoundArgs& a, int64_t max_chunks, cudaStream_t s) {
  if (a.n_total > 0 && max_chunks > 0) {
    const dim3 grid((unsigned)max_chunks, (unsigned)(a.n_prog < 65535 ? a.n_prog : 65535), (unsigned)a.split);
    if (a.f32) k_bound_pairs<float4><<<grid, kPairThreads, 0, s>>>(a);
    else k_bound_pairs_ff<<<grid, kPairThreads, 0, s>>>(a);
    const unsigned fb = (unsigned)((a.n_total + 255) / 256);
    if (a.f32) k_bound_finish<float4><<<fb, 256, 0, s>>>(a);
    else k_bound_finish<ScfD4><<<fb, 256, 0, s>>>(a);
  }
  if (a.f32) k_select<float4><<<a.n_prog, kSelectThreads, 0, s>>>(a);
  else k_select<ScfD4><<<a.n_prog, kSelectThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t scf_select_launch(const BoundArgs& a, cudaStream_t s) {
  if (a.f32) k_select<float4><<<a.n_prog, kSelectThreads, 0, s>>>(a);
  else k_select<ScfD4><<<a.n_prog, kSelectThreads, 0, s>>>(a);
  return cudaGetLastError();
}

namespace {
// Complete refresh: b = r_50 / div, the scale of the lowest-order density of
// the radial family whose half-mass radius is the bound stars' energy-based
// one (stats from a selection at frac = 0.5); unchanged for a progenitor with
// nothing bound.
__global__ void k_retune_b(const double* stats, double* b_prog, int n_prog, double div) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_prog) return;
  const double* st = stats + 4 * (size_t)p;
  if (st[0] > 0.0 && st[2] > 0.0) b_prog[p] = st[2] / div;
}
}  // namespace

double scf_half_mass_divisor(double alpha) {
  // enclosed mass of the lowest-order density: (t/(1+t))^(alpha+1), t = (r/b)^(1/alpha)
  if (alpha == 1.0) return 1.0 + 1.4142135623730950488;  // Hernquist
  return std::pow(std::pow(2.0, 1.0 / (alpha + 1.0)) - 1.0, -alpha);
}

cudaError_t scf_retune_b_launch(const double* stats, double* b_prog, int n_prog, double alpha, cudaStream_t s) {
  k_retune_b<<<(n_prog + 127) / 128, 128, 0, s>>>(stats, b_prog, n_prog, scf_half_mass_divisor(alpha));
  return cudaGetLastError();
}

cudaError_t scf_tidal_launch(const TidalArgs& a, cudaStream_t s) {
  k_tidal<<<(a.n_prog + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}
