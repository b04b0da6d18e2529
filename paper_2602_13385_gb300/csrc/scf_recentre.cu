// Re-centring of the cluster frame (Sec. 2.1): the expansion centre is put
// where a_000 is largest, and the frame velocity is the mass-weighted mean
// velocity of the particles inside the core radius
//   r_core^2 = sum_i rho_i^2 r_i^2 / sum_i rho_i^2,
// rho_i the expansion's density at particle i.
//
// Centre.  a_000 of the particles' expansion about x_c (alpha, b fixed) is a
// positive multiple of F(x_c) = sum_k m_k g(s_k), g(s) = (1 + s^(1/alpha))^-alpha,
// s_k = |x_k - x_c| / b, so grad F = 0 reads sum_k m_k w_k (x_k - x_c) = 0 with
// w_k = t_k (1 + t_k)^(-alpha-1) / s_k^2, t = s^(1/alpha).  Each iteration
// (k_centre_blocks + k_centre_sum, launched max_iter times) moves x_c by
// sum m w (x_k - x_c) / sum m w; a progenitor whose step fell below tol * b
// stops (its later launches return at once).  Weights in the handle's
// precision, sums in double.
//
// Core.  The density of degree-l, order-n radial pair is
//   rho_nl = -Phi_nl K_nl s^(1/alpha - 2) q^2 / (4 pi b^2),   q = 1/(1 + t),
// K_nl = (n + a_l)(n + a_l + 1)/alpha^2, a_l = (2l+1) alpha, so the density at a
// particle is that per-particle factor times the potential of the coefficients
// K_nl A_nlm, which kernel 3 evaluates (acc.w).  Only ratios of rho^2 enter
// r_core, so the constant factor is dropped.  Particles at r = 0 (where a
// cusped density is infinite) are left out of both sums.
//
// Every sum is a per-block row (kernel-3 block map, fixed shuffle tree) added
// per progenitor in block order by one warp: deterministic.
#include <cmath>

#include "scf_device.cuh"
#include "scf_internal.h"

namespace {

constexpr int kRcThreads = 128;
constexpr int kRcWarps = kRcThreads / 32;

// Fixed-order block sum of NV values per thread into part[blockIdx.x][0..NV).
template <int NV>
__device__ __forceinline__ void block_row(double (&v)[NV], double* part) {
  __shared__ double s_w[kRcWarps][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_w[warp][i] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double x = 0.0;
#pragma unroll
    for (int w = 0; w < kRcWarps; ++w) x += s_w[w][threadIdx.x];
    part[(size_t)blockIdx.x * 4 + threadIdx.x] = x;
  }
}

// One warp: the rows of progenitor p's blocks in block order (lane-strided,
// then a fixed shuffle tree); every lane returns the totals.
template <int NV>
__device__ __forceinline__ void prog_sum(const RecentreArgs& a, int p, double (&v)[NV]) {
  const int lane = threadIdx.x;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  for (int b = lane; b < a.n_blocks; b += 32) {
    if (a.blk_prog[b] != p) continue;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += a.part[(size_t)b * 4 + i];
  }
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
}

// Mean-shift weight t (1+t)^(-alpha-1) / s^2 of a squared distance s2 = s^2.
template <typename T>
__device__ __forceinline__ T centre_weight(T s2, double alpha, double inv_alpha) {
  if (sizeof(T) == 4) s2 = fmax(s2, (T)1e-30f);  // the double floor (1e-300) underflows in float
  if (alpha == 1.0) {
    const T s = sqrt(s2), q = (T)1 / ((T)1 + s);
    return q * q / s;  // t = s: s / (1+s)^2 / s^2
  }
  const T s = sqrt(s2), t = pow(s, (T)inv_alpha);
  return t * pow((T)1 + t, (T)(-alpha - 1.0)) / s2;
}

template <typename V4, typename T>
__global__ void __launch_bounds__(kRcThreads) k_centre_blocks(RecentreArgs a) {
  const int p = a.blk_prog[blockIdx.x];
  const double* st = a.state + 16 * (size_t)p;
  if (st[4] != 0.0) return;  // converged (the sum kernel skips it too)
  const double xc = st[0], yc = st[1], zc = st[2];
  const double b = a.b_prog[p], ib2 = 1.0 / (b * b);
  const V4* pos = reinterpret_cast<const V4*>(a.pos);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t end = a.blk_end[blockIdx.x];
  for (int64_t k = a.blk_begin[blockIdx.x] + threadIdx.x; k < end; k += kRcThreads) {
    if (a.mask && !a.mask[k]) continue;
    const V4 q = pos[k];
    const double dx = (double)q.x - xc, dy = (double)q.y - yc, dz = (double)q.z - zc;
    const double s2 = fmax((dx * dx + dy * dy + dz * dz) * ib2, 1e-300);
    const double w = (double)q.w * (double)centre_weight<T>((T)s2, a.alpha, a.inv_alpha);
    v[0] += w * dx;
    v[1] += w * dy;
    v[2] += w * dz;
    v[3] += w;
  }
  block_row<4>(v, a.part);
}

__global__ void k_centre_sum(RecentreArgs a) {
  const int p = blockIdx.x;
  double* st = a.state + 16 * (size_t)p;
  if (st[4] != 0.0) return;
  double v[4];
  prog_sum<4>(a, p, v);
  if (threadIdx.x != 0) return;
  if (!(v[3] > 0.0) || !isfinite(v[3])) {  // empty set: stay
    st[4] = 1.0;
    return;
  }
  const double sx = v[0] / v[3], sy = v[1] / v[3], sz = v[2] / v[3];
  st[0] += sx;
  st[1] += sy;
  st[2] += sz;
  st[3] += 1.0;
  if (sqrt(sx * sx + sy * sy + sz * sz) <= a.tol * a.b_prog[p]) st[4] = 1.0;
}

// x_k -= x_c of the particle's progenitor (every particle, in the set or not).
template <typename V4>
__global__ void __launch_bounds__(kRcThreads) k_shift_pos(RecentreArgs a) {
  const int p = a.blk_prog[blockIdx.x];
  const double* st = a.state + 16 * (size_t)p;
  V4* pos = reinterpret_cast<V4*>(a.pos);
  const int64_t end = a.blk_end[blockIdx.x];
  for (int64_t k = a.blk_begin[blockIdx.x] + threadIdx.x; k < end; k += kRcThreads) {
    V4 q = pos[k];
    q.x = (decltype(q.x))((double)q.x - st[0]);
    q.y = (decltype(q.y))((double)q.y - st[1]);
    q.z = (decltype(q.z))((double)q.z - st[2]);
    pos[k] = q;
  }
}

// K_nl A_nlm into KA (the coefficients whose potential gives the density).
__global__ void k_scale_k(const double* A, double* KA, int nmax, int lmax, int n_prog, double alpha) {
  const int nlm = (lmax + 1) * (lmax + 2) / 2, nc = (nmax + 1) * nlm;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)2 * nc * n_prog) return;
  const int j = (int)(i % (2 * nc)), ii = j < nc ? j : j - nc;
  const int n = ii / nlm, lm = ii - n * nlm;
  int l = 0;
  while ((l + 1) * (l + 2) / 2 <= lm) ++l;
  const double al = (2.0 * l + 1.0) * alpha;
  KA[i] = (n + al) * (n + al + 1.0) / (alpha * alpha) * A[i];
}

template <typename V4>
__global__ void __launch_bounds__(kRcThreads) k_core_blocks1(RecentreArgs a) {
  const int p = a.blk_prog[blockIdx.x];
  const double ib = 1.0 / a.b_prog[p];
  const V4* pos = reinterpret_cast<const V4*>(a.pos);
  const V4* acc = reinterpret_cast<const V4*>(a.acc);
  double v[2] = {0.0, 0.0};
  const int64_t end = a.blk_end[blockIdx.x];
  for (int64_t k = a.blk_begin[blockIdx.x] + threadIdx.x; k < end; k += kRcThreads) {
    const V4 q = pos[k];
    const double r2 = ((double)q.x * q.x + (double)q.y * q.y) + (double)q.z * q.z;
    if (!(r2 > 0.0)) continue;
    const double s = sqrt(r2) * ib;
    const double t = a.alpha == 1.0 ? s : pow(s, a.inv_alpha);
    const double qq = 1.0 / (1.0 + t);
    const double fac = (a.alpha == 1.0 ? 1.0 / s : pow(s, a.inv_alpha - 2.0)) * qq * qq;
    const double rho = fac * (double)acc[k].w;  // density up to a constant factor
    v[0] += rho * rho * r2;
    v[1] += rho * rho;
  }
  double w4[4] = {v[0], v[1], 0.0, 0.0};
  block_row<4>(w4, a.part);
}

__global__ void k_core_sum1(RecentreArgs a) {
  const int p = blockIdx.x;
  double v[2];
  prog_sum<2>(a, p, v);
  if (threadIdx.x == 0) a.state[16 * (size_t)p + 5] = v[1] > 0.0 ? v[0] / v[1] : 0.0;  // r_core^2
}

template <typename V4>
__global__ void __launch_bounds__(kRcThreads) k_core_blocks2(RecentreArgs a) {
  const int p = a.blk_prog[blockIdx.x];
  const double rc2 = a.state[16 * (size_t)p + 5];
  const V4* pos = reinterpret_cast<const V4*>(a.pos);
  const V4* vel = reinterpret_cast<const V4*>(a.vel);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t end = a.blk_end[blockIdx.x];
  for (int64_t k = a.blk_begin[blockIdx.x] + threadIdx.x; k < end; k += kRcThreads) {
    const V4 q = pos[k];
    const double r2 = ((double)q.x * q.x + (double)q.y * q.y) + (double)q.z * q.z;
    if (!(r2 < rc2)) continue;
    const V4 u = vel[k];
    const double m = q.w;
    v[0] += m * u.x;
    v[1] += m * u.y;
    v[2] += m * u.z;
    v[3] += m;
  }
  block_row<4>(v, a.part);
}

__global__ void k_core_sum2(RecentreArgs a) {
  const int p = blockIdx.x;
  double v[4];
  prog_sum<4>(a, p, v);
  if (threadIdx.x != 0) return;
  double* st = a.state + 16 * (size_t)p;
  for (int i = 0; i < 3; ++i) st[6 + i] = v[3] > 0.0 ? v[i] / v[3] : 0.0;
  if (a.com) {
    double* c = a.com + 6 * (size_t)p;
    for (int i = 0; i < 3; ++i) {
      c[i] += st[i];
      c[3 + i] += st[6 + i];
    }
  }
}

template <typename V4>
__global__ void __launch_bounds__(kRcThreads) k_shift_vel(RecentreArgs a) {
  const int p = a.blk_prog[blockIdx.x];
  const double* st = a.state + 16 * (size_t)p;
  V4* vel = reinterpret_cast<V4*>(a.vel);
  const int64_t end = a.blk_end[blockIdx.x];
  for (int64_t k = a.blk_begin[blockIdx.x] + threadIdx.x; k < end; k += kRcThreads) {
    V4 u = vel[k];
    u.x = (decltype(u.x))((double)u.x - st[6]);
    u.y = (decltype(u.y))((double)u.y - st[7]);
    u.z = (decltype(u.z))((double)u.z - st[8]);
    vel[k] = u;
  }
}

}  // namespace

cudaError_t scf_centre_launch(const RecentreArgs& a, int max_iter, cudaStream_t s) {
  if (cudaMemsetAsync(a.state, 0, sizeof(double) * 16 * (size_t)a.n_prog, s) != cudaSuccess)
    return cudaGetLastError();
  for (int it = 0; it < max_iter; ++it) {
    if (a.n_blocks > 0) {
      if (a.f32) k_centre_blocks<float4, float><<<a.n_blocks, kRcThreads, 0, s>>>(a);
      else k_centre_blocks<ScfD4, double><<<a.n_blocks, kRcThreads, 0, s>>>(a);
    }
    k_centre_sum<<<a.n_prog, 32, 0, s>>>(a);
  }
  if (a.n_blocks > 0) {
    if (a.f32) k_shift_pos<float4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
    else k_shift_pos<ScfD4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t scf_scale_k_launch(const double* A, double* KA, int nmax, int lmax, int n_prog, double alpha,
                               cudaStream_t s) {
  const int64_t n = (int64_t)2 * (nmax + 1) * ((lmax + 1) * (lmax + 2) / 2) * n_prog;
  k_scale_k<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, KA, nmax, lmax, n_prog, alpha);
  return cudaGetLastError();
}

cudaError_t scf_core_launch(const RecentreArgs& a, cudaStream_t s) {
  if (a.n_blocks > 0) {
    if (a.f32) k_core_blocks1<float4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
    else k_core_blocks1<ScfD4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
  }
  k_core_sum1<<<a.n_prog, 32, 0, s>>>(a);
  if (a.n_blocks > 0) {
    if (a.f32) k_core_blocks2<float4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
    else k_core_blocks2<ScfD4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
  }
  k_core_sum2<<<a.n_prog, 32, 0, s>>>(a);
  if (a.n_blocks > 0) {
    if (a.f32) k_shift_vel<float4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
    else k_shift_vel<ScfD4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Basis scale at the maximum of a_000 (Sec. 2; alpha and the centre fixed).
// In the bi-orthonormal normalisation of Eq. 3a, a_000(b) is a constant times
// h(b) = b^(-1/2) sum_k m_k g(r_k / b) over the coefficient set.  Search in
// ln b: kScaleRounds grids of kScalePoints values, the first over
// [b/span, b span], each next over one step either side of the previous best
// (the first best in grid order); the last best moves to the vertex of the
// parabola through it and its neighbours.  From there kScaleNewton
// safeguarded Newton steps solve the stationarity condition
//   D(x) = d ln h / d ln b = S1/S0 - 1/2 = 0,   x = ln b,  t = (r/b)^(1/alpha),
//   S0 = sum m (1+t)^-alpha,  S1 = sum m t (1+t)^(-alpha-1),
//   D'(x) = S2/S0 - (S1/S0)^2,  S2 = sum m (-t/alpha) (1+t)^(-alpha-2) (1 - alpha t)
// inside the last grid's bracket (a step that leaves the bracket, or a
// non-negative D', bisects it instead; the sign of D shrinks it), so b is the
// maximiser to rounding, not to the grid's resolution.  An empty set keeps b.
// state[p]: during the grids [0] ln b of the grid's first point, [1] the step;
// during the Newton steps [0], [1] the bracket, [2] 1 = refine, [3] x.
namespace {

template <typename V4>
__global__ void __launch_bounds__(kRcThreads) k_scale_blocks(ScaleArgs a) {
  constexpr int NP = kScalePoints;
  __shared__ double s_ib[NP];
  __shared__ double s_w[kRcWarps][NP + 1];
  const int p = a.blk_prog[blockIdx.x];
  const double* st = a.state + 4 * (size_t)p;
  if (threadIdx.x < NP) s_ib[threadIdx.x] = exp(-(st[0] + threadIdx.x * st[1]));  // 1 / b_j
  __syncthreads();
  double v[NP + 1];
#pragma unroll
  for (int j = 0; j <= NP; ++j) v[j] = 0.0;
  const V4* pos = reinterpret_cast<const V4*>(a.pos);
  const int64_t end = a.blk_end[blockIdx.x];
  for (int64_t k = a.blk_begin[blockIdx.x] + threadIdx.x; k < end; k += kRcThreads) {
    if (a.mask && !a.mask[k]) continue;
    const V4 q = pos[k];
    const double r = sqrt(((double)q.x * q.x + (double)q.y * q.y) + (double)q.z * q.z);
    const double m = q.w;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const double s = r * s_ib[j];
      v[j] += m * (a.alpha == 1.0 ? 1.0 / (1.0 + s) : pow(1.0 + pow(s, a.inv_alpha), -a.alpha));
    }
    v[NP] += m;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j <= NP; ++j) {
    double x = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_w[warp][j] = x;
  }
  __syncthreads();
  if (threadIdx.x <= NP) {
    double x = 0.0;
#pragma unroll
    for (int w = 0; w < kRcWarps; ++w) x += s_w[w][threadIdx.x];
    a.part[(size_t)blockIdx.x * (NP + 1) + threadIdx.x] = x;
  }
}

__global__ void k_scale_init(ScaleArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n_prog) return;
  double* st = a.state + 4 * (size_t)p;
  st[0] = log(a.b_prog[p]) - log(a.span);
  st[1] = 2.0 * log(a.span) / (kScalePoints - 1);
  st[2] = 0.0;
}

// One warp per progenitor: the grid's sums in block order, the best point,
// the next grid (or, after the last round, the new b).
__global__ void k_scale_sum(ScaleArgs a, int round) {
  constexpr int NP = kScalePoints;
  const int p = blockIdx.x, lane = threadIdx.x;
  __shared__ double s_h[NP + 1];
  double v[NP + 1];
#pragma unroll
  for (int j = 0; j <= NP; ++j) v[j] = 0.0;
  for (int b = lane; b < a.n_blocks; b += 32) {
    if (a.blk_prog[b] != p) continue;
#pragma unroll
    for (int j = 0; j <= NP; ++j) v[j] += a.part[(size_t)b * (NP + 1) + j];
  }
#pragma unroll
  for (int j = 0; j <= NP; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  if (lane != 0) return;
  double* st = a.state + 4 * (size_t)p;
  if (!(v[NP] > 0.0)) return;  // empty set: b unchanged
  int best = 0;
  double hb = -1.0;
  for (int j = 0; j < NP; ++j) {
    s_h[j] = exp(-0.5 * (st[0] + j * st[1])) * v[j];
    if (s_h[j] > hb) {
      hb = s_h[j];
      best = j;
    }
  }
  if (round + 1 < kScaleRounds) {
    st[0] += (best - 1) * st[1];
    st[1] = 2.0 * st[1] / (NP - 1);
    return;
  }
  double x = st[0] + best * st[1];
  const double lo = st[0] + (best - 1) * st[1], hi = st[0] + (best + 1) * st[1];
  const bool inner = best > 0 && best < NP - 1;
  if (inner) {
    const double hm = s_h[best - 1], h0 = s_h[best], hp = s_h[best + 1];
    const double den = hm - 2.0 * h0 + hp;
    if (den < 0.0) x += 0.5 * st[1] * (hm - hp) / den;
  }
  st[0] = lo;
  st[1] = hi;
  st[2] = inner ? 1.0 : 0.0;
  st[3] = x;
  a.b_prog[p] = exp(x);
}

// Block sums (S0, S1, S2, mass) of the Newton step at each progenitor's x.
template <typename V4>
__global__ void __launch_bounds__(kRcThreads) k_scale_newton_blocks(ScaleArgs a) {
  __shared__ double s_w[kRcWarps][4];
  const int p = a.blk_prog[blockIdx.x];
  const double ib = exp(-a.state[4 * (size_t)p + 3]);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const V4* pos = reinterpret_cast<const V4*>(a.pos);
  const int64_t end = a.blk_end[blockIdx.x];
  for (int64_t k = a.blk_begin[blockIdx.x] + threadIdx.x; k < end; k += kRcThreads) {
    if (a.mask && !a.mask[k]) continue;
    const V4 q = pos[k];
    const double r = sqrt(((double)q.x * q.x + (double)q.y * q.y) + (double)q.z * q.z);
    const double m = q.w;
    const double t = a.alpha == 1.0 ? r * ib : pow(r * ib, a.inv_alpha);
    const double u = 1.0 / (1.0 + t);                                   // (1+t)^-1
    const double g = a.alpha == 1.0 ? u : pow(u, a.alpha);              // (1+t)^-alpha
    const double w = t * g * u;                                         // t (1+t)^(-alpha-1)
    v[0] += m * g;
    v[1] += m * w;
    v[2] += m * (-w * u * (1.0 - a.alpha * t) * a.inv_alpha);           // (-t/alpha)(1+t)^(-alpha-2)(1 - alpha t)
    v[3] += m;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    double x = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_w[warp][j] = x;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double x = 0.0;
#pragma unroll
    for (int w = 0; w < kRcWarps; ++w) x += s_w[w][threadIdx.x];
    a.part[(size_t)blockIdx.x * (kScalePoints + 1) + threadIdx.x] = x;
  }
}

// One warp per progenitor: the sums in block order, then one safeguarded
// Newton step of D(x) = 0 within the bracket; b = exp(x).
__global__ void k_scale_newton_step(ScaleArgs a) {
  const int p = blockIdx.x, lane = threadIdx.x;
  double* st = a.state + 4 * (size_t)p;
  if (st[2] != 1.0) return;  // maximum at an end of the range, or an empty set
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = lane; b < a.n_blocks; b += 32) {
    if (a.blk_prog[b] != p) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] += a.part[(size_t)b * (kScalePoints + 1) + j];
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  if (lane != 0 || !(v[3] > 0.0) || !(v[0] > 0.0)) return;
  const double x = st[3], f = v[1] / v[0];
  const double D = f - 0.5, dD = v[2] / v[0] - f * f;
  if (D > 0.0) st[0] = x;  // the maximum lies above x
  else if (D < 0.0) st[1] = x;
  else return;
  double xn = x - D / dD;
  if (!(dD < 0.0) || !(xn > st[0] && xn < st[1])) xn = 0.5 * (st[0] + st[1]);
  st[3] = xn;
  a.b_prog[p] = exp(xn);
}

// Block sums of the exponent search at (alpha, b_p): S0 = sum m g, S1 =
// sum m g d ln g / d alpha, with g = (1 + t)^-alpha, t = (r/b)^(1/alpha) and
// d ln g / d alpha = -ln(1 + t) + t ln(r/b) / (alpha (1 + t)); and the mass.
template <typename V4>
__global__ void __launch_bounds__(kRcThreads) k_alpha_blocks(ScaleArgs a) {
  __shared__ double s_w[kRcWarps][3];
  const int p = a.blk_prog[blockIdx.x];
  const double ib = 1.0 / a.b_prog[p];
  double v[3] = {0.0, 0.0, 0.0};
  const V4* pos = reinterpret_cast<const V4*>(a.pos);
  const int64_t end = a.blk_end[blockIdx.x];
  for (int64_t k = a.blk_begin[blockIdx.x] + threadIdx.x; k < end; k += kRcThreads) {
    if (a.mask && !a.mask[k]) continue;
    const V4 q = pos[k];
    const double r = sqrt(((double)q.x * q.x + (double)q.y * q.y) + (double)q.z * q.z);
    const double m = q.w;
    const double s = r * ib;
    const double t = pow(s, a.inv_alpha);
    const double g = pow(1.0 + t, -a.alpha);
    const double dlng = -log1p(t) + (s > 0.0 ? t * log(s) : 0.0) * a.inv_alpha / (1.0 + t);
    v[0] += m * g;
    v[1] += m * g * dlng;
    v[2] += m;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double x = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_w[warp][j] = x;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double x = 0.0;
#pragma unroll
    for (int w = 0; w < kRcWarps; ++w) x += s_w[w][threadIdx.x];
    a.part[(size_t)blockIdx.x * (kScalePoints + 1) + threadIdx.x] = x;
  }
}

// One warp per progenitor: the block sums in block order into out[p][0..2].
__global__ void k_alpha_sum(ScaleArgs a, double* out) {
  const int p = blockIdx.x, lane = threadIdx.x;
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = lane; b < a.n_blocks; b += 32) {
    if (a.blk_prog[b] != p) continue;
#pragma unroll
    for (int j = 0; j < 3; ++j) v[j] += a.part[(size_t)b * (kScalePoints + 1) + j];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  if (lane == 0)
    for (int j = 0; j < 3; ++j) out[3 * (size_t)p + j] = v[j];
}

}  // namespace

cudaError_t scf_alpha_sums_launch(const ScaleArgs& a, double* out, cudaStream_t s) {
  if (a.n_blocks > 0) {
    if (a.f32) k_alpha_blocks<float4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
    else k_alpha_blocks<ScfD4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
  }
  if (a.n_prog > 0) k_alpha_sum<<<a.n_prog, 32, 0, s>>>(a, out);
  return cudaGetLastError();
}

cudaError_t scf_scale_a000_launch(const ScaleArgs& a, cudaStream_t s) {
  k_scale_init<<<(a.n_prog + 127) / 128, 128, 0, s>>>(a);
  for (int r = 0; r < kScaleRounds; ++r) {
    if (a.n_blocks > 0) {
      if (a.f32) k_scale_blocks<float4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
      else k_scale_blocks<ScfD4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
    }
    k_scale_sum<<<a.n_prog, 32, 0, s>>>(a, r);
  }
  for (int it = 0; it < kScaleNewton; ++it) {
    if (a.n_blocks > 0) {
      if (a.f32) k_scale_newton_blocks<float4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
      else k_scale_newton_blocks<ScfD4><<<a.n_blocks, kRcThreads, 0, s>>>(a);
    }
    k_scale_newton_step<<<a.n_prog, 32, 0, s>>>(a);
  }
  return cudaGetLastError();
}
