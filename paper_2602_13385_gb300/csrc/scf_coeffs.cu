// Kernel 1 (coefficient partial sums, Eq. 3b) and kernel 2 (deterministic
// reduction, normalisation, centre-of-mass step).
//
// Kernel 1 works on tiles of TP particles, one thread per particle in the
// basis phase.  For each degree l the block stages, in shared memory, the
// radial factors R[t][n] = Ch_n(xi_t) (the scaled Gegenbauer values
// C_n / gscale[l][n], one multiply and one FMA a step) and the angular factors
// Y[t][mm] = m_t s^l q^(2l+1) Pb_lm C_m (mm = m) or ... Pb_lm S_m (mm = l + m);
// the constant gscale is applied when the block writes its sums.  Then every thread
// contracts a slice of the (n, mm) outputs over the tile's particles and adds
// it to the block's running sums.  The sums leave the block as one partial
// vector per block; kernel 2 adds the partials of each progenitor in block
// order, so the result does not depend on scheduling.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "scf_device.cuh"
#include "scf_internal.h"

static __constant__ ScfConst c_tab;

cudaError_t scf_upload_const_coeffs(const ScfConst* t) { return cudaMemcpyToSymbol(c_tab, t, sizeof(ScfConst)); }

namespace {

template <typename T> struct Vec4;
template <> struct Vec4<double> { using type = ScfD4; };
template <> struct Vec4<float> { using type = float4; };

template <typename T> __device__ __forceinline__ T tab_gbeta(int l, int n);
template <> __device__ __forceinline__ double tab_gbeta<double>(int l, int n) { return c_tab.gbeta[l][n]; }
template <> __device__ __forceinline__ float tab_gbeta<float>(int l, int n) { return c_tab.gbetaf[l][n]; }
template <typename T> __device__ __forceinline__ T tab_la(int i) { return sizeof(T) == 8 ? (T)c_tab.la[i] : (T)c_tab.laf[i]; }
template <typename T> __device__ __forceinline__ T tab_lb(int i) { return sizeof(T) == 8 ? (T)c_tab.lb[i] : (T)c_tab.lbf[i]; }
template <typename T> __device__ __forceinline__ T tab_lsub(int l) { return sizeof(T) == 8 ? (T)c_tab.lsub[l] : (T)c_tab.lsubf[l]; }
template <typename T> __device__ __forceinline__ T tab_ldiag(int l) { return sizeof(T) == 8 ? (T)c_tab.ldiag[l] : (T)c_tab.ldiagf[l]; }

// Block running sums: plain double in the FP64 kernel; in the mixed kernel a
// float pair (hi, lo) updated by an error-free two-sum, so each tile's float
// sum is added without FP64 arithmetic and without losing its low bits.
template <typename T> struct BlockAcc;
template <> struct BlockAcc<double> {
  using slot = double;
  __device__ static void zero(double* a, int i) { a[i] = 0.0; }
  __device__ static void add(double* a, int i, double v) { a[i] += v; }
  __device__ static double value(const double* a, int i) { return a[i]; }
};
template <> struct BlockAcc<float> {
  using slot = float2;
  __device__ static void zero(float2* a, int i) { a[i] = make_float2(0.f, 0.f); }
  __device__ static void add(float2* a, int i, float v) {
    float2 c = a[i];
    const float s = c.x + v;
    const float bp = s - c.x;
    const float err = (c.x - (s - bp)) + (v - bp);
    c.x = s;
    c.y += err;
    a[i] = c;
  }
  __device__ static double value(const float2* a, int i) { return (double)a[i].x + (double)a[i].y; }
};

// Radial family of exponent alpha != 1 (GEN): the recurrence steps and scales
// come from the handle's tables in device memory instead of the constant bank.
template <typename T, bool GEN>
__device__ __forceinline__ T k1_gbeta(const K1Args& a, int l, int n) {
  if constexpr (GEN) return sizeof(T) == 8 ? (T)__ldg(&a.tab->gbeta[l][n]) : (T)__ldg(&a.tab->gbetaf[l][n]);
  else return tab_gbeta<T>(l, n);
}

__device__ __forceinline__ double scf_pow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float scf_pow(float x, float y) { return powf(x, y); }

template <typename T, int LMAX, int TP, bool GEN = false>
__global__ void __launch_bounds__(TP) k1_partials(K1Args a) {
  constexpr int YS = 2 * LMAX + 1;
  using V4 = typename Vec4<T>::type;
  using Acc = BlockAcc<T>;
  using Slot = typename Acc::slot;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NN = a.nmax + 1;
  Slot* acc = reinterpret_cast<Slot*>(smem_raw);              // [2*NC] running block sums
  T* R = reinterpret_cast<T*>(acc + 2 * a.nc);                // [TP][NN]
  T* Y = R + TP * NN;                                         // [TP][YS]
  const int tid = threadIdx.x;

  for (int i = tid; i < 2 * a.nc; i += TP) Acc::zero(acc, i);

  const int prog = a.blk_prog[blockIdx.x];
  const T binv = (T)(1.0 / a.b_prog[prog]);
  const int64_t k_begin = a.blk_begin[blockIdx.x], k_end = a.blk_end[blockIdx.x];
  V4* pos4 = reinterpret_cast<V4*>(a.pos);

  for (int64_t base = k_begin; base < k_end; base += TP) {
    const int64_t k = base + tid;
    T x = 0, y = 0, z = 0, mass = 0;
    if (k < k_end) {
      V4 p = pos4[k];
      if (a.mode == SCF_MODE_STEP) {
        V4* vel4 = reinterpret_cast<V4*>(a.vel);
        const V4* acc4 = reinterpret_cast<const V4*>(a.acc);
        V4 v = vel4[k];
        const V4 g = acc4[k];
        const T h = (T)(0.5 * a.dt), dt = (T)a.dt;
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
        mass = (a.mask == nullptr || a.mask[k]) ? p.w : (T)0;
      } else {
        atomicOr(a.status, 1u);
      }
    }
    // geometry
    const T r = sqrt(x * x + y * y + z * z);
    const T rinv = r > (T)0 ? (T)1 / r : (T)0;
    const T u = x * rinv, v = y * rinv, c = z * rinv;
    const T s = r * binv;
    // alpha = 1: q = 1/(1+s), prefactor s^l q^(2l+1); alpha != 1: t = s^(1/alpha)
    // replaces s in q and xi, and q^alpha carries the prefactor s^l q^((2l+1) alpha)
    const T q = (T)1 / ((T)1 + (GEN ? scf_pow(s, (T)a.inv_alpha) : s));
    const T xi = (T)1 - (T)2 * q;
    const T qa = GEN ? scf_pow(q, (T)a.alpha) : q;
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
    T pre = mass * qa;  // m_k s^l q^((2l+1) alpha) at l = 0

#pragma unroll
    for (int l = 0; l <= LMAX; ++l) {
      if (l > a.lmax) break;
      // Legendre row l
#pragma unroll
      for (int m = 0; m + 2 <= l; ++m)
        P[m] = tab_la<T>(scf_lm(l, m)) * c * P1[m] - tab_lb<T>(scf_lm(l, m)) * P2[m];
      if (l >= 1) P[l - 1] = tab_lsub<T>(l) * c * P1[l - 1];
      P[l] = tab_ldiag<T>(l);
      // radial factors: scaled Gegenbauer values Ch_n = C_n / gscale[l][n]
      {
        T cm1 = 0, c0 = 1;
        T* Rt = R + tid * NN;
        Rt[0] = 1;
        for (int n = 1; n < NN; ++n) {
          const T cn = xi * c0 - k1_gbeta<T, GEN>(a, l, n) * cm1;
          cm1 = c0;
          c0 = cn;
          Rt[n] = cn;
        }
      }
      // angular factors, carrying the radial prefactor m_k s^l q^(2l+1)
      {
        T* Yt = Y + tid * YS;
#pragma unroll
        for (int m = 0; m <= l; ++m) Yt[m] = (pre * P[m]) * Wc[m];
#pragma unroll
        for (int m = 1; m <= l; ++m) Yt[l + m] = (pre * P[m]) * Ws[m];
      }
      __syncthreads();
      // contraction over the tile's particles
      const int nout = NN * (2 * l + 1);
      for (int j = tid; j < nout; j += TP) {
        const int mm = j / NN, n = j - mm * NN;
        T sum = 0;
#pragma unroll 8
        for (int t = 0; t < TP; ++t) sum += R[t * NN + n] * Y[t * YS + mm];
        const int idx = (mm <= l) ? n * a.nlm + scf_lm(l, mm) : a.nc + n * a.nlm + scf_lm(l, mm - l);
        Acc::add(acc, idx, sum);
      }
      __syncthreads();
      pre *= sq2;
#pragma unroll
      for (int m = 0; m <= l; ++m) {
        P2[m] = P1[m];
        P1[m] = P[m];
      }
    }
  }
  __syncthreads();
  double* out = a.partials + (size_t)blockIdx.x * 2 * a.nc;
  for (int i = tid; i < 2 * a.nc; i += TP) {
    const int ii = i < a.nc ? i : i - a.nc;
    const int n = ii / a.nlm, lm = ii - n * a.nlm;
    int l = 0;
    while ((l + 1) * (l + 2) / 2 <= lm) ++l;
    const double gs = GEN ? a.tab->gscale[l][n] : c_tab.gscale[l][n];
    out[i] = Acc::value(acc, i) * gs;  // undo the scaling of the staged C_n
  }
}

template <typename T, int LMAX, int TP>
size_t k1_smem(int nmax, int nc) {
  using Slot = typename BlockAcc<T>::slot;
  return sizeof(Slot) * 2 * (size_t)nc + sizeof(T) * (size_t)TP * ((nmax + 1) + (2 * LMAX + 1));
}

// ---------------------------------------------------------------------------
// Kernel 1, register-tiled single-precision form.
//
// Per degree l the coefficient pass is the contraction
//   S_hat[n][mm] = sum_p R[p][l][n] Y[p][l][mm]
// over particles p, with only (nmax+1)(2l+1) outputs.  Reading both operands
// from shared memory for every FMA (the form above) ties it to shared-memory
// bandwidth: one wavefront per operand against four FMA instructions per
// clock.  Here every worker thread owns one TN x TM tile of outputs (degree l,
// TN radial orders, TM angular columns) for the block's lifetime, and one of
// `sub` particle sub-groups; per group of four particles it reads TN + TM
// float4 rows and issues 4 TN TM FMAs into registers.  The tile shape follows
// the expansion: all 21 radial orders by 3 columns at nmax = 20 (the 2l + 1
// columns of a degree then pad to a multiple of 3, not of 8: 132 instead of
// 168 columns at lmax = 10), 11 by 5 at nmax = 10, 7 by 8 otherwise.  At
// nmax = 20 the radial rows are staged as interleaved pairs of orders and the
// contraction issues packed FMAs (fma.rn.f32x2), each updating the sums of
// two radial orders with every lane rounding as fmaf, the particles in the
// same order (the odd last order in scalar FMAs): half the FMA instructions.
//
// The basis of each 60-particle tile is staged as rows [l][n] (the scaled
// Gegenbauer values Ch_n(xi) = C_n(xi) / gscale[l][n], see ScfConst) and
// [chunk (l, mm / TM)][mm % TM] (angular factors m s^l q^(2l+1) Pb_lm C_m and
// ... Pb_lm S_m), particle index fastest; the constant gscale is applied when
// the sums are flushed.  Eight warps compute it, four threads
// per particle: thread set q runs the Gegenbauer chains of the degrees
// l = q, q+4, q+8, ... and the Legendre columns of the orders m = q, q+4, ...
// interleaved, so its recurrence constants are warp-uniform and its chains
// independent.  Two blocks share an SM, so one block's basis phase overlaps
// the other's contraction.
//
// Every WINDOW_TILES tiles, and at the end, a worker stores its register sums
// (at most 64 x 16 single-precision terms each) into its own slot for
// that window and starts again from zero, so no sum grows long in single
// precision and nothing is read back; kernel 2 adds the slots of all windows,
// sub-groups and blocks in double precision in a fixed order.  Rows and
// columns of a tile beyond nmax or 2l read padding or the next degree's rows
// and are never written out.
// ---------------------------------------------------------------------------
namespace tiled {
constexpr int TP = 60;           // particles per tile (two basis halves of 30 lanes)
constexpr int TPP = TP;          // staged row stride in floats: 15 float4s, an odd number, so
                                 // float4 reads of rows that differ mod 8 hit different bank groups
constexpr int BASIS_WARPS = 8;   // 2 particle halves x 4 chain sets
constexpr int WINDOW_TILES = 64; // tiles summed in registers before a window's sums are stored
constexpr int MAX_THREADS = 256;

// Output tile of a worker: TN radial orders x TM angular columns.
// PAIRS (tiles that span all radial orders of a degree): the radial rows of a
// degree are staged as interleaved pairs, pair row p holding (R_2p[t],
// R_2p+1[t]) for every particle t, so that one float4 load gives the operands
// of two packed FMAs (fma.rn.f32x2), each updating the accumulators of two
// radial orders; a degree's block of pair rows is padded by one float4 so that
// it spans an odd number of float4s and lanes reading different degrees start
// in different bank groups.
template <int TN_, int TM_, bool PAIRS_ = false>
struct Tile {
  static constexpr int TN = TN_, TM = TM_;
  static constexpr bool kPairs = PAIRS_;
  static constexpr int TNP = (TN + 1) / 2;               // pair rows of a degree
  static constexpr int kDegFloats = TNP * 2 * TPP + 4;   // staged floats of a degree (PAIRS)
  static_assert(TN * TM <= 64, "the register budget holds at most 64 accumulators");
  static_assert(!kPairs || (kDegFloats / 4) % 2 == 1, "a degree's pair rows span an odd number of float4s");
  static __host__ __device__ constexpr int n_chunks(int nn) { return (nn + TN - 1) / TN; }
  static __host__ __device__ constexpr int m_chunks(int l) { return (2 * l + 1 + TM - 1) / TM; }
  // zero rows after the last degree's radial rows that its last chunk reads
  static __host__ __device__ constexpr int pad_rows(int nn) { return n_chunks(nn) * TN - nn; }
  static int n_items(int nmax, int lmax) {
    int c = 0;
    for (int l = 0; l <= lmax; ++l) c += m_chunks(l);
    return c * n_chunks(nmax + 1);
  }
  // Angular rows are stored by output chunk: chunk k = (l, mm / TM) occupies
  // the TM rows from YCH k, YCH the smallest odd count >= TM, so that the
  // chunks that the lanes of a warp read together (15 YCH float4s apart, an
  // odd number) start in different bank groups.
  static constexpr int YCH = TM | 1;
  static __host__ __device__ constexpr int chunk_base(int l) {  // chunks of the degrees below l
    int k = 0;
    for (int i = 0; i < l; ++i) k += m_chunks(i);
    return k;
  }
  static __host__ __device__ constexpr int y_row(int l, int mm) { return YCH * (chunk_base(l) + mm / TM) + mm % TM; }
  // Shared memory: [gen: the Gegenbauer steps gbeta[l][n] of the handle's
  // radial family] then the staging rows; at window ends the staging rows hold
  // the worker tiles (at most MAX_THREADS tiles of TN x TM floats) for the
  // cross-sub-group sums.
  static constexpr size_t kRedFloats = (size_t)MAX_THREADS * TN * TM;
  static size_t r_floats(int nmax, int lmax) {  // the staged radial rows
    return kPairs ? (size_t)(lmax + 1) * kDegFloats
                  : (size_t)TPP * ((size_t)(lmax + 1) * (nmax + 1) + pad_rows(nmax + 1));
  }
  static size_t smem_bytes(int nmax, int lmax, bool gen) {
    const size_t staged = r_floats(nmax, lmax) + (size_t)TPP * YCH * chunk_base(lmax + 1);
    const size_t sg = gen ? (size_t)(lmax + 1) * (nmax + 1) : 0;
    return sizeof(float) * (((sg + 3) & ~size_t(3)) + std::max(staged, kRedFloats));
  }
};
using TileGeneric = Tile<7, 8>;
// the tile of a compile-time shape: all radial orders where they fit
template <int NN>
// (paired radial rows at nmax = 20: 1-3% faster at alpha = 1 and 13% for the
// general family; at nmax = 10 the 11 x 5 tiles measured 3.6% slower paired)
using TileFor =
    std::conditional_t<NN == 21, Tile<21, 3, true>, std::conditional_t<NN == 11, Tile<11, 5>, TileGeneric>>;

// At the end of a window: every worker has written its tile to red[(sgrp *
// items + item) * TN * TM + i * TM + j]; the block adds the sub-groups' tiles
// in sub-group order and writes the window's row (times the constant gscale of
// the staged C_n) to dst: one float row of 2 NC per window and block, T_nl0
// not written (kernel 2 reads it as 0).  tab: the tables of a radial family
// with alpha != 1 (null: the constant bank's).
template <class S>
__device__ __forceinline__ void store_window(const float* __restrict__ red, float* __restrict__ dst, int items, int sub,
                                             const short (*item_lnm)[3], int nn, int nlm, int nc,
                                             const ScfConst* tab) {
  constexpr int TM = S::TM, E = S::TN * S::TM;
  for (int e = threadIdx.x; e < items * E; e += blockDim.x) {
    const int it = e / E, r = e - it * E, i = r / TM, j = r - i * TM;
    const int l = item_lnm[it][0], n = item_lnm[it][1] + i, mm = item_lnm[it][2] + j;
    if (n < nn && mm <= 2 * l) {
      float v = 0.f;
      for (int sg = 0; sg < sub; ++sg) v += red[(size_t)(sg * items + it) * E + r];
      const float gs = tab ? __ldg(&tab->gscalef[l][n]) : c_tab.gscalef[l][n];
      const int col = mm <= l ? scf_lm(l, mm) : nc + scf_lm(l, mm - l);
      dst[n * nlm + col] = v * gs;
    }
  }
}

// Basis of one particle for thread set q (runtime degrees and orders): the
// chains l = q + 4j (radial rows) and m = q + 4j (Legendre columns, angular rows).
// GEN: a radial family with alpha != 1, its Gegenbauer steps from sg (shared
// memory, [l][n] rows of NN); qv is then q^alpha and sq2 = s q^(2 alpha) (the
// factors of the prefactor).
template <int NCH, bool GEN = false>
struct BasisGeneric {
  static constexpr bool kGen = GEN;
  using S = TileGeneric;
  static __device__ __forceinline__ void run(int q, float* Rs, float* Ys, int t, int NN, int L, float mass, float u,
                                             float v, float c, float qv, float xi, float sq2, const float* sg) {
      // radial chains of the degrees l = q + 4j: R[l][n] = Ch_n(xi)
    {
      float c0[NCH], cm1[NCH];
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        c0[j] = 1.f;
        cm1[j] = 0.f;
        const int l = q + 4 * j;
        if (l <= L) Rs[(l * NN) * TPP + t] = 1.f;
      }
      for (int n = 1; n < NN; ++n) {
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
          const int l = q + 4 * j;
          if (l <= L) {
            const float gb = GEN ? sg[l * NN + n] : c_tab.gbetaf[l][n];
            const float cn = fmaf(-gb, cm1[j], xi * c0[j]);
            cm1[j] = c0[j];
            c0[j] = cn;
            Rs[(l * NN + n) * TPP + t] = cn;
          }
        }
      }
    }
    // Legendre columns of the orders m = q + 4j, times W_m = (u + i v)^m and
    // the radial prefactor m s^l q^(2l+1)
    {
      float wc = 1.f, ws = 0.f, pw = mass * qv;
      for (int i = 0; i < q; ++i) {
        const float tc = wc * u - ws * v;
        ws = wc * v + ws * u;
        wc = tc;
        pw *= sq2;
      }
      const float w2c = u * u - v * v, w2s = 2.f * u * v;
      const float w4c = w2c * w2c - w2s * w2s, w4s = 2.f * w2c * w2s;
      const float s2 = sq2 * sq2, s4 = s2 * s2;
      float Wc[NCH], Ws[NCH], P1[NCH], P2[NCH], pre[NCH];
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        Wc[j] = wc;
        Ws[j] = ws;
        pre[j] = pw;   // m s^m q^(2m+1) at l = m
        const float tc = wc * w4c - ws * w4s;
        ws = wc * w4s + ws * w4c;
        wc = tc;
        pw *= s4;
        P1[j] = 0.f;
        P2[j] = 0.f;
      }
      for (int l = q; l <= L; ++l) {
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
          const int m = q + 4 * j;
          if (m <= l) {
            float P;
            if (l == m) P = c_tab.ldiagf[l];
            else if (l == m + 1) P = c_tab.lsubf[l] * c * P1[j];
            else P = c_tab.laf[scf_lm(l, m)] * c * P1[j] - c_tab.lbf[scf_lm(l, m)] * P2[j];
            P2[j] = P1[j];
            P1[j] = P;
            const float Pp = P * pre[j];
            pre[j] *= sq2;
            Ys[S::y_row(l, m) * TPP + t] = Pp * Wc[j];
            if (m >= 1) Ys[S::y_row(l, l + m) * TPP + t] = Pp * Ws[j];
          }
        }
      }
    }
  }
};

// The same with the shape fixed at compile time: every recurrence constant is
// an immediate constant-bank operand and every staged row an immediate offset.
template <int Q, int NN, int L, bool GEN, class S>
__device__ __forceinline__ void basis_fixed(float* Rs, float* Ys, int t, float mass, float u, float v, float c,
                                            float qv, float xi, float sq2, const float* sg) {
  constexpr int NJ = Q <= L ? (L - Q) / 4 + 1 : 0;
  static_assert(!S::kPairs || S::TN == NN, "paired radial rows: the tile spans all radial orders");
  if constexpr (NJ > 0) {
    // radial rows Ch_n(xi) of the degrees l = Q + 4j (PAIRS: stored as the
    // pairs (Ch_n-1, Ch_n) at odd n, and (Ch_NN-1, 0) after the last odd n)
    float c0[NJ], cm1[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      c0[j] = 1.f;
      cm1[j] = 0.f;
      if constexpr (!S::kPairs) Rs[((Q + 4 * j) * NN) * TPP + t] = 1.f;
    }
#pragma unroll
    for (int n = 1; n < NN; ++n) {
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int l = Q + 4 * j;
        const float gb = GEN ? sg[l * NN + n] : c_tab.gbetaf[l][n];  // GEN: an immediate shared offset
        const float cn = fmaf(-gb, cm1[j], xi * c0[j]);
        cm1[j] = c0[j];
        c0[j] = cn;
        if constexpr (S::kPairs) {
          if (n & 1)
            *reinterpret_cast<float2*>(Rs + l * S::kDegFloats + (n >> 1) * 2 * TPP + 2 * t) = make_float2(cm1[j], cn);
        } else {
          Rs[(l * NN + n) * TPP + t] = cn;
        }
      }
    }
    if constexpr (S::kPairs && NN % 2 == 1) {
#pragma unroll
      for (int j = 0; j < NJ; ++j)
        *reinterpret_cast<float2*>(Rs + (Q + 4 * j) * S::kDegFloats + (NN >> 1) * 2 * TPP + 2 * t) =
            make_float2(c0[j], 0.f);
    }
    // angular rows m s^l q^(2l+1) Pb_lm {C_m, S_m} of the orders m = Q + 4j
    float wc = 1.f, ws = 0.f, pw = mass * qv;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float tc = wc * u - ws * v;
      ws = wc * v + ws * u;
      wc = tc;
      pw *= sq2;
    }
    const float w2c = u * u - v * v, w2s = 2.f * u * v;
    const float w4c = w2c * w2c - w2s * w2s, w4s = 2.f * w2c * w2s;
    const float s2 = sq2 * sq2, s4 = s2 * s2;
    float Wc[NJ], Ws[NJ], P1[NJ], P2[NJ], pre[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      Wc[j] = wc;
      Ws[j] = ws;
      pre[j] = pw;
      const float tc = wc * w4c - ws * w4s;
      ws = wc * w4s + ws * w4c;
      wc = tc;
      pw *= s4;
      P1[j] = 0.f;
      P2[j] = 0.f;
    }
#pragma unroll
    for (int l = Q; l <= L; ++l) {
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int m = Q + 4 * j;
        if (m <= l) {
          float P;
          if (l == m) P = c_tab.ldiagf[l];
          else if (l == m + 1) P = c_tab.lsubf[l] * c * P1[j];
          else P = c_tab.laf[scf_lm(l, m)] * c * P1[j] - c_tab.lbf[scf_lm(l, m)] * P2[j];
          P2[j] = P1[j];
          P1[j] = P;
          const float Pp = P * pre[j];
          pre[j] *= sq2;
          Ys[S::y_row(l, m) * TPP + t] = Pp * Wc[j];
          if (m >= 1) Ys[S::y_row(l, l + m) * TPP + t] = Pp * Ws[j];
        }
      }
    }
  }
}

template <int NN_, int L_, bool GEN = false>
struct BasisFixed {
  static constexpr bool kGen = GEN;
  using S = TileFor<NN_>;
  static __device__ __forceinline__ void run(int q, float* Rs, float* Ys, int t, int, int, float mass, float u,
                                             float v, float c, float qv, float xi, float sq2, const float* sg) {
    switch (q) {  // warp-uniform
      case 0: basis_fixed<0, NN_, L_, GEN, S>(Rs, Ys, t, mass, u, v, c, qv, xi, sq2, sg); break;
      case 1: basis_fixed<1, NN_, L_, GEN, S>(Rs, Ys, t, mass, u, v, c, qv, xi, sq2, sg); break;
      case 2: basis_fixed<2, NN_, L_, GEN, S>(Rs, Ys, t, mass, u, v, c, qv, xi, sq2, sg); break;
      default: basis_fixed<3, NN_, L_, GEN, S>(Rs, Ys, t, mass, u, v, c, qv, xi, sq2, sg); break;
    }
  }
};

// 128 registers: each quarter of the SM holds 16384, i.e. four warps of 128
// registers, so two blocks of 8 warps share an SM; the (at most 64)
// accumulators and the operands of the shorter tile side fit without spilling.
template <class B>  // basis policy: BasisGeneric<NCH> or BasisFixed<NN, L>
__global__ void __maxnreg__(128) k1_tiled(K1Args a) {
  using S = typename B::S;
  constexpr int TN = S::TN, TM = S::TM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ short item_lnm[MAX_THREADS][3];       // (l, n0, mm0) of every output tile
  const int NN = a.nmax + 1, L = a.lmax;
  const int rR = (L + 1) * NN, pad = S::pad_rows(NN);
  const int sg_floats = B::kGen ? ((rR + 3) & ~3) : 0;
  float* SG = reinterpret_cast<float*>(smem_raw);  // [L + 1][NN] Gegenbauer steps (radial family alpha != 1)
  float* Rs = SG + sg_floats;                      // [rR + pad][TPP]; PAIRS: [L + 1][kDegFloats]
  float* Ys = Rs + (S::kPairs ? (L + 1) * S::kDegFloats : (rR + pad) * TPP);  // [YCH * chunks][TPP]
  float* red = Rs;                                 // window ends: the worker tiles
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // padding rows and the angular rows past 2l of each degree's last chunk are
  // never written by the basis; they feed only accumulators that are never
  // stored, and are cleared once so that they hold no stale values
  {
    const int ny4 = S::YCH * S::chunk_base(L + 1) * (TPP / 4);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = tid; i < pad * (TPP / 4); i += blockDim.x) reinterpret_cast<float4*>(Rs + rR * TPP)[i] = z4;
    for (int i = tid; i < ny4; i += blockDim.x) reinterpret_cast<float4*>(Ys)[i] = z4;
  }
  if constexpr (B::kGen)
    for (int i = tid; i < rR; i += blockDim.x) SG[i] = a.tab->gbetaf[i / NN][i % NN];

  // contraction role: item (l, c, d) = output tile, sgrp = particle sub-group
  const bool worker = tid < a.items * a.sub;
  const int item = tid % a.items, sgrp = tid / a.items;
  int il = 0, ic = 0, id = 0;
  {
    const int ncn = S::n_chunks(NN);
    int r = item;
    for (int l = 0; l <= L; ++l) {
      const int cnt = S::m_chunks(l) * ncn;
      if (r < cnt) {
        il = l;
        id = r / ncn;
        ic = r - id * ncn;
        break;
      }
      r -= cnt;
    }
  }
  const int n0 = ic * TN, mm0 = id * TM;
  if (worker && sgrp == 0) {
    item_lnm[item][0] = (short)il;
    item_lnm[item][1] = (short)n0;
    item_lnm[item][2] = (short)mm0;
  }
  __syncthreads();
  const float* Rrow = S::kPairs ? Rs + il * S::kDegFloats : Rs + (il * NN + n0) * TPP;
  const float* Yrow = Ys + S::y_row(il, mm0) * TPP;
  // PAIRS: the radial orders (2p, 2p + 1) x TM in packed pairs, an odd last
  // order (its staged pair is (Ch_TN-1, 0)) in scalars
  constexpr int TN2 = TN / 2;
  float acc[TN][TM];
  float2 acc2[TN2][TM];
#pragma unroll
  for (int i = 0; i < TN; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = 0.f;
#pragma unroll
  for (int p = 0; p < TN2; ++p)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc2[p][j] = make_float2(0.f, 0.f);
  // window rows of this block: [window][2 NC] floats
  float* out = reinterpret_cast<float*>(a.partials) + (size_t)blockIdx.x * a.win * 2 * a.nc;
  const ScfConst* tabp = B::kGen ? a.tab : nullptr;
  int win = 0;

  const int prog = a.blk_prog[blockIdx.x];
  const float binv = (float)(1.0 / a.b_prog[prog]);
  const int64_t k_begin = a.blk_begin[blockIdx.x], k_end = a.blk_end[blockIdx.x];
  float4* pos4 = reinterpret_cast<float4*>(a.pos);
  const bool step = a.mode == SCF_MODE_STEP;
  int tiles = 0;
  for (int64_t base = k_begin; base < k_end; base += TP) {
    const bool last = base + TP >= k_end;
    // ---- basis of the tile
    float4 p_new = make_float4(0.f, 0.f, 0.f, 0.f), v_new = p_new;
    if (warp < BASIS_WARPS && lane < TP / 2) {
      const int t = (warp & 1) * (TP / 2) + lane;
      const int q = warp >> 1;
      const int64_t k = base + t;
      float x = 0.f, y = 0.f, z = 0.f, mass = 0.f;
      if (k < k_end) {
        float4 p = pos4[k];
        if (step) {
          float4 v = reinterpret_cast<float4*>(a.vel)[k];
          const float4 g = reinterpret_cast<const float4*>(a.acc)[k];
          const float h = (float)(0.5 * a.dt), dt = (float)a.dt;
          v.x += h * g.x;
          v.y += h * g.y;
          v.z += h * g.z;
          p.x += dt * v.x;
          p.y += dt * v.y;
          p.z += dt * v.z;
          p_new = p;
          v_new = v;
        }
        if (scf_finite3(p.x, p.y, p.z) && isfinite(p.w)) {
          x = p.x;
          y = p.y;
          z = p.z;
          mass = (a.mask == nullptr || a.mask[k]) ? p.w : 0.f;
        } else if (q == 0) {
          atomicOr(a.status, 1u);
        }
      }
      // the hardware reciprocal square root and reciprocal (a few ulp, no
      // slow-path branches; every thread of the particle's four repeats this)
      const float r2 = x * x + y * y + z * z;
      const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
      const float r = r2 * rinv;
      const float u = x * rinv, v = y * rinv, c = z * rinv;
      const float s = r * binv;
      // alpha != 1: t = s^(1/alpha) in q and xi, q^alpha in the prefactor
      const float qq = __fdividef(1.f, 1.f + (B::kGen ? powf(s, (float)a.inv_alpha) : s));
      const float xi = 1.f - 2.f * qq;
      const float qv = B::kGen ? powf(qq, (float)a.alpha) : qq;
      const float sq2 = s * qv * qv;
      B::run(q, Rs, Ys, t, NN, L, mass, u, v, c, qv, xi, sq2, SG);
    }
    __syncthreads();
    if (step && warp < 2 && lane < TP / 2) {  // chain set 0 writes the kicked and drifted state back
      const int64_t k = base + warp * (TP / 2) + lane;
      if (k < k_end) {
        pos4[k] = p_new;
        if (a.pos_copy) reinterpret_cast<float4*>(a.pos_copy)[k] = p_new;
        reinterpret_cast<float4*>(a.vel_out ? a.vel_out : a.vel)[k] = v_new;
      }
    }
    // ---- contraction of the tile into the register tiles
    if (worker) {
      for (int g = sgrp; g < TP / 4; g += a.sub) {
        const int t0 = 4 * g;
        if constexpr (TN <= TM) {  // the radial rows in registers, the angular ones streamed
          float4 rv[TN];
#pragma unroll
          for (int i = 0; i < TN; ++i) rv[i] = *reinterpret_cast<const float4*>(Rrow + i * TPP + t0);
#pragma unroll
          for (int j = 0; j < TM; ++j) {
            const float4 yv = *reinterpret_cast<const float4*>(Yrow + j * TPP + t0);
#pragma unroll
            for (int i = 0; i < TN; ++i) {
              acc[i][j] = fmaf(rv[i].x, yv.x, acc[i][j]);
              acc[i][j] = fmaf(rv[i].y, yv.y, acc[i][j]);
              acc[i][j] = fmaf(rv[i].z, yv.z, acc[i][j]);
              acc[i][j] = fmaf(rv[i].w, yv.w, acc[i][j]);
            }
          }
        } else if constexpr (S::kPairs) {
          // the angular rows in registers, the radial pair rows streamed: per
          // particle one packed FMA (each lane rounding as fmaf, the particles
          // in the same order) for the two radial orders of a pair
          // particles t0, t0 + 1 over all pair rows, then t0 + 2, t0 + 3
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float2 yv[TM];
#pragma unroll
            for (int j = 0; j < TM; ++j) yv[j] = *reinterpret_cast<const float2*>(Yrow + j * TPP + t0 + 2 * h);
#pragma unroll
            for (int p = 0; p < TN2; ++p) {
              const float4 r = *reinterpret_cast<const float4*>(Rrow + p * 2 * TPP + 2 * t0 + 4 * h);
#pragma unroll
              for (int j = 0; j < TM; ++j) {
                acc2[p][j] = __ffma2_rn(make_float2(r.x, r.y), make_float2(yv[j].x, yv[j].x), acc2[p][j]);
                acc2[p][j] = __ffma2_rn(make_float2(r.z, r.w), make_float2(yv[j].y, yv[j].y), acc2[p][j]);
              }
            }
            if constexpr (TN % 2 == 1) {
              const float4 r = *reinterpret_cast<const float4*>(Rrow + TN2 * 2 * TPP + 2 * t0 + 4 * h);
#pragma unroll
              for (int j = 0; j < TM; ++j) {
                acc[TN - 1][j] = fmaf(r.x, yv[j].x, acc[TN - 1][j]);
                acc[TN - 1][j] = fmaf(r.z, yv[j].y, acc[TN - 1][j]);
              }
            }
          }
        } else {  // the angular rows in registers, the radial ones streamed
          float4 yv[TM];
#pragma unroll
          for (int j = 0; j < TM; ++j) yv[j] = *reinterpret_cast<const float4*>(Yrow + j * TPP + t0);
#pragma unroll
          for (int i = 0; i < TN; ++i) {
            const float4 rv = *reinterpret_cast<const float4*>(Rrow + i * TPP + t0);
#pragma unroll
            for (int j = 0; j < TM; ++j) {
              acc[i][j] = fmaf(rv.x, yv[j].x, acc[i][j]);
              acc[i][j] = fmaf(rv.y, yv[j].y, acc[i][j]);
              acc[i][j] = fmaf(rv.z, yv[j].z, acc[i][j]);
              acc[i][j] = fmaf(rv.w, yv[j].w, acc[i][j]);
            }
          }
        }
      }
    }
    __syncthreads();
    if (++tiles == a.win_tiles || last) {  // the same on every thread of the block
      // end of a window: the worker tiles through shared memory, one row per window
      if (worker) {
        float* mine = red + (size_t)(sgrp * a.items + item) * (TN * TM);
        if constexpr (S::kPairs) {
#pragma unroll
          for (int p = 0; p < TN2; ++p)
#pragma unroll
            for (int j = 0; j < TM; ++j) {
              mine[2 * p * TM + j] = acc2[p][j].x;
              mine[(2 * p + 1) * TM + j] = acc2[p][j].y;
              acc2[p][j] = make_float2(0.f, 0.f);
            }
          if constexpr (TN % 2 == 1) {
#pragma unroll
            for (int j = 0; j < TM; ++j) {
              mine[(TN - 1) * TM + j] = acc[TN - 1][j];
              acc[TN - 1][j] = 0.f;
            }
          }
        } else if constexpr (TM % 4 == 0) {
#pragma unroll
          for (int i = 0; i < TN; ++i)
#pragma unroll
            for (int j = 0; j < TM; j += 4) {
              *reinterpret_cast<float4*>(mine + i * TM + j) =
                  make_float4(acc[i][j], acc[i][j + 1], acc[i][j + 2], acc[i][j + 3]);
              acc[i][j] = acc[i][j + 1] = acc[i][j + 2] = acc[i][j + 3] = 0.f;
            }
        } else {  // an odd tile (TN TM words per thread): word stores, no bank conflicts
#pragma unroll
          for (int i = 0; i < TN; ++i)
#pragma unroll
            for (int j = 0; j < TM; ++j) {
              mine[i * TM + j] = acc[i][j];
              acc[i][j] = 0.f;
            }
        }
      }
      __syncthreads();
      store_window<S>(red, out + (size_t)win * 2 * a.nc, a.items, a.sub, item_lnm, NN, a.nlm, a.nc, tabp);
      __syncthreads();  // the staging rows are the next tile's
      ++win;
      tiles = 0;
    }
  }
  // windows this block did not fill (fewer tiles than the longest block)
  for (; win < a.win; ++win)
    for (int i = tid; i < 2 * a.nc; i += blockDim.x) out[(size_t)win * 2 * a.nc + i] = 0.f;
}

template <class B>
struct K1Tiled {
  using S = typename B::S;
  static void* fn() { return (void*)k1_tiled<B>; }
  static void launch(const K1Args& a, int blocks, int threads, size_t smem, cudaStream_t s) {
    k1_tiled<B><<<blocks, threads, smem, s>>>(a);
  }
};

// Shapes with a compile-time basis: (nmax, lmax) = (20, 10), (20, 8), (10, 6), (10, 5);
// every other shape runs the runtime-indexed basis, and so does a radial
// family with alpha != 1 (gen), whose steps come from the handle's tables.
template <typename F>
auto dispatch_tiled(int nmax, int lmax, F&& f, bool gen = false) {
  if (gen) {
    if (nmax == 20 && lmax == 10) return f(K1Tiled<BasisFixed<21, 10, true>>());
    if (nmax == 20 && lmax == 8) return f(K1Tiled<BasisFixed<21, 8, true>>());
    if (nmax == 10 && lmax == 6) return f(K1Tiled<BasisFixed<11, 6, true>>());
    if (nmax == 10 && lmax == 5) return f(K1Tiled<BasisFixed<11, 5, true>>());
    switch ((lmax + 4) / 4) {
      case 1: return f(K1Tiled<BasisGeneric<1, true>>());
      case 2: return f(K1Tiled<BasisGeneric<2, true>>());
      case 3: return f(K1Tiled<BasisGeneric<3, true>>());
      default: return f(K1Tiled<BasisGeneric<4, true>>());
    }
  }
  if (nmax == 20 && lmax == 10) return f(K1Tiled<BasisFixed<21, 10>>());
  if (nmax == 20 && lmax == 8) return f(K1Tiled<BasisFixed<21, 8>>());
  if (nmax == 10 && lmax == 6) return f(K1Tiled<BasisFixed<11, 6>>());
  if (nmax == 10 && lmax == 5) return f(K1Tiled<BasisFixed<11, 5>>());
  switch ((lmax + 4) / 4) {
    case 1: return f(K1Tiled<BasisGeneric<1>>());
    case 2: return f(K1Tiled<BasisGeneric<2>>());
    case 3: return f(K1Tiled<BasisGeneric<3>>());
    default: return f(K1Tiled<BasisGeneric<4>>());
  }
}
}  // namespace tiled

// ---------------------------------------------------------------------------
// kernel 2
// ---------------------------------------------------------------------------
// Host acceleration at (x, y, z) evaluated by one warp: lane c computes
// component c and lane 0 adds them in component order, the same sum as
// scf_host_accel (the dependent double-precision chains of the components
// run side by side instead of one after another).  Result valid in lane 0.
__device__ void host_accel_warp(const ScfHostParams& hp, double x, double y, double z, double& ax, double& ay,
                                double& az) {
  const int lane = threadIdx.x & 31;
  double cx = 0.0, cy = 0.0, cz = 0.0;
  if (lane < hp.n) scf_host_comp_accel<double>(hp.kind[lane], hp.GM[lane], hp.a[lane], hp.b[lane], x, y, z, cx, cy, cz);
  ax = ay = az = 0.0;
  for (int c = 0; c < hp.n; ++c) {
    ax += __shfl_sync(0xffffffffu, cx, c);
    ay += __shfl_sync(0xffffffffu, cy, c);
    az += __shfl_sync(0xffffffffu, cz, c);
  }
}

// Kick-drift-kick of the centre (R, V) in the host field by one warp (every
// lane holds the same state), given a0 = a_host(R); returns a_host at the new
// R in a_new.
__device__ __forceinline__ void com_kdk_from(const ScfHostParams& hp, double* c, double dt, const double* a0,
                                             double* a_new) {
  double ax, ay, az;
  c[3] += 0.5 * dt * a0[0];
  c[4] += 0.5 * dt * a0[1];
  c[5] += 0.5 * dt * a0[2];
  c[0] += dt * c[3];
  c[1] += dt * c[4];
  c[2] += dt * c[5];
  host_accel_warp(hp, c[0], c[1], c[2], ax, ay, az);
  c[3] += 0.5 * dt * ax;
  c[4] += 0.5 * dt * ay;
  c[5] += 0.5 * dt * az;
  a_new[0] = ax;
  a_new[1] = ay;
  a_new[2] = az;
}

__device__ void com_kdk(const ScfHostParams& hp, double* c, double dt, double* a_new) {
  double a0[3];
  host_accel_warp(hp, c[0], c[1], c[2], a0[0], a0[1], a0[2]);
  com_kdk_from(hp, c, dt, a0, a_new);
}

__device__ __forceinline__ bool same_bits(double x, double y) {
  return __double_as_longlong(x) == __double_as_longlong(y);
}

// The R-only values of the single-precision tidal difference at centre c,
// component `lane` (< host.n) of progenitor p.
__device__ __forceinline__ void write_tidal_prep(const ScfHostParams& hp, float* tid_out, int p, int lane,
                                                 const double* c) {
  if (tid_out && lane < hp.n)
    scf_tidal_prep_f32(hp, lane, (float)c[0], (float)c[1], (float)c[2],
                       tid_out + ((size_t)p * SCF_HOST_CAP + lane) * SCF_TIDAL_W);
}

// The next step's centre kick-drift-kick, one warp per progenitor, from the
// state and a_host(R) that kernel 2 of this step left (see CentreArgs).
__global__ void __launch_bounds__(32) k_centre_next(CentreArgs a) {
  const int p = blockIdx.x;
  double c[6], a0[3], an[3];
  for (int d = 0; d < 6; ++d) c[d] = a.com[6 * p + d];
  for (int d = 0; d < 3; ++d) a0[d] = a.aR[4 * p + d];
  double* out = a.cnext + (size_t)kCentreW * p;
  if (threadIdx.x == 0)
    for (int d = 0; d < 6; ++d) out[d] = c[d];
  com_kdk_from(a.host, c, a.dt, a0, an);
  write_tidal_prep(a.host, a.tid_next, p, threadIdx.x, c);
  if (threadIdx.x == 0) {
    for (int d = 0; d < 6; ++d) out[6 + d] = c[d];
    for (int d = 0; d < 3; ++d) out[12 + d] = an[d];
    out[15] = a.dt;
  }
}

// Force-coefficient pair i of progenitor p (pi = p NC + i); single precision
// carries the field kernel's radial scale gscale (kscale_f[2i]; null: already
// applied by the caller).
__device__ __forceinline__ void write_force_pair(void* F, int f32, const float* kscale_f, size_t pi, int i, double c,
                                                 double s) {
  if (f32) {
    const double g = kscale_f ? (double)kscale_f[2 * i] : 1.0;
    reinterpret_cast<float2*>(F)[pi] = make_float2((float)(c * g), (float)(s * g));
  } else {
    reinterpret_cast<double2*>(F)[pi] = make_double2(c, s);
  }
}


// Kernel 2.  Block (groups, p) steps the centre of progenitor p and
// evaluates a_host there (a chain of dependent double-precision operations
// in one warp), concurrently with the reduction blocks.
// Block (g < groups, p): coefficient pairs 32g .. 32g + 31 (threadIdx.x, one
// 128-byte row segment per warp load) of progenitor p over all its partial
// rows, in SL = 8 row slices (threadIdx.y): slice y adds rows y, y + SL,
// ... in order, a batch of rows at a time whose loads are all
// issued before the first add (the kernel is a chain of memory latencies,
// not of bandwidth: one round trip per batch, one batch at the usual row
// counts); the slices are combined by a fixed binary tree (32 slices in
// 1024-thread blocks measured slower everywhere).  The epilogue's
// inputs (normalisation, 1/N_lm, b) are loaded before the rows.  Every sum
// has a fixed order, so the result is the same on every run.
constexpr int K2_X = 32, SL = 8;
__global__ void __launch_bounds__(K2_X * SL) k2_reduce(K2Args a) {
  __shared__ double s_c[SL][K2_X], s_s[SL][K2_X];
  const int p = blockIdx.y;
  const int x = threadIdx.x, y = threadIdx.y;
  const int groups = gridDim.x - 1;
  if ((int)blockIdx.x == groups) {  // the centre block: its first warp
    if (y == 0 && a.host.n > 0 && a.com != nullptr) {
      double c[6], an[3];
      for (int d = 0; d < 6; ++d) c[d] = a.com[6 * p + d];
      if (a.mode == SCF_MODE_STEP) {
        // the step computed ahead when it started from this very state
        const double* q = a.cnext ? a.cnext + (size_t)kCentreW * p : nullptr;
        bool hit = q != nullptr && same_bits(q[15], a.dt);
        for (int d = 0; d < 6 && hit; ++d) hit = same_bits(q[d], c[d]);
        if (hit) {
          for (int d = 0; d < 6; ++d) c[d] = q[6 + d];
          for (int d = 0; d < 3; ++d) an[d] = q[12 + d];
        } else {
          com_kdk(a.host, c, a.dt, an);
        }
        if (a.tid_out) {  // the tidal difference's R-only values, computed ahead or here
          constexpr int TW = SCF_HOST_CAP * SCF_TIDAL_W;
          if (hit && a.tid_next) {
            for (int k = x; k < TW; k += 32) a.tid_out[(size_t)p * TW + k] = a.tid_next[(size_t)p * TW + k];
          } else {
            write_tidal_prep(a.host, a.tid_out, p, x, c);
          }
        }
      } else {
        host_accel_warp(a.host, c[0], c[1], c[2], an[0], an[1], an[2]);
        write_tidal_prep(a.host, a.tid_out, p, x, c);
      }
      if (x == 0) {
        if (a.mode == SCF_MODE_STEP)
          for (int d = 0; d < 6; ++d) a.com[6 * p + d] = c[d];
        if (a.aR_out)
          for (int d = 0; d < 3; ++d) a.aR_out[4 * p + d] = an[d];
      }
    }
    return;
  }
  const int i = blockIdx.x * K2_X + x;
  const size_t stride = 2 * (size_t)a.nc;
  // the epilogue's factors first: their latency overlaps the row loads
  double nS = 0.0, nT = 0.0, w = 0.0;
  if (y == 0 && i < a.nc) {
    nS = a.norm[i];
    nT = a.norm[a.nc + i];
    if (a.F_out) {
      w = -a.G / a.b_prog[p] * c_tab.inv_nlm[i % a.nlm];
      if (a.f32) w *= (double)a.kscale_f[2 * i];  // single precision: F carries gscale
    }
  }
  double sc = 0.0, ss = 0.0;
  if (i < a.nc) {
    const int mul = a.sub == 0 ? 1 : a.sub;
    const int R0 = a.prog_blk_off[p] * mul, R1 = a.prog_blk_off[p + 1] * mul;
    if (a.sub == 0) {  // double rows, one per block
      constexpr int B = 8;
      const double* P = a.partials + i;
      for (int base = R0 + y; base < R1; base += B * SL) {
        double vc[B], vs[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const int r = base + k * SL;
          vc[k] = r < R1 ? P[(size_t)r * stride] : 0.0;
          vs[k] = r < R1 ? P[(size_t)r * stride + a.nc] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
          sc += vc[k];
          ss += vs[k];
        }
      }
    } else {  // float rows, a.sub per block; T_nl0 is not stored
      // a slice's rows are added as an unevaluated float pair (hi, lo) with an
      // error-free two-sum: single-precision arithmetic (the FP64 pipe is 1/64
      // of the FP32 one) at about twice single precision
      constexpr int B = 16;
      int lm = i % a.nlm, l = 0;
      while ((l + 1) * (l + 2) / 2 <= lm) ++l;
      const bool has_t = lm != scf_lm(l, 0);
      const float* P = reinterpret_cast<const float*>(a.partials) + i;
      float ch = 0.f, cl = 0.f, th = 0.f, tl = 0.f;
      auto two_sum = [](float& hi, float& lo, float v) {
        const float s = hi + v, bp = s - hi;
        lo += (hi - (s - bp)) + (v - bp);
        hi = s;
      };
      for (int base = R0 + y; base < R1; base += B * SL) {
        float vc[B], vs[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const int r = base + k * SL;
          vc[k] = r < R1 ? P[(size_t)r * stride] : 0.f;
          vs[k] = r < R1 && has_t ? P[(size_t)r * stride + a.nc] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
          two_sum(ch, cl, vc[k]);
          two_sum(th, tl, vs[k]);
        }
      }
      sc = (double)ch + (double)cl;
      ss = (double)th + (double)tl;
    }
  }
  s_c[y][x] = sc;
  s_s[y][x] = ss;
  __syncthreads();
#pragma unroll
  for (int h = SL / 2; h >= 1; h >>= 1) {
    if (y < h) {
      s_c[y][x] += s_c[y + h][x];
      s_s[y][x] += s_s[y + h][x];
    }
    __syncthreads();
  }
  if (y == 0 && i < a.nc) {
    const double S = s_c[0][x] * nS, T = s_s[0][x] * nT;
    double* A = a.A_out + (size_t)p * stride;
    A[i] = S;
    A[a.nc + i] = T;
    if (a.F_out) write_force_pair(a.F_out, a.f32, nullptr, (size_t)p * a.nc + i, i, w * S, w * T);
  }
}

__global__ void k_prep(PrepArgs a) {
  const int p = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.nc) {
    const double* A = a.A + (size_t)p * 2 * a.nc;
    const double w = -a.G / a.b_prog[p] * c_tab.inv_nlm[i % a.nlm];
    write_force_pair(a.F_out, a.f32, a.kscale_f, (size_t)p * a.nc + i, i, w * A[i], w * A[a.nc + i]);
  }
  if (blockIdx.x == 0 && a.host.n > 0 && a.com != nullptr) {
    const double* c = a.com + 6 * p;
    if (threadIdx.x == 0) {
      double* r = a.aR_out + 4 * p;
      scf_host_accel(a.host, c[0], c[1], c[2], r[0], r[1], r[2]);
    }
    write_tidal_prep(a.host, a.tid_out, p, threadIdx.x, c);
  }
}

template <typename T, int TP, int LMAX, bool GEN = false>
struct K1At {
  static void* fn() { return (void*)k1_partials<T, LMAX, TP, GEN>; }
  static size_t smem(int nmax, int nc) { return k1_smem<T, LMAX, TP>(nmax, nc); }
  static void launch(const K1Args& a, int blocks, size_t smem, cudaStream_t s) {
    k1_partials<T, LMAX, TP, GEN><<<blocks, TP, smem, s>>>(a);
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

template <typename T, int TP, typename F, bool GEN = false>
auto dispatch_lmax(int lmax, F&& f) {
  switch (lmax_bucket(lmax)) {
    case 2: return f(K1At<T, TP, 2, GEN>());
    case 4: return f(K1At<T, TP, 4, GEN>());
    case 6: return f(K1At<T, TP, 6, GEN>());
    case 8: return f(K1At<T, TP, 8, GEN>());
    case 10: return f(K1At<T, TP, 10, GEN>());
    default: return f(K1At<T, TP, 12, GEN>());
  }
}

// Kernel 1 instantiations: particle tiles of 64, 128 or 256 (the autotuner's choices).
template <typename T, typename F>
auto dispatch_k1(int tp, int lmax, F&& f) {
  switch (tp) {
    case 64: return dispatch_lmax<T, 64>(lmax, f);
    case 256: return dispatch_lmax<T, 256>(lmax, f);
    default: return dispatch_lmax<T, 128>(lmax, f);
  }
}

}  // namespace

template <typename T, bool GEN = false>
static cudaError_t k1_prepare_t(int lmax, int nmax, int tp, ScfLaunchInfo* info, int* blocks_per_sm) {
  const int nlm = (lmax + 1) * (lmax + 2) / 2, nc = (nmax + 1) * nlm;
  if (tp != 64 && tp != 128 && tp != 256) return cudaErrorInvalidValue;
  if (GEN && tp != 128) return cudaErrorInvalidValue;
  auto body = [&](auto k) -> cudaError_t {
    using KK = decltype(k);
    info->threads = tp;
    info->tile = tp;
    info->variant = GEN ? 3 : 0;
    info->smem = KK::smem(nmax, nc);
    if (info->smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(KK::fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)info->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, KK::fn(), info->threads, info->smem);
  };
  if constexpr (GEN) return dispatch_lmax<T, 128, decltype(body)&, true>(lmax, body);
  else return dispatch_k1<T>(tp, lmax, body);
}

cudaError_t scf_k1_prepare(int precision, int lmax, int nmax, int tp, ScfLaunchInfo* info, int* blocks_per_sm) {
  if (precision == 1) return k1_prepare_t<float>(lmax, nmax, tp, info, blocks_per_sm);
  return k1_prepare_t<double>(lmax, nmax, tp, info, blocks_per_sm);
}

cudaError_t scf_k1_gen_prepare(int precision, int lmax, int nmax, ScfLaunchInfo* info, int* blocks_per_sm) {
  if (precision == 1) return k1_prepare_t<float, true>(lmax, nmax, 128, info, blocks_per_sm);
  return k1_prepare_t<double, true>(lmax, nmax, 128, info, blocks_per_sm);
}

cudaError_t scf_k1_tiled_prepare(int lmax, int nmax, ScfLaunchInfo* info, int* blocks_per_sm, bool gen) {
  using namespace tiled;
  return dispatch_tiled(nmax, lmax, [&](auto k) -> cudaError_t {
    using KK = decltype(k);
    using S = typename KK::S;
    const int items = S::n_items(nmax, lmax);
    if (items > MAX_THREADS) return cudaErrorInvalidConfiguration;
    const int sub = std::min(TP / 4, std::max(1, MAX_THREADS / items));
    info->items = items;
    info->sub = sub;
    info->threads = std::max(BASIS_WARPS * 32, 32 * ((items * sub + 31) / 32));
    info->tile = TP;
    info->variant = 1;
    info->win = 1;  // set from the block map by the caller (scf_k1_windows)
    info->win_tiles = WINDOW_TILES;
    info->smem = S::smem_bytes(nmax, lmax, gen);
    if (info->smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(KK::fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)info->smem);
    if (e != cudaSuccess) return e;
    // two ~100 KB blocks per SM need the largest shared-memory carveout
    e = cudaFuncSetAttribute(KK::fn(), cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, KK::fn(), info->threads, info->smem);
  }, gen);
}

int scf_k1_windows(int64_t max_particles_per_block, const ScfLaunchInfo& info) {
  const int64_t tiles = (max_particles_per_block + info.tile - 1) / info.tile;
  return (int)std::max<int64_t>(1, (tiles + info.win_tiles - 1) / info.win_tiles);
}

cudaError_t scf_k1_launch(int precision, const K1Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s) {
  if (info.variant == 1) {
    K1Args b = a;
    b.items = info.items;
    b.sub = info.sub;
    b.win = info.win;
    b.win_tiles = info.win_tiles;
    tiled::dispatch_tiled(a.nmax, a.lmax, [&](auto k) -> int {
      decltype(k)::launch(b, blocks, info.threads, info.smem, s);
      return 0;
    }, a.tab != nullptr);
    return cudaGetLastError();
  }
  auto go = [&](auto k) -> int {
    decltype(k)::launch(a, blocks, info.smem, s);
    return 0;
  };
  if (info.variant == 3) {  // radial family of exponent alpha != 1, 128-particle tiles
    if (precision == 1) dispatch_lmax<float, 128, decltype(go)&, true>(a.lmax, go);
    else dispatch_lmax<double, 128, decltype(go)&, true>(a.lmax, go);
  } else if (precision == 1) {
    dispatch_k1<float>(info.tile, a.lmax, go);
  } else {
    dispatch_k1<double>(info.tile, a.lmax, go);
  }
  return cudaGetLastError();
}

cudaError_t scf_k2_launch(const K2Args& a, cudaStream_t s) {
  const int groups = (a.nc + K2_X - 1) / K2_X;
  dim3 grid(groups + 1, a.n_prog);  // + the centre block
  k2_reduce<<<grid, dim3(K2_X, SL), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t scf_centre_next_launch(const CentreArgs& a, int priority, cudaStream_t s) {
  // at the stream priority given: its blocks take the first SM slots that
  // kernel 3 frees instead of queueing behind all of kernel 3's blocks
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(a.n_prog);
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = priority;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_centre_next, a);
}

cudaError_t scf_prep_launch(const PrepArgs& a, cudaStream_t s) {
  dim3 grid((a.nc + 127) / 128, a.n_prog);
  k_prep<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}
