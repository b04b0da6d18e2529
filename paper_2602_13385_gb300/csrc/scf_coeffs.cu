// Kernel 1 (coefficient partial sums, Eq. 3b) and kernel 2 (deterministic
// reduction, normalisation, centre-of-mass step).
//
// Kernel 1 works on tiles of TP particles, one thread per particle in the
// basis phase.  For each degree l the block stages, in shared memory, the
// radial factors R[t][n] = m_t s^l q^(2l+1) C_n(xi_t) and the angular factors
// Y[t][mm] = Pb_lm C_m (mm = m) or Pb_lm S_m (mm = l + m), then every thread
// contracts a slice of the (n, mm) outputs over the tile's particles and adds
// it to the block's running sums.  The sums leave the block as one partial
// vector per block; kernel 2 adds the partials of each progenitor in block
// order, so the result does not depend on scheduling.
#include <cstdio>

#include "scf_device.cuh"
#include "scf_internal.h"

static __constant__ ScfConst c_tab;

cudaError_t scf_upload_const_coeffs(const ScfConst* t) { return cudaMemcpyToSymbol(c_tab, t, sizeof(ScfConst)); }

namespace {

template <typename T> struct Vec4;
template <> struct Vec4<double> { using type = ScfD4; };
template <> struct Vec4<float> { using type = float4; };

template <typename T> __device__ __forceinline__ T tab_gA(int l, int n);
template <> __device__ __forceinline__ double tab_gA<double>(int l, int n) { return c_tab.gA[l][n]; }
template <> __device__ __forceinline__ float tab_gA<float>(int l, int n) { return c_tab.gAf[l][n]; }
template <typename T> __device__ __forceinline__ T tab_gB(int l, int n);
template <> __device__ __forceinline__ double tab_gB<double>(int l, int n) { return c_tab.gB[l][n]; }
template <> __device__ __forceinline__ float tab_gB<float>(int l, int n) { return c_tab.gBf[l][n]; }
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

template <typename T, int LMAX, int TP>
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
    const T q = (T)1 / ((T)1 + s);
    const T xi = (T)1 - (T)2 * q;
    const T sq2 = s * q * q;
    T Wc[LMAX + 1], Ws[LMAX + 1];
    Wc[0] = 1;
    Ws[0] = 0;
#pragma unroll
    for (int m = 1; m <= LMAX; ++m) {
      Wc[m] = Wc[m - 1] * u - Ws[m - 1] * v;
      Ws[m] = Wc[m - 1] * v + Ws[m - 1] * u;
    }
    T P[LMAX + 1], P1[LMAX + 1], P2[LMAX + 1];
    T pre = mass * q;  // m_k s^l q^(2l+1) at l = 0

#pragma unroll
    for (int l = 0; l <= LMAX; ++l) {
      if (l > a.lmax) break;
      // Legendre row l
#pragma unroll
      for (int m = 0; m + 2 <= l; ++m)
        P[m] = tab_la<T>(scf_lm(l, m)) * c * P1[m] - tab_lb<T>(scf_lm(l, m)) * P2[m];
      if (l >= 1) P[l - 1] = tab_lsub<T>(l) * c * P1[l - 1];
      P[l] = tab_ldiag<T>(l);
      // radial factors
      {
        T cm1 = 0, c0 = 1;
        T* Rt = R + tid * NN;
        Rt[0] = pre;
        for (int n = 1; n < NN; ++n) {
          const T cn = tab_gA<T>(l, n) * xi * c0 - tab_gB<T>(l, n) * cm1;
          cm1 = c0;
          c0 = cn;
          Rt[n] = pre * cn;
        }
      }
      // angular factors
      {
        T* Yt = Y + tid * YS;
#pragma unroll
        for (int m = 0; m <= l; ++m) Yt[m] = P[m] * Wc[m];
#pragma unroll
        for (int m = 1; m <= l; ++m) Yt[l + m] = P[m] * Ws[m];
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
  for (int i = tid; i < 2 * a.nc; i += TP) out[i] = Acc::value(acc, i);
}

template <typename T, int LMAX, int TP>
size_t k1_smem(int nmax, int nc) {
  using Slot = typename BlockAcc<T>::slot;
  return sizeof(Slot) * 2 * (size_t)nc + sizeof(T) * (size_t)TP * ((nmax + 1) + (2 * LMAX + 1));
}

// ---------------------------------------------------------------------------
// kernel 2
// ---------------------------------------------------------------------------
__device__ void com_kdk(const ScfHostParams& hp, double* c, double dt) {
  double ax, ay, az;
  scf_host_accel(hp, c[0], c[1], c[2], ax, ay, az);
  c[3] += 0.5 * dt * ax;
  c[4] += 0.5 * dt * ay;
  c[5] += 0.5 * dt * az;
  c[0] += dt * c[3];
  c[1] += dt * c[4];
  c[2] += dt * c[5];
  scf_host_accel(hp, c[0], c[1], c[2], ax, ay, az);
  c[3] += 0.5 * dt * ax;
  c[4] += 0.5 * dt * ay;
  c[5] += 0.5 * dt * az;
}

__device__ __forceinline__ void write_force_pair(void* F, int f32, size_t i, double c, double s) {
  if (f32) reinterpret_cast<float2*>(F)[i] = make_float2((float)c, (float)s);
  else reinterpret_cast<double2*>(F)[i] = make_double2(c, s);
}

// One warp per (cosine, sine) coefficient pair of one progenitor: lane j
// sums the partials of blocks j, j+32, ... in order, then a fixed shuffle
// tree combines the lanes, so the result is the same on every run.
__global__ void k2_reduce(K2Args a) {
  const int p = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (i < a.nc) {
    const int b0 = a.prog_blk_off[p], b1 = a.prog_blk_off[p + 1];
    const size_t stride = 2 * (size_t)a.nc;
    double sc = 0.0, ss = 0.0;
    for (int b = b0 + lane; b < b1; b += 32) {
      const double* src = a.partials + (size_t)b * stride + i;
      sc += src[0];
      ss += src[a.nc];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sc += __shfl_xor_sync(0xffffffffu, sc, o);
      ss += __shfl_xor_sync(0xffffffffu, ss, o);
    }
    if (lane == 0) {
      const double S = sc * a.norm[i], T = ss * a.norm[a.nc + i];
      double* A = a.A_out + (size_t)p * stride;
      A[i] = S;
      A[a.nc + i] = T;
      if (a.F_out) {
        const double w = -a.G / a.b_prog[p] * c_tab.inv_nlm[i % a.nlm];
        write_force_pair(a.F_out, a.f32, (size_t)p * a.nc + i, w * S, w * T);
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.host.n > 0 && a.com != nullptr) {
    double* c = a.com + 6 * p;
    if (a.mode == SCF_MODE_STEP) com_kdk(a.host, c, a.dt);
    if (a.aR_out) {
      double* r = a.aR_out + 4 * p;
      scf_host_accel(a.host, c[0], c[1], c[2], r[0], r[1], r[2]);
    }
  }
}

__global__ void k_prep(PrepArgs a) {
  const int p = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.nc) {
    const double* A = a.A + (size_t)p * 2 * a.nc;
    const double w = -a.G / a.b_prog[p] * c_tab.inv_nlm[i % a.nlm];
    write_force_pair(a.F_out, a.f32, (size_t)p * a.nc + i, w * A[i], w * A[a.nc + i]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.host.n > 0 && a.com != nullptr) {
    const double* c = a.com + 6 * p;
    double* r = a.aR_out + 4 * p;
    scf_host_accel(a.host, c[0], c[1], c[2], r[0], r[1], r[2]);
  }
}

template <typename T, int TP, int LMAX>
struct K1At {
  static void* fn() { return (void*)k1_partials<T, LMAX, TP>; }
  static size_t smem(int nmax, int nc) { return k1_smem<T, LMAX, TP>(nmax, nc); }
  static void launch(const K1Args& a, int blocks, size_t smem, cudaStream_t s) {
    k1_partials<T, LMAX, TP><<<blocks, TP, smem, s>>>(a);
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

template <typename T, int TP, typename F>
auto dispatch_lmax(int lmax, F&& f) {
  switch (lmax_bucket(lmax)) {
    case 2: return f(K1At<T, TP, 2>());
    case 4: return f(K1At<T, TP, 4>());
    case 6: return f(K1At<T, TP, 6>());
    case 8: return f(K1At<T, TP, 8>());
    case 10: return f(K1At<T, TP, 10>());
    default: return f(K1At<T, TP, 12>());
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

template <typename T>
static cudaError_t k1_prepare_t(int lmax, int nmax, int tp, ScfLaunchInfo* info, int* blocks_per_sm) {
  const int nlm = (lmax + 1) * (lmax + 2) / 2, nc = (nmax + 1) * nlm;
  if (tp != 64 && tp != 128 && tp != 256) return cudaErrorInvalidValue;
  return dispatch_k1<T>(tp, lmax, [&](auto k) -> cudaError_t {
    using KK = decltype(k);
    info->threads = tp;
    info->tile = tp;
    info->variant = 0;
    info->smem = KK::smem(nmax, nc);
    if (info->smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(KK::fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)info->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, KK::fn(), info->threads, info->smem);
  });
}

cudaError_t scf_k1_prepare(int precision, int lmax, int nmax, int tp, ScfLaunchInfo* info, int* blocks_per_sm) {
  if (precision == 1) return k1_prepare_t<float>(lmax, nmax, tp, info, blocks_per_sm);
  return k1_prepare_t<double>(lmax, nmax, tp, info, blocks_per_sm);
}

cudaError_t scf_k1_launch(int precision, const K1Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s) {
  auto go = [&](auto k) -> int {
    decltype(k)::launch(a, blocks, info.smem, s);
    return 0;
  };
  if (precision == 1) dispatch_k1<float>(info.tile, a.lmax, go);
  else dispatch_k1<double>(info.tile, a.lmax, go);
  return cudaGetLastError();
}

cudaError_t scf_k2_launch(const K2Args& a, cudaStream_t s) {
  dim3 grid((a.nc + 7) / 8, a.n_prog);  // 8 warps per block, one pair per warp
  k2_reduce<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t scf_prep_launch(const PrepArgs& a, cudaStream_t s) {
  dim3 grid((a.nc + 127) / 128, a.n_prog);
  k_prep<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}
