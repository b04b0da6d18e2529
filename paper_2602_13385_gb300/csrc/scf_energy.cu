// Energy diagnostic of every progenitor in its accelerating, non-rotating
// frame (Sec. 2.1), double precision and deterministic:
//   K = sum_k 1/2 m_k |v_k|^2,
//   W = 1/2 sum_k m_k psi_SCF(x_k)  (psi_SCF = acc.w, as kernel 3 stores it),
//   U = sum_k m_k [psi_host(R + x_k) - psi_host(R) + x_k . a_host(R)],
// U being the potential of the frame's tidal acceleration a_host(R+x) - a_host(R).
// For an isolated cluster K + W is the conserved energy of the self-consistent
// system (the expansion's potential is a symmetric pair kernel).
//
// Kernel 1 below: one block per kernel-3 block range, a fixed shuffle tree in
// each warp and the warps in order, one row of partials per block.  Kernel 2:
// one warp per progenitor adds its blocks' rows in block order.
#include "scf_device.cuh"
#include "scf_internal.h"

namespace {

constexpr int kEnergyThreads = 128;

template <typename V4>
__global__ void __launch_bounds__(kEnergyThreads) k_energy_blocks(EnergyArgs a) {
  constexpr int NW = kEnergyThreads / 32;
  __shared__ double s_w[NW][3];
  __shared__ double s_R[3], s_aR[3], s_pR;
  const int tid = threadIdx.x;
  const int prog = a.blk_prog[blockIdx.x];
  const bool has_host = a.host.n > 0 && a.com != nullptr;
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) s_R[i] = has_host ? a.com[6 * prog + i] : 0.0;
    if (has_host) {
      scf_host_accel(a.host, s_R[0], s_R[1], s_R[2], s_aR[0], s_aR[1], s_aR[2]);
      s_pR = scf_host_pot(a.host, s_R[0], s_R[1], s_R[2]);
    }
  }
  __syncthreads();
  double e[3] = {0.0, 0.0, 0.0};
  const V4* pos = reinterpret_cast<const V4*>(a.pos);
  const V4* vel = reinterpret_cast<const V4*>(a.vel);
  const V4* acc = reinterpret_cast<const V4*>(a.acc);
  const int64_t end = a.blk_end[blockIdx.x];
  for (int64_t k = a.blk_begin[blockIdx.x] + tid; k < end; k += kEnergyThreads) {
    const V4 p = pos[k], v = vel[k], g = acc[k];
    const double m = p.w;
    e[0] += 0.5 * m * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
    e[1] += 0.5 * m * (double)g.w;
    if (has_host) {
      const double x = p.x, y = p.y, z = p.z;
      e[2] += m * (scf_host_pot(a.host, s_R[0] + x, s_R[1] + y, s_R[2] + z) - s_pR +
                   (x * s_aR[0] + y * s_aR[1] + z * s_aR[2]));
    }
  }
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double v = e[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_w[warp][i] = v;
  }
  __syncthreads();
  if (tid < 3) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) v += s_w[w][tid];
    a.part[(size_t)blockIdx.x * 4 + tid] = v;
  }
}

__global__ void k_energy_sum(EnergyArgs a) {
  const int p = blockIdx.x, lane = threadIdx.x;
  double e[3] = {0.0, 0.0, 0.0};
  for (int b = lane; b < a.n_blocks; b += 32) {
    if (a.blk_prog[b] != p) continue;
    for (int i = 0; i < 3; ++i) e[i] += a.part[(size_t)b * 4 + i];
  }
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e[i] += __shfl_xor_sync(0xffffffffu, e[i], o);
  if (lane == 0) {
    double* out = a.E_out + 4 * (size_t)p;
    out[0] = e[0];
    out[1] = e[1];
    out[2] = e[2];
    out[3] = e[0] + e[1] + e[2];
  }
}

}  // namespace

cudaError_t scf_energy_launch(const EnergyArgs& a, cudaStream_t s) {
  if (a.n_blocks > 0) {
    if (a.f32) k_energy_blocks<float4><<<a.n_blocks, kEnergyThreads, 0, s>>>(a);
    else k_energy_blocks<ScfD4><<<a.n_blocks, kEnergyThreads, 0, s>>>(a);
  }
  k_energy_sum<<<a.n_prog, 32, 0, s>>>(a);
  return cudaGetLastError();
}
