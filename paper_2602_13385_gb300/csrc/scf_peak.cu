// Throughput of independent FMA chains on the single- and double-precision
// pipes.  The field and coefficient kernels are bound by these pipes (no
// tensor cores, no HBM limit), so this rate is the measured counterpart of the
// nominal peak (units per SM x SMs x clock) that their roofline fractions use.
#include <cuda_runtime.h>

#include "../../include/scf.h"

namespace {

__device__ double g_peak_sink;

// CH independent chains per thread, x <- x a + b, with a just below 1 so the
// values stay near 1 (no overflow, no subnormals).  The final test depends on
// every chain, so none of them is dead code; it is never true.
template <typename T, int CH, int UNROLL>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b) {
  T x[CH];
#pragma unroll
  for (int j = 0; j < CH; ++j) x[j] = (T)1 + (T)(threadIdx.x + 37 * j) * (T)1e-4;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u)
#pragma unroll
      for (int j = 0; j < CH; ++j) x[j] = fma(x[j], a, b);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < CH; ++j) s += x[j];
  if (s == (T)-1.2345) g_peak_sink = (double)s;
}

constexpr int kChains = 8, kUnroll = 16, kThreads = 256, kBlocksPerSm = 8;

}  // namespace

extern "C" int scf_fma_peak(int precision, int iters, void* stream, double* flops_out, double* ms_out) {
  if (!flops_out) return SCF_ERR_NULL_POINTER;
  if (iters < 1 || (precision != SCF_FP64 && precision != SCF_MIXED)) return SCF_ERR_INVALID_ARG;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SCF_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = n_sm * kBlocksPerSm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SCF_ERR_CUDA;
  auto launch = [&] {
    if (precision == SCF_FP64)
      k_fma_chains<double, kChains, kUnroll><<<blocks, kThreads, 0, s>>>(iters, 0.9999999999, 1e-10);
    else
      k_fma_chains<float, kChains, kUnroll><<<blocks, kThreads, 0, s>>>(iters, 0.9999999f, 1e-7f);
  };
  launch();  // warm-up
  float best = 1e30f;
  int rc = SCF_OK;
  for (int r = 0; r < 3 && rc == SCF_OK; ++r) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = SCF_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  if (rc == SCF_OK && cudaGetLastError() != cudaSuccess) rc = SCF_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SCF_OK) return rc;
  const double fmas = (double)blocks * kThreads * kChains * kUnroll * (double)iters;
  *flops_out = 2.0 * fmas / (best * 1e-3);
  if (ms_out) *ms_out = best;
  return SCF_OK;
}
