// scf_coeffs_noalloc: the coefficient sums of one cluster without allocating
// anything, for callers that cannot call cudaMalloc.  Typical such callers:
// a stage that runs inside somebody else's memory pool or arena and must
// not fragment it; a code path that runs where device allocation is not
// permitted or would synchronise the device (e.g. between the steps of an
// externally managed integrator); or a plugin that gets device pointers from
// its host application but no allocator.  They pass inputs and outputs;
// everything else lives in one file-scope device array declared here.
//
// The scratch is a static __device__ array: every GPU that loads this
// library holds it (about 10.5 MiB) from load until process exit.  Host code
// cannot use the array's name as a device address, so the first call on a
// device looks up its address with cudaGetSymbolAddress (with that device
// current) and passes that pointer to the kernels.  Because that first call
// does this set-up (and uploads the recurrence tables), it should come before
// any stream capture.  All calls share the one array and it keeps the last
// call's contents; each call rewrites everything it reads (block map,
// normalisation, status word, and the partial sums of every block it
// launches), so no state leaks from one call to the next.  Calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// the array and give wrong results: serialise them.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <mutex>

#include "../../include/scf.h"
#include "scf_device.cuh"
#include "scf_internal.h"

namespace {

struct NoallocScratch {
  double partials[SCF_NOALLOC_MAX_BLOCKS * SCF_NOALLOC_MAX_COEFS];
  double norm[SCF_NOALLOC_MAX_COEFS];
  int64_t blk_begin[SCF_NOALLOC_MAX_BLOCKS];
  int64_t blk_end[SCF_NOALLOC_MAX_BLOCKS];
  int blk_prog[SCF_NOALLOC_MAX_BLOCKS];
  int prog_blk_off[2];
  double b[1];
  unsigned status[4];
};

static __device__ __align__(256) NoallocScratch g_scratch;

struct DeviceSetup {
  bool ready = false;
  NoallocScratch* scratch = nullptr;  // device address of g_scratch on this device
  int n_sm = 0;
};

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];
ScfConst g_tables_host;  // static storage: the set-up allocates nothing

// Writes the block map, the basis scale, the normalisation of Eq. 3b and a
// cleared status word into the scratch.  Normalisation: S = -(2 - delta_m0)
// N_lm / I_nl(b = 1) * (raw sum), the same factor the handle path uses.
__global__ void noalloc_setup(NoallocScratch* s, int64_t n, int64_t span, int blocks, double b, int nmax, int lmax) {
  const int nlm = (lmax + 1) * (lmax + 2) / 2, nc = (nmax + 1) * nlm;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < blocks) {
    s->blk_prog[i] = 0;
    s->blk_begin[i] = (int64_t)i * span;
    s->blk_end[i] = min((int64_t)(i + 1) * span, n);
  }
  if (i == 0) {
    s->prog_blk_off[0] = 0;
    s->prog_blk_off[1] = blocks;
    s->b[0] = b;
    s->status[0] = 0u;
  }
  if (i < nc) {
    const int nn = i / nlm, lm = i - nn * nlm;
    int l = 0;
    while ((l + 1) * (l + 2) / 2 <= lm) ++l;
    const int m = lm - l * (l + 1) / 2;
    double ratio = 1.0;
    for (int k = l - m + 1; k <= l + m; ++k) ratio /= (double)k;
    const double nlm_norm = sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846) * ratio);
    const double knl = 0.5 * nn * (nn + 4.0 * l + 3.0) + (l + 1.0) * (2.0 * l + 1.0);
    const double lg = lgamma(nn + 4.0 * l + 3.0) - (8.0 * l + 6.0) * log(2.0) - lgamma(nn + 1.0) -
                      log(nn + 2.0 * l + 1.5) - 2.0 * lgamma(2.0 * l + 1.5);
    const double inl = -knl * exp(lg);
    const double f = -(m == 0 ? 1.0 : 2.0) * nlm_norm / inl;
    s->norm[i] = f;
    s->norm[nc + i] = (m == 0) ? 0.0 : f;
  }
}

int setup_device(int device, DeviceSetup** out) {
  if (device < 0 || device >= kMaxDevices) return SCF_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& d = g_setup[device];
  if (!d.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || ptr == nullptr) return SCF_ERR_CUDA;
    scf_make_const(&g_tables_host);
    if (scf_upload_const_coeffs(&g_tables_host) != cudaSuccess) return SCF_ERR_CUDA;
    if (cudaDeviceGetAttribute(&d.n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return SCF_ERR_CUDA;
    d.scratch = static_cast<NoallocScratch*>(ptr);
    d.ready = true;
  }
  *out = &d;
  return SCF_OK;
}

}  // namespace

extern "C" int scf_coeffs_noalloc(const scf_config* cfg, int64_t n, const void* pos, const uint8_t* mask,
                                  double* A_out, void* stream) {
  if (!cfg || !A_out || (!pos && n > 0)) return SCF_ERR_NULL_POINTER;
  if (n < 0 || cfg->nmax < 0 || cfg->lmax < 0) return SCF_ERR_INVALID_ARG;
  if (cfg->nmax > SCF_MAX_NMAX || cfg->lmax > SCF_MAX_LMAX || cfg->alpha != 1.0) return SCF_ERR_UNSUPPORTED;
  if (cfg->precision != SCF_FP64 && cfg->precision != SCF_MIXED) return SCF_ERR_INVALID_ARG;
  if (!(cfg->b > 0.0) || !std::isfinite(cfg->b)) return SCF_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(pos) & 15u) != 0) return SCF_ERR_MISALIGNED;
  const int nlm = (cfg->lmax + 1) * (cfg->lmax + 2) / 2, nc = (cfg->nmax + 1) * nlm;
  if (2 * nc > SCF_NOALLOC_MAX_COEFS) return SCF_ERR_TOO_LARGE;

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return SCF_ERR_CUDA;
  DeviceSetup* d = nullptr;
  int rc = setup_device(device, &d);
  if (rc != SCF_OK) return rc;
  ScfLaunchInfo info{};
  int bps = 0;
  if (scf_k1_prepare(cfg->precision, cfg->lmax, cfg->nmax, 128, &info, &bps) != cudaSuccess || bps < 1)
    return SCF_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  // Block map: whole tiles of info.tile particles, about one wave of
  // resident blocks, at most as many blocks as the scratch holds partials for.
  const int64_t tp = info.tile;
  const int64_t tiles = (n + tp - 1) / tp;
  int64_t max_blocks = std::min<int64_t>(SCF_NOALLOC_MAX_BLOCKS, SCF_NOALLOC_MAX_COEFS * (int64_t)SCF_NOALLOC_MAX_BLOCKS / (2 * nc));
  max_blocks = std::min<int64_t>(max_blocks, (int64_t)d->n_sm * bps);
  const int64_t tiles_per_block = tiles == 0 ? 1 : (tiles + max_blocks - 1) / max_blocks;
  const int blocks = (int)((tiles + tiles_per_block - 1) / tiles_per_block);
  const int64_t span = tiles_per_block * tp;

  NoallocScratch* sc = d->scratch;
  const int setup_threads = std::max(blocks, nc);
  noalloc_setup<<<(setup_threads + 127) / 128, 128, 0, s>>>(sc, n, span, blocks, cfg->b, cfg->nmax, cfg->lmax);
  if (cudaGetLastError() != cudaSuccess) return SCF_ERR_CUDA;
  if (blocks > 0) {
    K1Args a{};
    a.pos = const_cast<void*>(pos);
    a.mask = mask;
    a.partials = sc->partials;
    a.blk_prog = sc->blk_prog;
    a.blk_begin = sc->blk_begin;
    a.blk_end = sc->blk_end;
    a.b_prog = sc->b;
    a.nmax = cfg->nmax;
    a.lmax = cfg->lmax;
    a.nc = nc;
    a.nlm = nlm;
    a.mode = SCF_MODE_COEFFS;
    a.status = sc->status;
    if (scf_k1_launch(cfg->precision, a, blocks, info, s) != cudaSuccess) return SCF_ERR_CUDA;
  }
  K2Args r{};
  r.partials = sc->partials;
  r.prog_blk_off = sc->prog_blk_off;
  r.norm = sc->norm;
  r.A_out = A_out;
  r.nc = nc;
  r.nlm = nlm;
  r.n_prog = 1;
  r.mode = SCF_MODE_COEFFS;
  return scf_k2_launch(r, s) == cudaSuccess ? SCF_OK : SCF_ERR_CUDA;
}

extern "C" int scf_noalloc_status(void* stream, int* status) {
  if (status) *status = 0;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return SCF_ERR_CUDA;
  if (device < 0 || device >= kMaxDevices) return SCF_ERR_UNSUPPORTED;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_setup[device].ready) return SCF_OK;  // no call has run on this device
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned word = 0;
  if (cudaMemcpyFromSymbolAsync(&word, g_scratch, sizeof(unsigned), offsetof(NoallocScratch, status),
                                cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SCF_ERR_CUDA;
  if (status) *status = (int)word;
  return word != 0 ? SCF_ERR_DEVICE_STATUS : SCF_OK;
}
