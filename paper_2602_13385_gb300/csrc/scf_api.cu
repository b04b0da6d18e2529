// C ABI of the SCF gravity step (declared in include/scf.h): argument
// validation, workspace ownership, block maps and kernel launches.
#include <algorithm>
#include <queue>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/scf.h"
#include "scf_device.cuh"
#include "scf_internal.h"
#include "scf_escape.h"

struct scf_handle {
  scf_config cfg;
  int n_prog = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  int nlm = 0, nc = 0;
  int64_t n_total = 0;
  int n_sm = 0;
  std::vector<int64_t> offsets;
  size_t cap_blk1 = 0, cap_blk3 = 0;  // block-map capacity (largest candidate)
  size_t cap_rows = 0;                 // partial rows of 2*NC 8-byte entries (largest candidate)
  // kernel 1 / 2
  ScfLaunchInfo k1{};
  bool k1_ff = false;  // double-precision handles: float-float kernel 1
  bool gen = false;    // radial family of exponent alpha != 1: the general kernels 1 and 3
  ScfConst* d_tab = nullptr;  // their recurrence tables (device memory; allocated for every handle, so that
                              // scf_retune_alpha can move a handle to another exponent)
  float4* d_cs = nullptr;     // [lmax + 1][nmax + 1] single-precision radial steps of kernel 3 (gbeta, hbeta, hratio)
  float* d_tidf = nullptr;    // [n_prog][SCF_HOST_CAP][SCF_TIDAL_W] R-only values of the float tidal difference
  double* d_alpha = nullptr;  // [n_prog][4] exponent search: trial b, S0, S1, mass
  double* d_rc = nullptr;     // [n_prog][16] re-centring state (scf_recentre)
  double* d_sp = nullptr;     // [k3 blocks][kScalePoints + 1] partial sums of the b search
  int k1_blocks = 0;
  int* d_blk1_prog = nullptr;
  int64_t* d_blk1_begin = nullptr;
  int64_t* d_blk1_end = nullptr;
  int* d_prog_blk_off = nullptr;
  // kernel 3 (k3: the kernel of the forward modes; k3_native: the native
  // kernel of the same shape, used by the adjoint's ADJ_J mode)
  ScfLaunchInfo k3{};
  ScfLaunchInfo k3_native{};
  bool k3_ff = false;  // double-precision handles: float-float kernel 3
  int k3_blocks = 0;
  int* d_blk3_prog = nullptr;
  int64_t* d_blk3_begin = nullptr;
  int64_t* d_blk3_end = nullptr;
  // buffers
  double* d_partials = nullptr;
  double* d_A = nullptr;
  void* d_F = nullptr;          // [n_prog][NC] force-coefficient pairs (float2 or double2)
  double* d_aR = nullptr;       // [n_prog][4] a_host(R)
  double* d_norm = nullptr;
  void* d_kscale = nullptr;     // [NC] scale pairs of kernel 3 (element type of the precision)
  double* d_b = nullptr;
  unsigned* d_status = nullptr;
  void* d_base = nullptr;
  ScfHostParams host{};
  // CUDA graph of one scf_step step, keyed by the caller's buffers
  bool graphs = true;
  cudaGraphExec_t step_exec = nullptr;
  const void* step_key[4] = {nullptr, nullptr, nullptr, nullptr};
  bool step_split = false;      // the graph is of a split-state step (scf_step_host, below)
  // scf_step_host on mapped host memory (mixed precision, register-tiled
  // kernel 1): device copies of the drifted positions and the half-kicked
  // velocities, so that kernel 3 reads them from device memory; allocated by
  // the first such call
  void* d_split = nullptr;      // [2][n_total] float4
  // adjoint: per-block tidal partials (double-precision handles only) and
  // the dual kernels' launch shapes (set by the first scf_adjoint_level call)
  double* d_adj_part = nullptr;       // [k3 blocks][SCF_ADJ_Q]
  double* d_en_part = nullptr;        // [k3 blocks][4] energy partials
  // escape physics: particle offsets, pair-sum segments, radius keys, tidal scales
  int64_t* d_off = nullptr;              // [n_prog+1]
  double* d_bpart = nullptr;             // [bound_split][n_total]
  unsigned long long* d_key = nullptr;   // [n_total]
  double* d_tid = nullptr;               // [n_prog][16]
  double* d_half = nullptr;              // [n_prog][4] selection at frac 1/2 (complete refresh)
  int bound_split = 1;
  int64_t bound_chunks = 0;              // pair-kernel i-blocks of the largest progenitor
  const uint8_t* step_mask = nullptr;    // coefficient set of scf_step (scf_set_mask)
  double* d_Atmp = nullptr;              // [n_prog][2*NC] scratch coefficients
  ScfLaunchInfo k1d{}, k3d{};
  bool adj_ready = false;
  // launch timing (scf_profile)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;   // pairs (start, stop)
  std::vector<int> prof_kind;         // kernel index of each recorded pair
  int prof_used = 0;                  // pairs recorded
  // host copies of the block maps (scf_step_host splits the launches at block boundaries)
  std::vector<int64_t> h_blk1_begin, h_blk1_end, h_blk3_begin, h_blk3_end;
  // scf_step_host: copy stream and events, created by its first call
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> stage_ev;
  // the centre's next kick-drift-kick computed beside kernel 3 (SCF_OPT_CENTRE_AHEAD)
  bool centre_ahead = true;
  double* d_cnext = nullptr;             // [n_prog][kCentreW], keys NaN until computed
  float* d_tidnext = nullptr;            // [n_prog][SCF_HOST_CAP][SCF_TIDAL_W] with d_cnext (single precision)
  cudaStream_t side_stream = nullptr;                 // created at the greatest stream priority
  int side_priority = 0;
  cudaEvent_t side_ev[2] = {nullptr, nullptr};
};

namespace {

std::mutex g_const_mutex;
std::vector<bool> g_const_ready;

int upload_tables_once(int device) {
  std::lock_guard<std::mutex> lock(g_const_mutex);
  if ((int)g_const_ready.size() <= device) g_const_ready.resize(device + 1, false);
  if (g_const_ready[device]) return SCF_OK;
  ScfConst* t = new (std::nothrow) ScfConst;
  if (!t) return SCF_ERR_OUT_OF_MEMORY;
  scf_make_const(t);
  cudaError_t e1 = scf_upload_const_coeffs(t);
  cudaError_t e2 = scf_upload_const_forces(t);
  cudaError_t e3 = scf_upload_const_adjoint(t);
  cudaError_t e4 = scf_upload_const_forces_ff(t);
  cudaError_t e5 = scf_upload_const_coeffs_ff(t);
  delete t;
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess || e5 != cudaSuccess)
    return SCF_ERR_CUDA;
  g_const_ready[device] = true;
  return SCF_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Re-centring at complete refreshes (scf_evolve): iteration cap and step tolerance.
constexpr int kRecentreIters = 100;
constexpr double kRecentreTol = 1e-12;

// The general kernels read these entries for l <= lmax, n <= nmax; in single
// precision (f32) the scales and ratios must also stay finite and non-zero.
bool tables_finite(const ScfConst& t, int lmax, int nmax, bool f32) {
  for (int l = 0; l <= lmax; ++l)
    for (int n = 0; n <= nmax; ++n) {
      const double d[4] = {t.gbeta[l][n], t.hbeta[l][n], t.gscale[l][n], t.hscale[l][n]};
      const float f[5] = {t.gbetaf[l][n], t.hbetaf[l][n], t.gscalef[l][n], t.hscalef[l][n], t.hratiof[l][n]};
      for (double x : d)
        if (!std::isfinite(x)) return false;
      if (!f32) continue;
      for (float x : f)
        if (!std::isfinite(x)) return false;
      if (t.gscalef[l][n] == 0.f || t.hscalef[l][n] == 0.f) return false;
    }
  return true;
}

void drop_graph(scf_handle* h) {
  if (h->step_exec) cudaGraphExecDestroy(h->step_exec);
  h->step_exec = nullptr;
  for (auto& k : h->step_key) k = nullptr;
  h->step_split = false;
}

size_t round_up(size_t x) { return (x + 255) & ~size_t(255); }

int check_config(const scf_config* c) {
  if (c->nmax < 0 || c->lmax < 0 || c->n_host < 0 || c->n_host > SCF_MAX_HOST_COMPONENTS) return SCF_ERR_INVALID_ARG;
  if (c->nmax > SCF_MAX_NMAX || c->lmax > SCF_MAX_LMAX) return SCF_ERR_UNSUPPORTED;
  if (!(c->alpha > 0.0) || !std::isfinite(c->alpha)) return SCF_ERR_INVALID_ARG;
  if (c->alpha < SCF_ALPHA_MIN || c->alpha > SCF_ALPHA_MAX) return SCF_ERR_UNSUPPORTED;
  if (c->precision != SCF_FP64 && c->precision != SCF_MIXED) return SCF_ERR_INVALID_ARG;
  if (!std::isfinite(c->G) || !std::isfinite(c->dt) || !std::isfinite(c->b)) return SCF_ERR_INVALID_ARG;
  for (int i = 0; i < c->n_host; ++i) {
    const scf_host_component& h = c->host[i];
    if (h.kind != SCF_HOST_HERNQUIST && h.kind != SCF_HOST_NFW && h.kind != SCF_HOST_MN && h.kind != SCF_HOST_POWCUT)
      return SCF_ERR_INVALID_ARG;
    if (!(h.a > 0.0) || !std::isfinite(h.M) || !std::isfinite(h.a)) return SCF_ERR_INVALID_ARG;
    if (h.kind == SCF_HOST_MN && !(h.b >= 0.0 && std::isfinite(h.b))) return SCF_ERR_INVALID_ARG;
    if (h.kind == SCF_HOST_POWCUT && !(h.b >= 0.0 && h.b < 2.0)) return SCF_ERR_INVALID_ARG;
  }
  return SCF_OK;
}

int cuda_fail(cudaError_t e) { return e == cudaSuccess ? SCF_OK : SCF_ERR_CUDA; }

constexpr int kProfPairs = 4096;

// Runs `launch` and, when profiling, brackets it with a recorded event pair.
template <typename F>
cudaError_t timed(scf_handle* h, int kind, F&& launch) {
  const bool rec = h->prof_on && h->prof_used < kProfPairs;
  if (rec) cudaEventRecord(h->prof_ev[2 * h->prof_used], h->stream);
  cudaError_t e = launch();
  if (rec) {
    cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], h->stream);
    h->prof_kind[h->prof_used++] = kind;
  }
  return e;
}

void prof_release(scf_handle* h) {
  for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
  h->prof_ev.clear();
  h->prof_kind.clear();
  h->prof_used = 0;
  h->prof_on = false;
}

K1Args k1_args(scf_handle* h, void* pos, void* vel, const void* acc, const uint8_t* mask, int mode) {
  K1Args a{};
  a.pos = pos;
  a.vel = vel;
  a.acc = acc;
  a.mask = mask;
  a.partials = h->d_partials;
  a.blk_prog = h->d_blk1_prog;
  a.blk_begin = h->d_blk1_begin;
  a.blk_end = h->d_blk1_end;
  a.b_prog = h->d_b;
  a.nmax = h->cfg.nmax;
  a.lmax = h->cfg.lmax;
  a.nc = h->nc;
  a.nlm = h->nlm;
  a.mode = mode;
  a.dt = h->cfg.dt;
  a.status = h->d_status;
  a.tab = h->gen ? h->d_tab : nullptr;
  a.alpha = h->cfg.alpha;
  a.inv_alpha = 1.0 / h->cfg.alpha;
  return a;
}

K2Args k2_args(scf_handle* h, double* A_out, double* com, int mode) {
  K2Args a{};
  a.nlm = h->nlm;
  a.F_out = h->d_F;
  a.f32 = h->cfg.precision == SCF_MIXED;
  a.kscale_f = static_cast<const float*>(h->d_kscale);
  a.tid_out = a.f32 ? h->d_tidf : nullptr;
  a.b_prog = h->d_b;
  a.G = h->cfg.G;
  a.aR_out = h->d_aR;
  a.partials = h->d_partials;
  a.prog_blk_off = h->d_prog_blk_off;
  a.norm = h->d_norm;
  a.A_out = A_out;
  a.nc = h->nc;
  a.n_prog = h->n_prog;
  a.mode = mode;
  a.dt = h->cfg.dt;
  a.com = com;
  a.host = h->host;
  a.sub = h->k1.variant == 1 ? h->k1.win : 0;  // register-tiled kernel 1: float rows, one per window
  a.cnext = mode == SCF_MODE_STEP && h->centre_ahead ? h->d_cnext : nullptr;
  a.tid_next = a.cnext && a.f32 ? h->d_tidnext : nullptr;
  return a;
}

K3Args k3_args(scf_handle* h, const void* pos, void* vel, void* acc, const double* com, int mode) {
  K3Args a{};
  a.pos = pos;
  a.vel = vel;
  a.acc = acc;
  a.F = h->d_F;
  a.aR = h->d_aR;
  a.kscale = h->d_kscale;
  a.com = com;
  a.blk_prog = h->d_blk3_prog;
  a.blk_begin = h->d_blk3_begin;
  a.blk_end = h->d_blk3_end;
  a.b_prog = h->d_b;
  a.nmax = h->cfg.nmax;
  a.lmax = h->cfg.lmax;
  a.nc = h->nc;
  a.nlm = h->nlm;
  a.mode = mode;
  a.G = h->cfg.G;
  a.dt = h->cfg.dt;
  a.host = h->host;
  a.status = h->d_status;
  a.tab = h->gen ? h->d_tab : nullptr;
  a.alpha = h->cfg.alpha;
  a.inv_alpha = 1.0 / h->cfg.alpha;
  a.cs = h->d_cs;
  a.tid = h->d_tidf;
  return a;
}

int run_coeffs(scf_handle* h, void* pos, void* vel, const void* acc, const uint8_t* mask, double* A_out, double* com,
               int mode, void* pos_copy = nullptr, void* vel_out = nullptr) {
  if (h->k1_blocks > 0) {
    K1Args a = k1_args(h, pos, vel, acc, mask, mode);
    a.pos_copy = pos_copy;
    a.vel_out = vel_out;
    if (timed(h, 0, [&] {
          return h->k1.variant == 2 ? scf_k1_ff_launch(a, h->k1_blocks, h->k1, h->stream)
                                    : scf_k1_launch(h->cfg.precision, a, h->k1_blocks, h->k1, h->stream);
        }) != cudaSuccess)
      return SCF_ERR_CUDA;
  }
  K2Args b = k2_args(h, A_out, com, mode);
  return cuda_fail(timed(h, 1, [&] { return scf_k2_launch(b, h->stream); }));
}

// Force coefficients F and a_host(R) from caller-supplied coefficients.
int run_prep(scf_handle* h, const double* A, const double* com) {
  PrepArgs p{};
  p.A = A;
  p.com = com;
  p.F_out = h->d_F;
  p.f32 = h->cfg.precision == SCF_MIXED;
  p.kscale_f = static_cast<const float*>(h->d_kscale);
  p.tid_out = p.f32 ? h->d_tidf : nullptr;
  p.b_prog = h->d_b;
  p.G = h->cfg.G;
  p.aR_out = h->d_aR;
  p.nc = h->nc;
  p.nlm = h->nlm;
  p.n_prog = h->n_prog;
  p.host = h->host;
  return cuda_fail(timed(h, 1, [&] { return scf_prep_launch(p, h->stream); }));
}

// Kernel 3 on the handle's F / a_host(R) (from kernel 2 or run_prep).
int run_forces(scf_handle* h, const void* pos, void* vel, void* acc, const double* com, int mode,
               const void* vel_in = nullptr) {
  if (h->k3_blocks == 0) return SCF_OK;
  K3Args a = k3_args(h, pos, vel, acc, com, mode);
  a.vel_in = vel_in;
  if (h->k3.variant == 2 && mode != SCF_MODE_ADJ_J)
    return cuda_fail(timed(h, 2, [&] { return scf_k3_ff_launch(a, h->k3_blocks, h->k3, h->stream); }));
  return cuda_fail(
      timed(h, 2, [&] { return scf_k3_launch(h->cfg.precision, a, h->k3_blocks, h->k3_native, h->stream); }));
}

// Kernel 1 block map: contiguous ranges of whole tiles, one progenitor per
// block, about one wave of resident blocks in total.
struct Map1 {
  std::vector<int> prog, prog_off;
  std::vector<int64_t> begin, end;
};
Map1 make_map1(const std::vector<int64_t>& off, int n_prog, int64_t tp, int64_t slots) {
  Map1 m;
  m.prog_off.assign(n_prog + 1, 0);
  std::vector<int64_t> tiles(n_prog), nb(n_prog, 0);
  int64_t used = 0;
  for (int p = 0; p < n_prog; ++p) {
    tiles[p] = (off[p + 1] - off[p] + tp - 1) / tp;
    nb[p] = tiles[p] > 0 ? 1 : 0;
    used += nb[p];
  }
  // Blocks per progenitor: one each, then every further block to the
  // progenitor whose blocks are the longest, while the blocks fit in one wave
  // (slots).  The longest block sets the kernel's time, and a block beyond
  // the wave would run after the others: so at most `slots` blocks, with the
  // smallest longest block.
  auto longest = [&](int p) { return nb[p] > 0 ? (tiles[p] + nb[p] - 1) / nb[p] : 0; };
  std::priority_queue<std::pair<int64_t, int>> q;
  for (int p = 0; p < n_prog; ++p)
    if (nb[p] > 0) q.push({longest(p), p});
  while (used < slots && !q.empty()) {
    const int p = q.top().second;
    q.pop();
    if (longest(p) <= 1) break;
    ++nb[p];
    ++used;
    q.push({longest(p), p});
  }
  // each progenitor's tiles split into nb[p] contiguous runs as even as possible
  for (int p = 0; p < n_prog; ++p) {
    m.prog_off[p] = (int)m.prog.size();
    int64_t t0 = 0;
    for (int64_t b = 0; b < nb[p]; ++b) {
      const int64_t t1 = tiles[p] * (b + 1) / nb[p];
      m.prog.push_back(p);
      m.begin.push_back(off[p] + t0 * tp);
      m.end.push_back(std::min(off[p] + t1 * tp, off[p + 1]));
      t0 = t1;
    }
  }
  m.prog_off[n_prog] = (int)m.prog.size();
  return m;
}

// Kernel 3 block map: one thread per particle, one progenitor per block.
struct Map3 {
  std::vector<int> prog;
  std::vector<int64_t> begin, end;
};
Map3 make_map3(const std::vector<int64_t>& off, int n_prog, int64_t tb) {
  Map3 m;
  for (int p = 0; p < n_prog; ++p)
    for (int64_t k = off[p]; k < off[p + 1]; k += tb) {
      m.prog.push_back(p);
      m.begin.push_back(k);
      m.end.push_back(std::min(k + tb, off[p + 1]));
    }
  return m;
}

bool put(void* dst, const void* src, size_t bytes) {
  return bytes == 0 || cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
}

// Kernel 3's single-precision radial steps of the family in t, one float4
// (gbeta, hbeta, hratio, 0) per (l, n): staged by every block with coalesced
// 16-byte loads.
bool put_steps(scf_handle* h, const ScfConst& t) {
  const int nn = h->cfg.nmax + 1;
  std::vector<float4> cs((size_t)(h->cfg.lmax + 1) * nn);
  for (int l = 0; l <= h->cfg.lmax; ++l)
    for (int n = 0; n < nn; ++n)
      cs[(size_t)l * nn + n] = make_float4(t.gbetaf[l][n], t.hbetaf[l][n], t.hratiof[l][n], 0.f);
  return put(h->d_cs, cs.data(), sizeof(float4) * cs.size());
}

// Kernel 1 launch shape: the simple kernel with a particle tile of 64, 128
// or 256 (tp), or the register-tiled single-precision kernel (tp = 0).  For a
// radial family of exponent alpha != 1: the general simple kernel with
// 128-particle tiles, or (mixed precision) the register-tiled kernel's
// runtime-indexed basis.
int k1_shape(const scf_config& cfg, int tp, bool ff, ScfLaunchInfo* info, int* bps) {
  if (cfg.alpha != 1.0) {
    if ((tp != 128 && tp != 0) || ff) return SCF_ERR_UNSUPPORTED;
    const cudaError_t e = tp == 0 ? scf_k1_tiled_prepare(cfg.lmax, cfg.nmax, info, bps, true)
                                  : scf_k1_gen_prepare(cfg.precision, cfg.lmax, cfg.nmax, info, bps);
    if (e != cudaSuccess || *bps < 1) {
      cudaGetLastError();
      return SCF_ERR_UNSUPPORTED;
    }
    return SCF_OK;
  }
  cudaError_t e = tp == 0 ? scf_k1_tiled_prepare(cfg.lmax, cfg.nmax, info, bps)
                  : ff    ? scf_k1_ff_prepare(cfg.lmax, cfg.nmax, tp, info, bps)
                          : scf_k1_prepare(cfg.precision, cfg.lmax, cfg.nmax, tp, info, bps);
  if (e != cudaSuccess || *bps < 1) {
    cudaGetLastError();
    return SCF_ERR_UNSUPPORTED;
  }
  return SCF_OK;
}

// Partial rows in units of 2*NC doubles: one per block, or for the
// register-tiled kernel win float rows per block (two per double row).
size_t k1_rows(const ScfLaunchInfo& info, size_t blocks) {
  return info.variant == 1 ? (blocks * info.win + 1) / 2 : blocks;
}

int64_t longest_block(const Map1& m) {
  int64_t n = 0;
  for (size_t b = 0; b < m.prog.size(); ++b) n = std::max(n, m.end[b] - m.begin[b]);
  return n;
}

// Selects kernel 1's shape: launch info, block map, upload.
int use_k1(scf_handle* h, int tp) {
  if (tp == 0 && h->cfg.precision != SCF_MIXED) return SCF_ERR_UNSUPPORTED;
  ScfLaunchInfo info{};
  int bps = 0;
  if (k1_shape(h->cfg, tp, h->k1_ff && tp != 0, &info, &bps) != SCF_OK) return SCF_ERR_UNSUPPORTED;
  Map1 m = make_map1(h->offsets, h->n_prog, info.tile, (int64_t)h->n_sm * bps);
  if (info.variant == 1) info.win = scf_k1_windows(longest_block(m), info);
  if (m.prog.size() > h->cap_blk1 || k1_rows(info, m.prog.size()) > h->cap_rows) return SCF_ERR_UNSUPPORTED;
  bool ok = put(h->d_blk1_prog, m.prog.data(), sizeof(int) * m.prog.size()) &&
            put(h->d_blk1_begin, m.begin.data(), sizeof(int64_t) * m.begin.size()) &&
            put(h->d_blk1_end, m.end.data(), sizeof(int64_t) * m.end.size()) &&
            put(h->d_prog_blk_off, m.prog_off.data(), sizeof(int) * m.prog_off.size());
  if (!ok) return SCF_ERR_CUDA;
  h->k1 = info;
  h->k1_blocks = (int)m.prog.size();
  h->h_blk1_begin = m.begin;
  h->h_blk1_end = m.end;
  drop_graph(h);
  return SCF_OK;
}

// Selects kernel 3's block size: launch info, block map, upload.
int use_k3(scf_handle* h, int tb) {
  ScfLaunchInfo native{}, info{};
  int bps = 0;
  if (h->gen && (tb != 128 || h->k3_ff)) return SCF_ERR_UNSUPPORTED;  // general kernel: 128 threads
  if ((h->gen ? scf_k3_gen_prepare(h->cfg.precision, h->cfg.lmax, h->cfg.nmax, &native, &bps)
              : scf_k3_prepare(h->cfg.precision, h->cfg.lmax, h->cfg.nmax, tb, &native, &bps)) != cudaSuccess ||
      bps < 1) {
    cudaGetLastError();
    return SCF_ERR_UNSUPPORTED;
  }
  info = native;
  if (h->k3_ff && (scf_k3_ff_prepare(h->cfg.lmax, h->cfg.nmax, tb, &info, &bps) != cudaSuccess || bps < 1 ||
                   info.tile != native.tile)) {
    cudaGetLastError();
    return SCF_ERR_UNSUPPORTED;
  }
  Map3 m = make_map3(h->offsets, h->n_prog, info.tile);
  if (m.prog.size() > h->cap_blk3) return SCF_ERR_UNSUPPORTED;
  bool ok = put(h->d_blk3_prog, m.prog.data(), sizeof(int) * m.prog.size()) &&
            put(h->d_blk3_begin, m.begin.data(), sizeof(int64_t) * m.begin.size()) &&
            put(h->d_blk3_end, m.end.data(), sizeof(int64_t) * m.end.size());
  if (!ok) return SCF_ERR_CUDA;
  h->k3 = info;
  h->k3_native = native;
  h->k3_blocks = (int)m.prog.size();
  h->h_blk3_begin = m.begin;
  h->h_blk3_end = m.end;
  drop_graph(h);
  return SCF_OK;
}

}  // namespace

extern "C" {

int scf_init(const scf_config* cfg, int n_prog, const int64_t* offsets, const double* b_per_prog, void* stream,
             scf_handle** out) {
  if (!cfg || !offsets || !out) return SCF_ERR_NULL_POINTER;
  int rc = check_config(cfg);
  if (rc != SCF_OK) return rc;
  if (n_prog < 1 || offsets[0] != 0) return SCF_ERR_INVALID_ARG;
  for (int p = 0; p < n_prog; ++p)
    if (offsets[p + 1] < offsets[p]) return SCF_ERR_INVALID_ARG;
  std::vector<double> bs(n_prog);
  for (int p = 0; p < n_prog; ++p) {
    bs[p] = b_per_prog ? b_per_prog[p] : cfg->b;
    if (!(bs[p] > 0.0) || !std::isfinite(bs[p])) return SCF_ERR_INVALID_ARG;
  }

  scf_handle* h = new (std::nothrow) scf_handle;
  if (!h) return SCF_ERR_OUT_OF_MEMORY;
  h->cfg = *cfg;
  h->n_prog = n_prog;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->nlm = (cfg->lmax + 1) * (cfg->lmax + 2) / 2;
  h->nc = (cfg->nmax + 1) * h->nlm;
  h->n_total = offsets[n_prog];
  h->host.n = cfg->n_host;
  for (int i = 0; i < cfg->n_host; ++i) {
    h->host.kind[i] = cfg->host[i].kind;
    h->host.GM[i] = cfg->G * cfg->host[i].M;
    h->host.a[i] = cfg->host[i].a;
    h->host.b[i] = cfg->host[i].b;
  }
  auto fail = [&](int code) {
    if (h->d_base) cudaFree(h->d_base);
    delete h;
    return code;
  };
  h->gen = cfg->alpha != 1.0;
  if (cudaGetDevice(&h->device) != cudaSuccess) return fail(SCF_ERR_CUDA);
  rc = upload_tables_once(h->device);
  if (rc != SCF_OK) return fail(rc);
  if (cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
    return fail(SCF_ERR_CUDA);
  h->offsets.assign(offsets, offsets + n_prog + 1);

  // Capacity of the block maps and partial rows: the largest any candidate shape can need.
  // Both radial families count (alpha = 1 and the general kernels), since
  // scf_retune_alpha can move the handle from one to the other.
  for (int cand = 0; cand < 10; ++cand) {
    const int c5 = cand % 5;
    const int tp = c5 < 3 ? 64 << c5 : c5 == 3 ? 0 : 128;  // the last: float-float, 128
    const bool ff = c5 == 4;
    if (tp == 0 && cfg->precision != SCF_MIXED) continue;
    if (ff && cfg->precision != SCF_FP64) continue;
    scf_config cc = *cfg;
    cc.alpha = cand < 5 ? 1.0 : 0.5;
    ScfLaunchInfo info{};
    int bps = 0;
    if (k1_shape(cc, tp, ff, &info, &bps) != SCF_OK) continue;
    const Map1 m = make_map1(h->offsets, n_prog, info.tile, (int64_t)h->n_sm * bps);
    const size_t blocks = m.prog.size();
    if (info.variant == 1) info.win = scf_k1_windows(longest_block(m), info);
    h->cap_blk1 = std::max(h->cap_blk1, blocks);
    h->cap_rows = std::max(h->cap_rows, k1_rows(info, blocks));
  }
  h->cap_blk3 = make_map3(h->offsets, n_prog, 32).prog.size();  // smallest kernel 3 tile (64 threads, split)
  if (h->cap_blk1 == 0 && h->n_total > 0) return fail(SCF_ERR_UNSUPPORTED);

  // one allocation for the whole workspace
  const size_t nb1 = std::max<size_t>(1, h->cap_blk1), nb3 = std::max<size_t>(1, h->cap_blk3);
  const size_t nrows = std::max<size_t>(1, h->cap_rows);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += round_up(bytes);
    return o;
  };
  const size_t o_part = take(sizeof(double) * 2 * (size_t)h->nc * nrows);
  const size_t o_A = take(sizeof(double) * 2 * (size_t)h->nc * n_prog);
  const size_t o_F = take(sizeof(double) * 2 * (size_t)h->nc * n_prog);
  const size_t o_aR = take(sizeof(double) * 4 * (size_t)n_prog);
  const size_t o_norm = take(sizeof(double) * 2 * (size_t)h->nc);
  const size_t o_ksc = take(sizeof(double) * 2 * (size_t)h->nc);
  const size_t o_b = take(sizeof(double) * n_prog);
  const size_t o_b1p = take(sizeof(int) * nb1);
  const size_t o_b1b = take(sizeof(int64_t) * nb1);
  const size_t o_b1e = take(sizeof(int64_t) * nb1);
  const size_t o_pbo = take(sizeof(int) * (n_prog + 1));
  const size_t o_b3p = take(sizeof(int) * nb3);
  const size_t o_b3b = take(sizeof(int64_t) * nb3);
  const size_t o_b3e = take(sizeof(int64_t) * nb3);
  const size_t o_st = take(sizeof(unsigned) * 4);
  const size_t o_en = take(sizeof(double) * 4 * nb3);
  const size_t o_adj = cfg->precision == SCF_FP64 ? take(sizeof(double) * SCF_ADJ_Q * nb3) : off;
  {
    const int64_t chunk = scf_bound_chunk(cfg->precision == SCF_MIXED);
    int64_t chunks = 0;
    for (int p = 0; p < n_prog; ++p) {
      const int64_t c = (h->offsets[p + 1] - h->offsets[p] + chunk - 1) / chunk;
      chunks += c;
      h->bound_chunks = std::max(h->bound_chunks, c);
    }
    h->bound_split = scf_bound_split(chunks, h->n_sm);
  }
  const size_t o_off = take(sizeof(int64_t) * (n_prog + 1));
  const size_t o_bpart = take(sizeof(double) * (size_t)h->bound_split * (size_t)h->n_total);
  const size_t o_key = take(sizeof(unsigned long long) * (size_t)h->n_total);
  const size_t o_tid = take(sizeof(double) * 16 * (size_t)n_prog);
  const size_t o_half = take(sizeof(double) * 4 * (size_t)n_prog);
  const size_t o_Atmp = take(sizeof(double) * 2 * (size_t)h->nc * n_prog);
  const size_t o_tab = take(sizeof(ScfConst));
  const size_t o_alpha = take(sizeof(double) * 4 * (size_t)n_prog);
  const size_t o_rc = take(sizeof(double) * 16 * (size_t)n_prog);
  const size_t o_sp = take(sizeof(double) * (kScalePoints + 1) * nb3);
  const size_t o_cn = take(sizeof(double) * kCentreW * (size_t)n_prog);
  const size_t o_cs = take(sizeof(float4) * (size_t)(cfg->lmax + 1) * (cfg->nmax + 1));
  const size_t o_tidf = take(sizeof(float) * SCF_HOST_CAP * SCF_TIDAL_W * (size_t)n_prog);
  const size_t o_tidn = take(sizeof(float) * SCF_HOST_CAP * SCF_TIDAL_W * (size_t)n_prog);
  if (cudaMalloc(&h->d_base, off) != cudaSuccess) {
    cudaGetLastError();
    return fail(SCF_ERR_OUT_OF_MEMORY);
  }
  char* base = static_cast<char*>(h->d_base);
  h->d_partials = reinterpret_cast<double*>(base + o_part);
  h->d_A = reinterpret_cast<double*>(base + o_A);
  h->d_F = reinterpret_cast<void*>(base + o_F);
  h->d_aR = reinterpret_cast<double*>(base + o_aR);
  h->d_norm = reinterpret_cast<double*>(base + o_norm);
  h->d_kscale = reinterpret_cast<void*>(base + o_ksc);
  h->d_b = reinterpret_cast<double*>(base + o_b);
  h->d_blk1_prog = reinterpret_cast<int*>(base + o_b1p);
  h->d_blk1_begin = reinterpret_cast<int64_t*>(base + o_b1b);
  h->d_blk1_end = reinterpret_cast<int64_t*>(base + o_b1e);
  h->d_prog_blk_off = reinterpret_cast<int*>(base + o_pbo);
  h->d_blk3_prog = reinterpret_cast<int*>(base + o_b3p);
  h->d_blk3_begin = reinterpret_cast<int64_t*>(base + o_b3b);
  h->d_blk3_end = reinterpret_cast<int64_t*>(base + o_b3e);
  h->d_status = reinterpret_cast<unsigned*>(base + o_st);
  h->d_en_part = reinterpret_cast<double*>(base + o_en);
  if (cfg->precision == SCF_FP64) h->d_adj_part = reinterpret_cast<double*>(base + o_adj);
  h->d_off = reinterpret_cast<int64_t*>(base + o_off);
  h->d_bpart = reinterpret_cast<double*>(base + o_bpart);
  h->d_key = reinterpret_cast<unsigned long long*>(base + o_key);
  h->d_tid = reinterpret_cast<double*>(base + o_tid);
  h->d_half = reinterpret_cast<double*>(base + o_half);
  h->d_Atmp = reinterpret_cast<double*>(base + o_Atmp);
  h->d_rc = reinterpret_cast<double*>(base + o_rc);
  h->d_sp = reinterpret_cast<double*>(base + o_sp);
  h->d_cnext = reinterpret_cast<double*>(base + o_cn);
  h->d_cs = reinterpret_cast<float4*>(base + o_cs);
  h->d_tidf = reinterpret_cast<float*>(base + o_tidf);
  h->d_tidnext = reinterpret_cast<float*>(base + o_tidn);

  h->d_tab = reinterpret_cast<ScfConst*>(base + o_tab);
  h->d_alpha = reinterpret_cast<double*>(base + o_alpha);
  {  // recurrence tables of the handle's radial family
    std::unique_ptr<ScfConst> t(new (std::nothrow) ScfConst);
    if (!t) return fail(SCF_ERR_OUT_OF_MEMORY);
    scf_make_const(t.get(), cfg->alpha);
    if (h->gen && !tables_finite(*t, cfg->lmax, cfg->nmax, cfg->precision == SCF_MIXED))
      return fail(SCF_ERR_UNSUPPORTED);
    if (h->gen && !put(h->d_tab, t.get(), sizeof(ScfConst))) return fail(SCF_ERR_CUDA);
    if (!put_steps(h, *t)) return fail(SCF_ERR_CUDA);
  }
  std::vector<double> norm(2 * (size_t)h->nc), ksc(2 * (size_t)h->nc);
  scf_make_norm(cfg->nmax, cfg->lmax, norm.data(), cfg->alpha);
  scf_make_kscale(cfg->nmax, cfg->lmax, ksc.data(), cfg->alpha);
  for (double x : norm)
    if (!std::isfinite(x)) return fail(SCF_ERR_UNSUPPORTED);
  std::vector<float> ksc_f(ksc.begin(), ksc.end());
  const bool ksc_ok = cfg->precision == SCF_MIXED ? put(h->d_kscale, ksc_f.data(), sizeof(float) * ksc_f.size())
                                                  : put(h->d_kscale, ksc.data(), sizeof(double) * ksc.size());
  bool ok = ksc_ok && put(h->d_norm, norm.data(), sizeof(double) * norm.size()) &&
            put(h->d_b, bs.data(), sizeof(double) * n_prog) &&
            put(h->d_off, h->offsets.data(), sizeof(int64_t) * (n_prog + 1)) &&
            cudaMemset(h->d_status, 0, sizeof(unsigned) * 4) == cudaSuccess &&
            cudaMemset(h->d_cnext, 0xff, sizeof(double) * kCentreW * (size_t)n_prog) == cudaSuccess &&  // NaN keys
            cudaMemset(h->d_A, 0, sizeof(double) * 2 * (size_t)h->nc * n_prog) == cudaSuccess;
  if (!ok) return fail(SCF_ERR_CUDA);
  // default shapes: the register-tiled kernel 1 in mixed precision (128-particle
  // tiles of the simple kernel in double precision) and 128-thread kernel 3
  // blocks; scf_autotune may change them
  rc = cfg->precision == SCF_MIXED ? use_k1(h, 0) : SCF_ERR_UNSUPPORTED;
  if (rc != SCF_OK) rc = use_k1(h, 128);
  if (rc != SCF_OK) return fail(rc);
  rc = use_k3(h, 128);
  if (rc != SCF_OK) return fail(rc);
  *out = h;
  return SCF_OK;
}

int scf_coeffs(scf_handle* h, const void* pos, const uint8_t* mask, double* A_out) {
  if (!h || !A_out || (!pos && h->n_total > 0)) return SCF_ERR_NULL_POINTER;
  if (!aligned16(pos)) return SCF_ERR_MISALIGNED;
  return run_coeffs(h, const_cast<void*>(pos), nullptr, nullptr, mask, A_out, nullptr, SCF_MODE_COEFFS);
}

int scf_forces(scf_handle* h, const void* pos, const double* A, const double* com, void* acc) {
  if (!h || !A || ((!pos || !acc) && h->n_total > 0)) return SCF_ERR_NULL_POINTER;
  if (h->host.n > 0 && !com) return SCF_ERR_NULL_POINTER;
  if (!aligned16(pos) || !aligned16(acc)) return SCF_ERR_MISALIGNED;
  int rc = run_prep(h, A, com);
  if (rc != SCF_OK) return rc;
  return run_forces(h, pos, nullptr, acc, com, SCF_MODE_COEFFS);
}

namespace {

// One step.  split (scf_step_host on mapped host memory): kernel 1 also
// writes the drifted positions to the device copy and the half-kicked
// velocities only there, and kernel 3 reads both from it, so the host link
// carries the state in once and out once.
int launch_step(scf_handle* h, void* pos, void* vel, void* acc, double* com, bool split = false) {
  void* spos = split ? h->d_split : nullptr;
  void* svel = split ? static_cast<char*>(h->d_split) + 16 * (size_t)h->n_total : nullptr;
  int rc = run_coeffs(h, pos, vel, acc, h->step_mask, h->d_A, com, SCF_MODE_STEP, spos, svel);
  if (rc != SCF_OK) return rc;
  // the next step's centre kick-drift-kick, on a second stream beside kernel 3
  // (its FP64 dependency chain then leaves kernel 2's critical path); joined
  // back before the step ends
  const bool ahead = h->centre_ahead && h->host.n > 0 && com != nullptr;
  if (ahead) {
    if (!h->side_stream) {
      int least = 0, greatest = 0;
      if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return SCF_ERR_CUDA;
      h->side_priority = greatest;
      if (cudaStreamCreateWithPriority(&h->side_stream, cudaStreamNonBlocking, greatest) != cudaSuccess) {
        h->side_stream = nullptr;
        return SCF_ERR_CUDA;
      }
      for (cudaEvent_t& e : h->side_ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return SCF_ERR_CUDA;
    }
    CentreArgs c{};
    c.com = com;
    c.aR = h->d_aR;
    c.cnext = h->d_cnext;
    c.tid_next = h->cfg.precision == SCF_MIXED ? h->d_tidnext : nullptr;
    c.dt = h->cfg.dt;
    c.n_prog = h->n_prog;
    c.host = h->host;
    if (cudaEventRecord(h->side_ev[0], h->stream) != cudaSuccess ||
        cudaStreamWaitEvent(h->side_stream, h->side_ev[0], 0) != cudaSuccess ||
        scf_centre_next_launch(c, h->side_priority, h->side_stream) != cudaSuccess ||
        cudaEventRecord(h->side_ev[1], h->side_stream) != cudaSuccess)
      return SCF_ERR_CUDA;
  }
  rc = split ? run_forces(h, spos, vel, acc, com, SCF_MODE_STEP, svel) : run_forces(h, pos, vel, acc, com, SCF_MODE_STEP);
  if (ahead && cudaStreamWaitEvent(h->stream, h->side_ev[1], 0) != cudaSuccess) return SCF_ERR_CUDA;
  return rc;
}

// Captures one step on the handle's stream into an executable graph.  Returns
// false (and leaves the handle without a graph) when the stream cannot be
// captured, e.g. the legacy default stream.
bool capture_step(scf_handle* h, void* pos, void* vel, void* acc, double* com, bool split) {
  drop_graph(h);
  if (h->stream == nullptr || h->stream == cudaStreamLegacy) return false;
  if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int rc = launch_step(h, pos, vel, acc, com, split);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  bool ok = rc == SCF_OK && e == cudaSuccess && g != nullptr &&
            cudaGraphInstantiate(&h->step_exec, g, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    h->step_exec = nullptr;
    return false;
  }
  h->step_key[0] = pos;
  h->step_key[1] = vel;
  h->step_key[2] = acc;
  h->step_key[3] = com;
  h->step_split = split;
  return true;
}

int step_impl(scf_handle* h, void* pos, void* vel, void* acc, double* com, int nsteps, bool split) {
  // one graph launch per step when the stream can be captured (the kernels
  // and their arguments are the same every step); plain launches otherwise
  if (h->graphs && !h->prof_on) {
    const bool same = h->step_exec && h->step_key[0] == pos && h->step_key[1] == vel && h->step_key[2] == acc &&
                      h->step_key[3] == com && h->step_split == split;
    if (same || capture_step(h, pos, vel, acc, com, split)) {
      for (int st = 0; st < nsteps; ++st)
        if (cudaGraphLaunch(h->step_exec, h->stream) != cudaSuccess) return SCF_ERR_CUDA;
      return SCF_OK;
    }
  }
  for (int st = 0; st < nsteps; ++st) {
    const int rc = launch_step(h, pos, vel, acc, com, split);
    if (rc != SCF_OK) return rc;
  }
  return SCF_OK;
}

}  // namespace

int scf_step(scf_handle* h, void* pos, void* vel, void* acc, double* com, int nsteps) {
  if (!h) return SCF_ERR_NULL_POINTER;
  if (nsteps < 0) return SCF_ERR_INVALID_ARG;
  if ((!pos || !vel || !acc) && h->n_total > 0) return SCF_ERR_NULL_POINTER;
  if (h->host.n > 0 && !com) return SCF_ERR_NULL_POINTER;
  if (!aligned16(pos) || !aligned16(vel) || !aligned16(acc)) return SCF_ERR_MISALIGNED;
  if (nsteps == 0) return SCF_OK;
  return step_impl(h, pos, vel, acc, com, nsteps, false);
}

namespace {

// Chunk c of `chunks` equal block ranges of a map with `blocks` blocks.
void block_range(int blocks, int chunks, int c, int* b0, int* b1) {
  *b0 = (int)((int64_t)blocks * c / chunks);
  *b1 = (int)((int64_t)blocks * (c + 1) / chunks);
}

}  // namespace

int scf_step_host(scf_handle* h, void* pos, void* vel, void* acc, double* com, void* host_pos, void* host_vel,
                  void* host_acc, double* host_com, int chunks) {
  if (!h) return SCF_ERR_NULL_POINTER;
  if (chunks < 1 || chunks > SCF_STAGE_MAX_CHUNKS) return SCF_ERR_INVALID_ARG;
  if ((!host_pos || !host_vel || !host_acc) && h->n_total > 0) return SCF_ERR_NULL_POINTER;
  const bool with_com = h->host.n > 0;
  if (with_com && !host_com) return SCF_ERR_NULL_POINTER;
  // Mapped page-locked host memory: the step's kernels read and write the
  // host arrays in place over the host link, so the transfers run inside
  // the kernels, overlapped with their arithmetic (the usual case with
  // cudaHostAlloc / torch pin_memory under unified addressing).
  void* hp[4] = {host_pos, host_vel, host_acc, host_com};
  void* mp[4] = {nullptr, nullptr, nullptr, nullptr};
  bool mapped = true;
  for (int i = 0; i < 4 && mapped; ++i) {
    if (!hp[i]) continue;
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, hp[i]) != cudaSuccess) {
      cudaGetLastError();
      mapped = false;
    } else if (attr.type == cudaMemoryTypeHost && attr.devicePointer != nullptr) {
      mp[i] = attr.devicePointer;
    } else {
      mapped = false;
    }
  }
  if (mapped && aligned16(mp[0]) && aligned16(mp[1]) && aligned16(mp[2])) {
    // mixed precision with the register-tiled kernel 1 and the native kernel
    // 3: the intermediate state stays on the device (launch_step, split)
    const bool split = h->cfg.precision == SCF_MIXED && h->k1.variant == 1 && h->k3.variant != 2 &&
                       h->n_total > 0;
    if (split && !h->d_split) {
      if (cudaMalloc(&h->d_split, 2 * 16 * (size_t)h->n_total) != cudaSuccess) {
        cudaGetLastError();
        h->d_split = nullptr;
        return SCF_ERR_OUT_OF_MEMORY;
      }
    }
    if (h->host.n > 0 && !mp[3]) return SCF_ERR_NULL_POINTER;
    return step_impl(h, mp[0], mp[1], mp[2], static_cast<double*>(mp[3]), 1, split);
  }

  // Otherwise the state is staged through the device arrays: copied in, kernel
  // 1 and 2, and copied back while kernel 3 still runs -- positions (final
  // after kernel 1) during kernels 2 and 3, velocities and accelerations
  // chunk by chunk of kernel 3's block map.
  if ((!pos || !vel || !acc) && h->n_total > 0) return SCF_ERR_NULL_POINTER;
  if (with_com && !com) return SCF_ERR_NULL_POINTER;
  if (!aligned16(pos) || !aligned16(vel) || !aligned16(acc)) return SCF_ERR_MISALIGNED;
  if (!h->copy_stream) {
    if (cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
      h->copy_stream = nullptr;
      return SCF_ERR_CUDA;
    }
    h->stage_ev.assign(SCF_STAGE_MAX_CHUNKS + 4, nullptr);  // start, in, done, kernels 1-2, one per chunk
    for (cudaEvent_t& e : h->stage_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return SCF_ERR_CUDA;
  }
  cudaStream_t cs = h->copy_stream;
  cudaEvent_t ev_start = h->stage_ev[0], ev_in = h->stage_ev[1], ev_done = h->stage_ev[2];
  cudaEvent_t* ev_out = &h->stage_ev[3];
  const size_t rec = h->cfg.precision == SCF_MIXED ? 16 : 32;
  const size_t bytes = rec * (size_t)h->n_total, com_bytes = sizeof(double) * 6 * (size_t)h->n_prog;
  char* dp[3] = {static_cast<char*>(pos), static_cast<char*>(vel), static_cast<char*>(acc)};
  char* hh[3] = {static_cast<char*>(host_pos), static_cast<char*>(host_vel), static_cast<char*>(host_acc)};
  auto ok = [](cudaError_t e) { return e == cudaSuccess; };
  // the device arrays may still be in use by work queued earlier on the handle's stream
  if (!ok(cudaEventRecord(ev_start, h->stream)) || !ok(cudaStreamWaitEvent(cs, ev_start, 0))) return SCF_ERR_CUDA;
  for (int i = 0; i < 3; ++i)
    if (bytes && !ok(cudaMemcpyAsync(dp[i], hh[i], bytes, cudaMemcpyHostToDevice, cs))) return SCF_ERR_CUDA;
  if (with_com && !ok(cudaMemcpyAsync(com, host_com, com_bytes, cudaMemcpyHostToDevice, cs))) return SCF_ERR_CUDA;
  if (!ok(cudaEventRecord(ev_in, cs)) || !ok(cudaStreamWaitEvent(h->stream, ev_in, 0))) return SCF_ERR_CUDA;
  int rc = run_coeffs(h, pos, vel, acc, h->step_mask, h->d_A, com, SCF_MODE_STEP);
  if (rc != SCF_OK) return rc;
  // kernel 2 (already queued) does not touch the positions; kernel 3 only reads them
  if (!ok(cudaEventRecord(ev_out[0], h->stream)) || !ok(cudaStreamWaitEvent(cs, ev_out[0], 0))) return SCF_ERR_CUDA;
  if (bytes && !ok(cudaMemcpyAsync(hh[0], dp[0], bytes, cudaMemcpyDeviceToHost, cs))) return SCF_ERR_CUDA;
  if (with_com && !ok(cudaMemcpyAsync(host_com, com, com_bytes, cudaMemcpyDeviceToHost, cs))) return SCF_ERR_CUDA;
  const int c3 = std::max(1, std::min(chunks, h->k3_blocks));
  for (int c = 0; c < c3 && h->k3_blocks > 0; ++c) {
    int b0, b1;
    block_range(h->k3_blocks, c3, c, &b0, &b1);
    if (b1 <= b0) continue;
    K3Args a = k3_args(h, pos, vel, acc, com, SCF_MODE_STEP);
    a.blk_prog += b0;
    a.blk_begin += b0;
    a.blk_end += b0;
    const cudaError_t e = timed(h, 2, [&] {
      return h->k3.variant == 2 ? scf_k3_ff_launch(a, b1 - b0, h->k3, h->stream)
                                : scf_k3_launch(h->cfg.precision, a, b1 - b0, h->k3_native, h->stream);
    });
    if (e != cudaSuccess) return SCF_ERR_CUDA;
    if (!ok(cudaEventRecord(ev_out[1 + c], h->stream)) || !ok(cudaStreamWaitEvent(cs, ev_out[1 + c], 0)))
      return SCF_ERR_CUDA;
    const size_t k0 = (size_t)h->h_blk3_begin[b0], k1 = (size_t)h->h_blk3_end[b1 - 1];
    for (int i = 1; i < 3; ++i)
      if (k1 > k0 && !ok(cudaMemcpyAsync(hh[i] + k0 * rec, dp[i] + k0 * rec, (k1 - k0) * rec, cudaMemcpyDeviceToHost, cs)))
        return SCF_ERR_CUDA;
  }
  // the handle's stream covers the copies too
  if (!ok(cudaEventRecord(ev_done, cs)) || !ok(cudaStreamWaitEvent(h->stream, ev_done, 0))) return SCF_ERR_CUDA;
  return SCF_OK;
}

int scf_set_option(scf_handle* h, int option, int value) {
  if (!h) return SCF_ERR_NULL_POINTER;
  if (option == SCF_OPT_GRAPHS) {
    h->graphs = value != 0;
    if (!h->graphs) drop_graph(h);
    return SCF_OK;
  }
  if (option == SCF_OPT_CENTRE_AHEAD) {
    if (value != 0 && value != 1) return SCF_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SCF_ERR_CUDA;
    h->centre_ahead = value == 1;
    drop_graph(h);
    return SCF_OK;
  }
  if (option == SCF_OPT_K1_TILE || option == SCF_OPT_K3_BLOCK) {
    if (value != 64 && value != 128 && value != 256 && !(option == SCF_OPT_K3_BLOCK && value == 320))
      return SCF_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SCF_ERR_CUDA;
    return option == SCF_OPT_K1_TILE ? use_k1(h, value) : use_k3(h, value);
  }
  if (option == SCF_OPT_K3_VARIANT) {
    if (value != 0 && value != 1) return SCF_ERR_INVALID_ARG;
    if (value == 1 && h->cfg.precision != SCF_FP64) return SCF_ERR_UNSUPPORTED;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SCF_ERR_CUDA;
    const bool old = h->k3_ff;
    h->k3_ff = value == 1;
    const int rc = use_k3(h, h->k3.threads);
    if (rc != SCF_OK) h->k3_ff = old;
    return rc;
  }
  if (option == SCF_OPT_K1_VARIANT) {
    if (value < 0 || value > 2) return SCF_ERR_INVALID_ARG;
    if (value == 2 && h->cfg.precision != SCF_FP64) return SCF_ERR_UNSUPPORTED;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SCF_ERR_CUDA;
    const bool old = h->k1_ff;
    h->k1_ff = value == 2;
    const int rc = use_k1(h, value == 1 ? 0 : 128);
    if (rc != SCF_OK) h->k1_ff = old;
    return rc;
  }
  return SCF_ERR_INVALID_ARG;
}

int scf_get_option(const scf_handle* h, int option, int* value) {
  if (!h || !value) return SCF_ERR_NULL_POINTER;
  if (option == SCF_OPT_GRAPHS) *value = h->graphs ? 1 : 0;
  else if (option == SCF_OPT_K1_TILE) *value = h->k1.variant == 1 ? 0 : h->k1.tile;
  else if (option == SCF_OPT_K1_VARIANT) *value = h->k1.variant;
  else if (option == SCF_OPT_K3_BLOCK) *value = h->k3.threads;
  else if (option == SCF_OPT_K3_VARIANT) *value = h->k3_ff ? 1 : 0;
  else if (option == SCF_OPT_CENTRE_AHEAD) *value = h->centre_ahead ? 1 : 0;
  else return SCF_ERR_INVALID_ARG;
  return SCF_OK;
}

int scf_autotune(scf_handle* h, const void* pos, const double* com, void* acc, int reps, double* ms_out) {
  if (!h) return SCF_ERR_NULL_POINTER;
  if ((!pos || !acc) && h->n_total > 0) return SCF_ERR_NULL_POINTER;
  if (h->host.n > 0 && !com) return SCF_ERR_NULL_POINTER;
  if (!aligned16(pos) || !aligned16(acc)) return SCF_ERR_MISALIGNED;
  if (reps < 1) return SCF_ERR_INVALID_ARG;
  if (h->n_total == 0) return SCF_OK;
  const bool prof = h->prof_on;
  h->prof_on = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SCF_ERR_CUDA;
  int rc = SCF_OK;
  auto time_it = [&](auto&& work, double* ms) -> int {
    for (int w = 0; w < 2; ++w)
      if ((rc = work()) != SCF_OK) return rc;
    cudaEventRecord(e0, h->stream);
    for (int r = 0; r < reps; ++r)
      if ((rc = work()) != SCF_OK) return rc;
    cudaEventRecord(e1, h->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return SCF_ERR_CUDA;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t / reps;
    return SCF_OK;
  };
  void* p = const_cast<void*>(pos);
  double best1 = 1e30, best3 = 1e30;
  int tp_best = h->k1.variant == 1 ? 0 : h->k1.tile, tb_best = h->k3.threads;
  if (ms_out)
    for (int i = 0; i < 8; ++i) ms_out[i] = 0.0;
  const int k1_candidates[4] = {64, 128, 256, 0};
  const int k1_slot[4] = {0, 1, 2, 6};
  for (int i = 0; i < 4 && rc == SCF_OK; ++i) {
    if (use_k1(h, k1_candidates[i]) != SCF_OK) continue;
    double ms = 0.0;
    rc = time_it([&] { return run_coeffs(h, p, nullptr, nullptr, nullptr, h->d_A, nullptr, SCF_MODE_COEFFS); }, &ms);
    if (ms_out) ms_out[k1_slot[i]] = ms;
    if (rc == SCF_OK && ms < best1) {
      best1 = ms;
      tp_best = k1_candidates[i];
    }
  }
  if (rc == SCF_OK) rc = use_k1(h, tp_best);
  if (rc == SCF_OK) rc = run_coeffs(h, p, nullptr, nullptr, nullptr, h->d_A, nullptr, SCF_MODE_COEFFS);
  if (rc == SCF_OK) rc = run_prep(h, h->d_A, com);
  const int k3_candidates[4] = {64, 128, 256, 320};
  const int k3_slot[4] = {3, 4, 5, 7};
  for (int i = 0; i < 4 && rc == SCF_OK; ++i) {
    if (use_k3(h, k3_candidates[i]) != SCF_OK) continue;
    double ms = 0.0;
    // the field pass as a step runs it, with its closing half kick (acc, which
    // is scratch here, standing in for the velocities)
    rc = time_it([&] { return run_forces(h, pos, acc, acc, com, SCF_MODE_STEP); }, &ms);
    if (ms_out) ms_out[k3_slot[i]] = ms;
    if (rc == SCF_OK && ms < best3) {
      best3 = ms;
      tb_best = k3_candidates[i];
    }
  }
  if (rc == SCF_OK) rc = use_k3(h, tb_best);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->prof_on = prof;
  return rc;
}

int scf_adjoint_level(scf_handle* h, const void* pos, const double* com, double weight, int drift, void* xbar,
                      void* vbar, double* combar, double* thetabar) {
  if (!h) return SCF_ERR_NULL_POINTER;
  if (h->cfg.precision != SCF_FP64) return SCF_ERR_ADJOINT_FP64;
  if (h->gen) return SCF_ERR_UNSUPPORTED;  // the adjoint kernels are written for alpha = 1
  for (int i = 0; i < h->host.n; ++i)        // and for the Hernquist, NFW and Miyamoto-Nagai components
    if (h->host.kind[i] == SCF_HOST_POWCUT) return SCF_ERR_UNSUPPORTED;
  if ((!pos || !xbar || !vbar) && h->n_total > 0) return SCF_ERR_NULL_POINTER;
  if (h->host.n > 0 && (!com || !combar || !thetabar)) return SCF_ERR_NULL_POINTER;
  if (!aligned16(pos) || !aligned16(xbar) || !aligned16(vbar)) return SCF_ERR_MISALIGNED;
  if (!std::isfinite(weight)) return SCF_ERR_INVALID_ARG;
  if (h->n_total == 0) return SCF_OK;
  if (!h->adj_ready) {
    int bps = 0;
    if (scf_k1_dual_prepare(h->cfg.lmax, h->cfg.nmax, &h->k1d, &bps) != cudaSuccess || bps < 1 ||
        scf_k3_dual_prepare(h->cfg.lmax, h->cfg.nmax, &h->k3d, &bps) != cudaSuccess || bps < 1) {
      cudaGetLastError();
      return SCF_ERR_UNSUPPORTED;
    }
    h->adj_ready = true;
  }
  drop_graph(h);  // the sweep rewrites the force coefficients a captured step reads
  void* p = const_cast<void*>(pos);
  const bool host = h->host.n > 0;
  AdjArgs adj{};
  adj.xbar = xbar;
  adj.vbar = vbar;
  adj.weight = weight;
  adj.drift = drift ? 1 : 0;
  adj.part = h->d_adj_part;
  // 1. coefficients and force coefficients at x_t
  int rc = run_coeffs(h, p, nullptr, nullptr, nullptr, h->d_A, nullptr, SCF_MODE_COEFFS);
  if (rc != SCF_OK) return rc;
  // 2. own-position term and tidal partials (dual numbers)
  if (h->k3_blocks > 0) {
    K3Args a = k3_args(h, pos, nullptr, nullptr, host ? com : nullptr, SCF_MODE_ADJ_DUAL);
    a.adj = adj;
    if (scf_k3_dual_launch(a, h->k3_blocks, h->k3d, h->stream) != cudaSuccess) return SCF_ERR_CUDA;
  }
  // 3. centre orbit and host parameters
  if (host) {
    ComAdjArgs c{};
    c.part = h->d_adj_part;
    c.blk3_prog = h->d_blk3_prog;
    c.n_blocks = h->k3_blocks;
    c.com = com;
    c.combar = combar;
    c.thetabar = thetabar;
    c.n_prog = h->n_prog;
    c.weight = weight;
    c.dt = h->cfg.dt;
    c.drift = adj.drift;
    c.host = h->host;
    if (scf_com_adj_launch(c, h->stream) != cudaSuccess) return SCF_ERR_CUDA;
  }
  // 4. A^J = sum_i d_i . grad B(x_i) (dual numbers, unit weights), normalised by kernel 2
  if (h->k1_blocks > 0) {
    K1Args a = k1_args(h, p, nullptr, nullptr, nullptr, SCF_MODE_ADJ_DUAL);
    a.adj = adj;
    if (scf_k1_dual_launch(a, h->k1_blocks, h->k1d, h->stream) != cudaSuccess) return SCF_ERR_CUDA;
  }
  K2Args b = k2_args(h, h->d_A, nullptr, SCF_MODE_COEFFS);
  if (scf_k2_launch(b, h->stream) != cudaSuccess) return SCF_ERR_CUDA;
  // 5. xbar_k += m_k f(x_k; A^J), then the drift is undone
  if (h->k3_blocks > 0) {
    K3Args a = k3_args(h, pos, nullptr, nullptr, nullptr, SCF_MODE_ADJ_J);
    a.adj = adj;
    if (scf_k3_launch(SCF_FP64, a, h->k3_blocks, h->k3_native, h->stream) != cudaSuccess) return SCF_ERR_CUDA;
  }
  return SCF_OK;
}

int scf_energy(scf_handle* h, const void* pos, const void* vel, const void* acc, const double* com, double* E_out) {
  if (!h || !E_out) return SCF_ERR_NULL_POINTER;
  if ((!pos || !vel || !acc) && h->n_total > 0) return SCF_ERR_NULL_POINTER;
  if (h->host.n > 0 && !com) return SCF_ERR_NULL_POINTER;
  if (!aligned16(pos) || !aligned16(vel) || !aligned16(acc)) return SCF_ERR_MISALIGNED;
  EnergyArgs a{};
  a.pos = pos;
  a.vel = vel;
  a.acc = acc;
  a.com = com;
  a.blk_prog = h->d_blk3_prog;
  a.blk_begin = h->d_blk3_begin;
  a.blk_end = h->d_blk3_end;
  a.n_blocks = h->k3_blocks;
  a.n_prog = h->n_prog;
  a.f32 = h->cfg.precision == SCF_MIXED;
  a.host = h->host;
  a.part = h->d_en_part;
  a.E_out = E_out;
  return cuda_fail(scf_energy_launch(a, h->stream));
}

int scf_bound(scf_handle* h, const void* pos, const void* vel, double kin, double frac, double* E_out,
              uint8_t* bound_out, uint8_t* mask_out, double* stats_out) {
  if (!h || !stats_out) return SCF_ERR_NULL_POINTER;
  if ((!pos || !vel || !bound_out) && h->n_total > 0) return SCF_ERR_NULL_POINTER;
  if (!aligned16(pos) || !aligned16(vel)) return SCF_ERR_MISALIGNED;
  if (!(kin > 0.0) || !std::isfinite(kin) || !(frac > 0.0 && frac <= 1.0)) return SCF_ERR_INVALID_ARG;
  BoundArgs a{};
  a.pos = pos;
  a.vel = vel;
  a.prog_off = h->d_off;
  a.n_prog = h->n_prog;
  a.n_total = h->n_total;
  a.f32 = h->cfg.precision == SCF_MIXED;
  a.split = h->bound_split;
  a.G = h->cfg.G;
  a.kin = kin;
  a.frac = frac;
  a.part = h->d_bpart;
  a.key = h->d_key;
  a.E_out = E_out;
  a.bound = bound_out;
  a.mask = mask_out;
  a.stats = stats_out;
  return cuda_fail(scf_bound_launch(a, h->bound_chunks, h->stream));
}

namespace {

int launch_tidal(scf_handle* h, const double* com, const double* M_c, int M_stride, double eta, double* out) {
  TidalArgs a{};
  a.com = com;
  a.M_c = M_c;
  a.M_stride = M_stride;
  a.n_prog = h->n_prog;
  a.G = h->cfg.G;
  a.eta = eta;
  a.host = h->host;
  a.out = out;
  return cuda_fail(scf_tidal_launch(a, h->stream));
}

}  // namespace

int scf_tidal(scf_handle* h, const double* com, const double* M_c, double eta, double* out) {
  if (!h || !out) return SCF_ERR_NULL_POINTER;
  if (h->host.n > 0 && !com) return SCF_ERR_NULL_POINTER;
  if (!(eta > 0.0) || !std::isfinite(eta)) return SCF_ERR_INVALID_ARG;
  return launch_tidal(h, com, M_c, 1, eta, out);
}

int scf_set_mask(scf_handle* h, const uint8_t* mask) {
  if (!h) return SCF_ERR_NULL_POINTER;
  if (mask != h->step_mask) {
    // the captured step holds the old pointer
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SCF_ERR_CUDA;
    drop_graph(h);
    h->step_mask = mask;
  }
  return SCF_OK;
}

int scf_evolve(scf_handle* h, void* pos, void* vel, void* acc, double* com, int nsteps, const scf_escape_params* ep,
               uint8_t* bound, uint8_t* mask, double* stats, int* n_refresh) {
  if (!h || !ep || !stats) return SCF_ERR_NULL_POINTER;
  if ((!pos || !vel || !acc || !bound || !mask) && h->n_total > 0) return SCF_ERR_NULL_POINTER;
  if (h->host.n > 0 && !com) return SCF_ERR_NULL_POINTER;
  if (!aligned16(pos) || !aligned16(vel) || !aligned16(acc)) return SCF_ERR_MISALIGNED;
  if (nsteps < 0 || ep->max_steps < 1 || !(ep->eta > 0.0) || !std::isfinite(ep->eta) || !(h->cfg.dt > 0.0))
    return SCF_ERR_INVALID_ARG;
  if (!(ep->kin > 0.0) || !std::isfinite(ep->kin) || !(ep->frac > 0.0 && ep->frac <= 1.0) || ep->retune_every < 0 ||
      (ep->recentre != 0 && ep->recentre != 1) || ep->retune_rule < 0 || ep->retune_rule > 2)
    return SCF_ERR_INVALID_ARG;
  if (ep->retune_rule == 2 && ep->retune_every > 0 &&
      (!(ep->alpha_lo > 0.0) || !(ep->alpha_hi > ep->alpha_lo) || !std::isfinite(ep->alpha_hi)))
    return SCF_ERR_INVALID_ARG;
  int rc = scf_set_mask(h, mask);
  if (rc != SCF_OK) return rc;
  std::vector<double> tid(16 * (size_t)h->n_prog);
  int done = 0, refreshes = 0;
  while (done < nsteps) {
    // boundedness and the coefficient set r <= r_x
    rc = scf_bound(h, pos, vel, ep->kin, ep->frac, nullptr, bound, mask, stats);
    if (rc != SCF_OK) return rc;
    if (ep->retune_every > 0 && refreshes % ep->retune_every == 0) {
      // complete refresh: the frame moved to the SCF centre and core velocity
      // (boundedness again in the new frame), then b from the bound stars'
      // half-mass radius (alpha fixed)
      if (ep->recentre) {
        rc = scf_recentre(h, pos, vel, acc, com, mask, kRecentreIters, kRecentreTol, nullptr);
        if (rc == SCF_OK) rc = scf_bound(h, pos, vel, ep->kin, ep->frac, nullptr, bound, mask, stats);
        if (rc != SCF_OK) return rc;
      }
      if (ep->retune_rule == 1) {  // b at the maximum of a_000 of the coefficient set
        rc = scf_retune_a000(h, pos, mask);
        if (rc != SCF_OK) return rc;
      } else if (ep->retune_rule == 2) {  // alpha and b at the joint maximum
        rc = scf_retune_alpha(h, pos, mask, ep->alpha_lo, ep->alpha_hi, nullptr);
        if (rc != SCF_OK) return rc;
      } else {
        BoundArgs a{};
        a.pos = pos;
        a.prog_off = h->d_off;
        a.n_prog = h->n_prog;
        a.n_total = h->n_total;
        a.f32 = h->cfg.precision == SCF_MIXED;
        a.frac = 0.5;
        a.key = h->d_key;
        a.bound = bound;
        a.mask = nullptr;
        a.stats = h->d_half;
        if (cuda_fail(scf_select_launch(a, h->stream)) != SCF_OK ||
            cuda_fail(scf_retune_b_launch(h->d_half, h->d_b, h->n_prog, h->cfg.alpha, h->stream)) != SCF_OK)
          return SCF_ERR_CUDA;
      }
    }
    // the field of the new set at the current positions (the next opening kick uses it)
    rc = run_coeffs(h, pos, nullptr, nullptr, mask, h->d_A, nullptr, SCF_MODE_COEFFS);
    if (rc == SCF_OK) rc = run_prep(h, h->d_A, com);
    if (rc == SCF_OK) rc = run_forces(h, pos, nullptr, acc, com, SCF_MODE_COEFFS);
    if (rc != SCF_OK) return rc;
    // leapfrog steps up to the next integration timestep (the shortest over progenitors)
    int k = ep->max_steps;
    if (h->host.n > 0) {
      rc = launch_tidal(h, com, stats + 1, 4, ep->eta, h->d_tid);
      if (rc != SCF_OK) return rc;
      if (cudaMemcpyAsync(tid.data(), h->d_tid, sizeof(double) * tid.size(), cudaMemcpyDeviceToHost, h->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(h->stream) != cudaSuccess)
        return SCF_ERR_CUDA;
      double dmin = HUGE_VAL;
      for (int p = 0; p < h->n_prog; ++p) dmin = std::min(dmin, tid[16 * (size_t)p + 15]);
      const double ks = std::floor(dmin / h->cfg.dt);
      if (ks < (double)k) k = ks < 1.0 ? 1 : (int)ks;
    }
    k = std::min(k, nsteps - done);
    rc = scf_step(h, pos, vel, acc, com, k);
    if (rc != SCF_OK) return rc;
    done += k;
    ++refreshes;
  }
  if (n_refresh) *n_refresh = refreshes;
  return SCF_OK;
}

int scf_recentre(scf_handle* h, void* pos, void* vel, void* acc, double* com, const uint8_t* mask, int max_iter,
                 double tol, double* out) {
  if (!h) return SCF_ERR_NULL_POINTER;
  if ((!pos || !vel || !acc) && h->n_total > 0) return SCF_ERR_NULL_POINTER;
  if (!aligned16(pos) || !aligned16(vel) || !aligned16(acc)) return SCF_ERR_MISALIGNED;
  if (max_iter < 1 || max_iter > 1000 || !(tol >= 0.0) || !std::isfinite(tol)) return SCF_ERR_INVALID_ARG;
  RecentreArgs a{};
  a.pos = pos;
  a.vel = vel;
  a.acc = acc;
  a.mask = mask;
  a.blk_prog = h->d_blk3_prog;
  a.blk_begin = h->d_blk3_begin;
  a.blk_end = h->d_blk3_end;
  a.n_blocks = h->k3_blocks;
  a.n_prog = h->n_prog;
  a.f32 = h->cfg.precision == SCF_MIXED;
  a.b_prog = h->d_b;
  a.alpha = h->cfg.alpha;
  a.inv_alpha = 1.0 / h->cfg.alpha;
  a.tol = tol;
  a.part = h->d_en_part;
  a.state = h->d_rc;
  a.com = com;
  // 1. the centre, particles shifted to it
  if (cuda_fail(scf_centre_launch(a, max_iter, h->stream)) != SCF_OK) return SCF_ERR_CUDA;
  // 2. the set's coefficients about it; the density's potential (K_nl A) in acc.w
  int rc = run_coeffs(h, pos, nullptr, nullptr, mask, h->d_A, nullptr, SCF_MODE_COEFFS);
  if (rc != SCF_OK) return rc;
  if (cuda_fail(scf_scale_k_launch(h->d_A, h->d_Atmp, h->cfg.nmax, h->cfg.lmax, h->n_prog, h->cfg.alpha,
                                   h->stream)) != SCF_OK)
    return SCF_ERR_CUDA;
  rc = run_prep(h, h->d_Atmp, nullptr);
  if (rc == SCF_OK) rc = run_forces(h, pos, nullptr, acc, nullptr, SCF_MODE_COEFFS);
  if (rc != SCF_OK) return rc;
  // 3. core radius and velocity, the frame moved to (x_c, V_core)
  if (cuda_fail(scf_core_launch(a, h->stream)) != SCF_OK) return SCF_ERR_CUDA;
  if (!out) return SCF_OK;
  std::vector<double> st(16 * (size_t)h->n_prog);
  if (cudaMemcpyAsync(st.data(), h->d_rc, sizeof(double) * st.size(), cudaMemcpyDeviceToHost, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return SCF_ERR_CUDA;
  for (int p = 0; p < h->n_prog; ++p) {
    const double* s = st.data() + 16 * (size_t)p;
    double* o = out + 8 * (size_t)p;
    o[0] = s[0];
    o[1] = s[1];
    o[2] = s[2];
    o[3] = s[6];
    o[4] = s[7];
    o[5] = s[8];
    o[6] = std::sqrt(s[5]);
    o[7] = s[3];
  }
  return SCF_OK;
}

int scf_retune_a000(scf_handle* h, const void* pos, const uint8_t* mask) {
  if (!h) return SCF_ERR_NULL_POINTER;
  if (!pos && h->n_total > 0) return SCF_ERR_NULL_POINTER;
  if (!aligned16(pos)) return SCF_ERR_MISALIGNED;
  ScaleArgs a{};
  a.pos = pos;
  a.mask = mask;
  a.blk_prog = h->d_blk3_prog;
  a.blk_begin = h->d_blk3_begin;
  a.blk_end = h->d_blk3_end;
  a.n_blocks = h->k3_blocks;
  a.n_prog = h->n_prog;
  a.f32 = h->cfg.precision == SCF_MIXED;
  a.b_prog = h->d_b;
  a.alpha = h->cfg.alpha;
  a.inv_alpha = 1.0 / h->cfg.alpha;
  a.span = 8.0;
  a.part = h->d_sp;
  a.state = h->d_rc;
  return cuda_fail(scf_scale_a000_launch(a, h->stream));
}

namespace {

// Digamma function psi(x), x > 0: the recurrence psi(x) = psi(x + 1) - 1/x up
// to x >= 8, then the asymptotic series ln x - 1/(2x) - sum_k B_2k / (2k x^2k)
// (Abramowitz & Stegun 6.3.5 and 6.3.18).
double digamma_host(double x) {
  double acc = 0.0;
  while (x < 8.0) {
    acc -= 1.0 / x;
    x += 1.0;
  }
  const double i2 = 1.0 / (x * x);
  const double series =
      i2 * (1.0 / 12 - i2 * (1.0 / 120 - i2 * (1.0 / 252 - i2 * (1.0 / 240 - i2 * (1.0 / 132 - i2 * (691.0 / 32760))))));
  return acc + std::log(x) - 0.5 / x - series;
}

// ln|I_00(alpha)| at b = 1 and its alpha derivative, for the lowest pair of
// the Zhao family: |I_00| = (alpha + 1) Gamma(2 alpha + 1) /
// (2^(4 alpha + 3) (alpha + 1/2) Gamma(alpha + 1/2)^2).
double ln_i00(double al) {
  return std::log(al + 1.0) + std::lgamma(2.0 * al + 1.0) - (4.0 * al + 3.0) * std::log(2.0) - std::log(al + 0.5) -
         2.0 * std::lgamma(al + 0.5);
}
double dln_i00(double al) {
  return 1.0 / (al + 1.0) + 2.0 * digamma_host(2.0 * al + 1.0) - 4.0 * std::log(2.0) - 1.0 / (al + 0.5) -
         2.0 * digamma_host(al + 0.5);
}

// Moves the handle to the radial family of exponent alpha: recurrence tables,
// normalisation and field-kernel scales rebuilt and uploaded, the general
// kernels selected for alpha != 1 (default shapes; no float-float variants).
int set_alpha(scf_handle* h, double alpha) {
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SCF_ERR_CUDA;
  const bool gen = alpha != 1.0;
  {
    std::unique_ptr<ScfConst> t(new (std::nothrow) ScfConst);
    if (!t) return SCF_ERR_OUT_OF_MEMORY;
    scf_make_const(t.get(), alpha);
    if (gen && !tables_finite(*t, h->cfg.lmax, h->cfg.nmax, h->cfg.precision == SCF_MIXED))
      return SCF_ERR_UNSUPPORTED;
    if (gen && !put(h->d_tab, t.get(), sizeof(ScfConst))) return SCF_ERR_CUDA;
    if (!put_steps(h, *t)) return SCF_ERR_CUDA;
  }
  std::vector<double> norm(2 * (size_t)h->nc), ksc(2 * (size_t)h->nc);
  scf_make_norm(h->cfg.nmax, h->cfg.lmax, norm.data(), alpha);
  scf_make_kscale(h->cfg.nmax, h->cfg.lmax, ksc.data(), alpha);
  for (double x : norm)
    if (!std::isfinite(x)) return SCF_ERR_UNSUPPORTED;
  std::vector<float> ksc_f(ksc.begin(), ksc.end());
  const bool ok = (h->cfg.precision == SCF_MIXED ? put(h->d_kscale, ksc_f.data(), sizeof(float) * ksc_f.size())
                                                 : put(h->d_kscale, ksc.data(), sizeof(double) * ksc.size())) &&
                  put(h->d_norm, norm.data(), sizeof(double) * norm.size());
  if (!ok) return SCF_ERR_CUDA;
  h->cfg.alpha = alpha;
  h->gen = gen;
  if (gen) h->k1_ff = h->k3_ff = false;
  int rc = h->cfg.precision == SCF_MIXED ? use_k1(h, 0) : SCF_ERR_UNSUPPORTED;
  if (rc != SCF_OK) rc = use_k1(h, 128);
  if (rc == SCF_OK) rc = use_k3(h, 128);
  drop_graph(h);
  return rc;
}

}  // namespace

int scf_retune_alpha(scf_handle* h, const void* pos, const uint8_t* mask, double alpha_lo, double alpha_hi,
                     double* alpha_out) {
  if (!h) return SCF_ERR_NULL_POINTER;
  if (!pos && h->n_total > 0) return SCF_ERR_NULL_POINTER;
  if (!aligned16(pos)) return SCF_ERR_MISALIGNED;
  if (!(alpha_lo > 0.0) || !(alpha_hi > alpha_lo) || !std::isfinite(alpha_hi)) return SCF_ERR_INVALID_ARG;
  if (alpha_lo < SCF_ALPHA_MIN || alpha_hi > SCF_ALPHA_MAX) return SCF_ERR_UNSUPPORTED;
  const int P = h->n_prog;
  std::vector<double> b0(P), st(4 * (size_t)P);
  if (cudaMemcpyAsync(b0.data(), h->d_b, sizeof(double) * P, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return SCF_ERR_CUDA;
  ScaleArgs a{};
  a.pos = pos;
  a.mask = mask;
  a.blk_prog = h->d_blk3_prog;
  a.blk_begin = h->d_blk3_begin;
  a.blk_end = h->d_blk3_end;
  a.n_blocks = h->k3_blocks;
  a.n_prog = P;
  a.f32 = h->cfg.precision == SCF_MIXED;
  a.span = 8.0;
  a.part = h->d_sp;
  a.state = h->d_rc;
  double* d_bt = h->d_alpha;            // trial scales b_p(alpha)
  double* d_sums = h->d_alpha + P;      // [P][3] sums at (alpha, b_p(alpha))
  // ln of the product of the progenitors' a_000 at alpha (each at its own
  // maximising b) and its alpha derivative (envelope theorem), from one
  // b search and one pass of sums; `live` counts progenitors with a set
  int live = 0;
  auto eval = [&](double al, double* H, double* dH, std::vector<double>* bs) -> int {
    if (!put(d_bt, b0.data(), sizeof(double) * P)) return SCF_ERR_CUDA;
    a.b_prog = d_bt;
    a.alpha = al;
    a.inv_alpha = 1.0 / al;
    if (scf_scale_a000_launch(a, h->stream) != cudaSuccess || scf_alpha_sums_launch(a, d_sums, h->stream) != cudaSuccess)
      return SCF_ERR_CUDA;
    std::vector<double> bt(P), sm(3 * (size_t)P);
    if (cudaMemcpyAsync(bt.data(), d_bt, sizeof(double) * P, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(sm.data(), d_sums, sizeof(double) * 3 * P, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return SCF_ERR_CUDA;
    double hs = 0.0, ds = 0.0;
    live = 0;
    for (int p = 0; p < P; ++p) {
      if (!(sm[3 * p + 2] > 0.0) || !(sm[3 * p] > 0.0)) continue;
      ++live;
      hs += -0.5 * ln_i00(al) - 0.5 * std::log(bt[p]) + std::log(sm[3 * p]);
      ds += -0.5 * dln_i00(al) + sm[3 * p + 1] / sm[3 * p];
    }
    *H = hs;
    *dH = ds;
    if (bs) *bs = bt;
    return SCF_OK;
  };
  constexpr int kGrid = 17;
  const double x_lo = std::log(alpha_lo), x_hi = std::log(alpha_hi), step = (x_hi - x_lo) / (kGrid - 1);
  double hbest = -HUGE_VAL, dummy = 0.0;
  int jbest = 0, rc = SCF_OK;
  for (int j = 0; j < kGrid; ++j) {
    double hj = 0.0;
    if ((rc = eval(std::exp(x_lo + j * step), &hj, &dummy, nullptr)) != SCF_OK) return rc;
    if (live == 0) {  // no progenitor has a coefficient set: nothing to fit
      if (alpha_out) *alpha_out = h->cfg.alpha;
      return SCF_OK;
    }
    if (hj > hbest) {
      hbest = hj;
      jbest = j;
    }
  }
  double x = x_lo + jbest * step;
  if (jbest > 0 && jbest < kGrid - 1) {
    // root of dH in the bracket by the Illinois variant of regula falsi
    double a0 = x - step, a1 = x + step, f0 = 0.0, f1 = 0.0, hh = 0.0;
    if ((rc = eval(std::exp(a0), &hh, &f0, nullptr)) != SCF_OK || (rc = eval(std::exp(a1), &hh, &f1, nullptr)) != SCF_OK)
      return rc;
    if (f0 > 0.0 && f1 < 0.0) {
      int side = 0;
      for (int it = 0; it < 100 && a1 - a0 > 1e-15 * (1.0 + std::fabs(a0)); ++it) {
        const double xm = (a0 * f1 - a1 * f0) / (f1 - f0);
        double fm = 0.0;
        if ((rc = eval(std::exp(xm), &hh, &fm, nullptr)) != SCF_OK) return rc;
        x = xm;
        if (fm == 0.0) break;
        if (fm > 0.0) {
          a0 = xm;
          f0 = fm;
          if (side == 1) f1 *= 0.5;
          side = 1;
        } else {
          a1 = xm;
          f1 = fm;
          if (side == -1) f0 *= 0.5;
          side = -1;
        }
      }
    }
  }
  const double alpha = std::exp(x);
  std::vector<double> bs;
  double hh = 0.0;
  if ((rc = eval(alpha, &hh, &dummy, &bs)) != SCF_OK) return rc;
  // the new exponent: tables, normalisation, kernels; then each progenitor's b
  const double old = h->cfg.alpha;
  rc = set_alpha(h, alpha);
  if (rc != SCF_OK) {
    set_alpha(h, old);
    return rc;
  }
  for (int p = 0; p < P; ++p)
    if (!(bs[p] > 0.0) || !std::isfinite(bs[p])) bs[p] = b0[p];
  if (!put(h->d_b, bs.data(), sizeof(double) * P)) return SCF_ERR_CUDA;
  if (alpha_out) *alpha_out = alpha;
  return SCF_OK;
}

int scf_get_alpha(const scf_handle* h, double* alpha) {
  if (!h || !alpha) return SCF_ERR_NULL_POINTER;
  *alpha = h->cfg.alpha;
  return SCF_OK;
}

int scf_get_scales(scf_handle* h, double* b_out) {
  if (!h || !b_out) return SCF_ERR_NULL_POINTER;
  return cuda_fail(
      cudaMemcpyAsync(b_out, h->d_b, sizeof(double) * h->n_prog, cudaMemcpyDeviceToDevice, h->stream));
}

int scf_last_coeffs(scf_handle* h, double* A_out) {
  if (!h || !A_out) return SCF_ERR_NULL_POINTER;
  return cuda_fail(cudaMemcpyAsync(A_out, h->d_A, sizeof(double) * 2 * (size_t)h->nc * h->n_prog,
                                   cudaMemcpyDeviceToDevice, h->stream));
}

int scf_status(scf_handle* h, int* status) {
  if (!h) return SCF_ERR_NULL_POINTER;
  unsigned word = 0;
  if (cudaMemcpyAsync(&word, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return SCF_ERR_CUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SCF_ERR_CUDA;
  if (cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), h->stream) != cudaSuccess) return SCF_ERR_CUDA;
  if (status) *status = (int)word;
  return word ? SCF_ERR_DEVICE_STATUS : SCF_OK;
}

int scf_launches_per_call(const scf_handle* h, int which) {
  if (!h) return SCF_ERR_NULL_POINTER;
  const int k1 = h->k1_blocks > 0 ? 1 : 0, k3 = h->k3_blocks > 0 ? 1 : 0;
  if (which == 0) return k1 + 1;
  if (which == 1) return 1 + k3;
  if (which == 2) return k1 + 1 + k3;
  return SCF_ERR_INVALID_ARG;
}

int scf_profile(scf_handle* h, int enable) {
  if (!h) return SCF_ERR_NULL_POINTER;
  if (!enable) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SCF_ERR_CUDA;
    prof_release(h);
    return SCF_OK;
  }
  if (h->prof_ev.empty()) {
    h->prof_ev.resize(2 * kProfPairs, nullptr);
    h->prof_kind.resize(kProfPairs, 0);
    for (auto& e : h->prof_ev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        prof_release(h);
        return SCF_ERR_CUDA;
      }
  }
  h->prof_used = 0;
  h->prof_on = true;
  return SCF_OK;
}

int scf_profile_read(scf_handle* h, double* ms, int64_t* launches) {
  if (!h) return SCF_ERR_NULL_POINTER;
  double t[3] = {0, 0, 0};
  int64_t n[3] = {0, 0, 0};
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SCF_ERR_CUDA;
  for (int i = 0; i < h->prof_used; ++i) {
    float e = 0.f;
    if (cudaEventElapsedTime(&e, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]) != cudaSuccess) return SCF_ERR_CUDA;
    t[h->prof_kind[i]] += e;
    n[h->prof_kind[i]] += 1;
  }
  h->prof_used = 0;
  for (int k = 0; k < 3; ++k) {
    if (ms) ms[k] = t[k];
    if (launches) launches[k] = n[k];
  }
  return SCF_OK;
}

int scf_free(scf_handle* h) {
  if (!h) return SCF_OK;
  int rc = SCF_OK;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = SCF_ERR_CUDA;
  prof_release(h);
  drop_graph(h);
  if (h->copy_stream && cudaStreamSynchronize(h->copy_stream) != cudaSuccess) rc = SCF_ERR_CUDA;
  for (cudaEvent_t e : h->stage_ev) cudaEventDestroy(e);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->side_stream && cudaStreamSynchronize(h->side_stream) != cudaSuccess) rc = SCF_ERR_CUDA;
  for (cudaEvent_t e : h->side_ev)
    if (e) cudaEventDestroy(e);
  if (h->side_stream) cudaStreamDestroy(h->side_stream);
  if (h->d_base && cudaFree(h->d_base) != cudaSuccess) rc = SCF_ERR_CUDA;
  if (h->d_split && cudaFree(h->d_split) != cudaSuccess) rc = SCF_ERR_CUDA;
  delete h;
  return rc;
}

const char* scf_strerror(int code) {
  switch (code) {
    case SCF_OK: return "ok";
    case SCF_ERR_INVALID_ARG: return "invalid argument (size, count, offset or option out of range)";
    case SCF_ERR_NULL_POINTER: return "required pointer is NULL";
    case SCF_ERR_MISALIGNED: return "particle pointer is not 16-byte aligned";
    case SCF_ERR_UNSUPPORTED:
      return "unsupported configuration (nmax/lmax above the compiled limits, alpha outside its range, or a kernel "
             "variant or the adjoint with alpha != 1)";
    case SCF_ERR_CUDA: return "CUDA runtime error";
    case SCF_ERR_OUT_OF_MEMORY: return "workspace allocation failed";
    case SCF_ERR_DEVICE_STATUS: return "device reported non-finite particle data";
    case SCF_ERR_ADJOINT_FP64: return "the adjoint needs a double-precision (SCF_FP64) handle";
    case SCF_ERR_TOO_LARGE: return "problem exceeds the static scratch of scf_coeffs_noalloc (2*NC > SCF_NOALLOC_MAX_COEFS)";
    default: return "unknown error code";
  }
}

}  // extern "C"
