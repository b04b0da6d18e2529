// Internal interfaces between the C ABI layer (scf_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "scf_device.cuh"

enum ScfMode {
  SCF_MODE_COEFFS = 0,   // plain evaluation
  SCF_MODE_STEP = 1,     // with the leapfrog kick (and drift in kernel 1)
  SCF_MODE_ADJ_J = 2,    // kernel 3 (double): xbar += m f(x; J), then vbar += dt xbar
  SCF_MODE_ADJ_DUAL = 3  // dual numbers along d = weight * vbar (scf_adjoint.cu)
};

// Adjoint state of the particles used by the adjoint modes.  At level t of the
// reverse sweep the acceleration a(x_t) is pulled back along d_k = weight * vbar_k
// (weight = dt/2 at the first and last level, dt in between: a(x_t) feeds the
// closing kick of step t and the opening kick of step t+1).
struct AdjArgs {
  void* xbar;            // [N][4] double, adjoint of positions (updated)
  void* vbar;            // [N][4] double, adjoint of velocities (read; updated by ADJ_J with drift)
  double weight;
  int drift;             // 1: after the pull-back, undo the drift (vbar += dt xbar)
  double* part;          // kernel 3 dual mode: per-block partial sums [blocks][SCF_ADJ_Q]
};

// Per-block adjoint partials of the tidal term, over the block's particles k
// (P_k = R + x_k): sum d_k (3), sum T(P_k) d_k (3), then per host component c
// sum d_k . a_c(P_k)/GM_c and sum d_k . da_c(P_k)/d(scale length a_c).
#define SCF_ADJ_Q (6 + 2 * SCF_HOST_CAP)

// Kernel 1: per-block partial sums of the coefficients (optionally after the
// half kick + drift of a leapfrog step).
struct K1Args {
  void* pos;          // [N][4] float or double (read; written in step mode)
  void* vel;          // [N][4] (step mode)
  const void* acc;    // [N][4] (step mode)
  // step mode, register-tiled kernel, optional: a second copy of the drifted
  // positions, and where the half-kicked velocities go (null: vel)
  void* pos_copy;
  void* vel_out;
  const uint8_t* mask;
  double* partials;   // [n_blocks][2*NC]
  const int* blk_prog;
  const int64_t* blk_begin;
  const int64_t* blk_end;
  const double* b_prog;
  int nmax, lmax, nc, nlm;
  int mode;
  double dt;
  unsigned* status;
  AdjArgs adj;
  // register-tiled single-precision kernel: contraction items, particle
  // sub-groups per block, windows per block and tiles per window (partials
  // are then float rows, sub * win per block)
  int items, sub, win, win_tiles;
  // radial family of exponent alpha != 1 (the general kernels): the handle's
  // tables in device memory, alpha and 1/alpha
  const ScfConst* tab;
  double alpha, inv_alpha;
};

// Kernel 2: fixed-order reduction of the partials, normalisation, and the
// centre-of-mass leapfrog step.
struct K2Args {
  const double* partials;
  const int* prog_blk_off;  // [n_prog+1]
  const double* norm;       // [2*NC]
  double* A_out;            // [n_prog][2*NC]
  int nc, n_prog, nlm;
  int mode;
  double dt;
  double* com;              // [n_prog][6] (step mode with host)
  ScfHostParams host;
  // optional: force coefficients F = -G {S,T} / (b N_lm) as (cos, sin) pairs
  // of the field kernel's element type (single precision: times gscale[l][n],
  // the scale of the field kernel's radial recurrence), and a_host(R) per
  // progenitor
  void* F_out;              // [n_prog][NC] float2 (f32) or double2, or null
  int f32;                  // element type of F_out
  const float* kscale_f;    // f32: [NC] (gscale, hscale) pairs
  // f32 with a host: the values of the single-precision tidal difference that
  // depend on R alone, [n_prog][SCF_HOST_CAP][SCF_TIDAL_W] (scf_tidal_prep_f32)
  float* tid_out;
  const float* tid_next;    // the same for the centre steps computed ahead (with cnext), or null
  const double* b_prog;
  double G;
  double* aR_out;           // [n_prog][4], or null
  // partials layout: sub == 0: [blocks][2*NC] doubles; sub > 0: [blocks][sub][2*NC]
  // floats (sub rows per block, one per window of the register-tiled kernel 1)
  // without the T_nl0 entries (read as 0)
  int sub;
  // optional (step mode): centre steps computed ahead, [n_prog][kCentreW]
  // doubles (see CentreArgs); the centre block takes entry p's result when
  // its key equals the state it is about to step
  const double* cnext;
};

// The centre's next kick-drift-kick computed ahead (beside kernel 3, on a
// second stream): entry p of cnext holds [0, 6) the state it started from
// (the key), [6, 12) the stepped state, [12, 15) a_host at the new R, [15]
// the dt used.  The first kick takes a_host(R) from aR, which kernel 2
// wrote for that same R.
constexpr int kCentreW = 16;
struct CentreArgs {
  const double* com;        // [n_prog][6]
  const double* aR;         // [n_prog][4]
  double* cnext;            // [n_prog][kCentreW]
  float* tid_next;          // f32: the tidal difference's R-only values at the stepped R, or null
  double dt;
  int n_prog;
  ScfHostParams host;
};
cudaError_t scf_centre_next_launch(const CentreArgs& a, int priority, cudaStream_t s);

// Force coefficients and a_host(R) from given coefficients (scf_forces).
struct PrepArgs {
  const double* A;          // [n_prog][2*NC]
  const double* com;        // [n_prog][6] or null
  void* F_out;
  int f32;
  const float* kscale_f;    // as in K2Args
  float* tid_out;           // as in K2Args
  const double* b_prog;
  double G;
  double* aR_out;
  int nc, nlm, n_prog;
  ScfHostParams host;
};

// Kernel 3: acceleration (+ tidal term) and, in step mode, the closing half kick.
struct K3Args {
  const void* pos;
  void* vel;
  void* acc;
  const void* vel_in;       // step mode, optional: the velocities to kick (null: vel); the result goes to vel
  const void* F;            // [n_prog][NC] (cos, sin) force-coefficient pairs
  const double* com;        // [n_prog][6] or null (R is read)
  const double* aR;         // [n_prog][4] a_host(R)
  const void* kscale;       // [NC] (gscale[l][n], hscale[l][n-1]) pairs of the element type
  const int* blk_prog;
  const int64_t* blk_begin;
  const int64_t* blk_end;
  const double* b_prog;
  int nmax, lmax, nc, nlm;
  int mode;
  double G, dt;
  ScfHostParams host;
  unsigned* status;
  AdjArgs adj;
  const ScfConst* tab;  // radial family of exponent alpha != 1, as in K1Args
  double alpha, inv_alpha;
  // single precision: the per-(l, n) radial recurrence constants (gbeta,
  // hbeta, hratio, 0) of the handle's family, [lmax + 1][nmax + 1], and the
  // R-only values of the tidal difference that kernel 2 left (see K2Args)
  const float4* cs;
  const float* tid;
};

// Adjoint of the tidal term and of the centre orbit at one level of the reverse sweep.
struct ComAdjArgs {
  const double* part;        // kernel 3 dual-mode partials [blocks][SCF_ADJ_Q]
  const int* blk3_prog;      // progenitor of each kernel 3 block
  int n_blocks;
  const double* com;         // [n_prog][6] centre state at this level
  double* combar;            // [n_prog][6] adjoint of (R, V), updated
  double* thetabar;          // [n_prog][2 n_host] adjoint of (GM_c, a_c), accumulated
  int n_prog;
  double weight, dt;
  int drift;
  ScfHostParams host;
};

// Energy diagnostic (scf_energy.cu): per kernel-3 block partial sums of the
// kinetic, self and tidal energy, then a fixed-order sum per progenitor.
struct EnergyArgs {
  const void* pos;
  const void* vel;
  const void* acc;           // acc.w = psi_SCF at pos
  const double* com;         // [n_prog][6] or null
  const int* blk_prog;
  const int64_t* blk_begin;
  const int64_t* blk_end;
  int n_blocks, n_prog;
  int f32;                   // particle arrays are float4 (mixed) or double4
  ScfHostParams host;
  double* part;              // [n_blocks][4]
  double* E_out;             // [n_prog][4]
};
cudaError_t scf_energy_launch(const EnergyArgs& a, cudaStream_t s);

// Re-centring (scf_recentre.cu): the SCF centre at the maximum of a_000 and the
// core frame velocity, per kernel-3 block range with fixed-order sums.
struct RecentreArgs {
  void* pos;                 // [N][4], shifted in place by -x_c
  void* vel;                 // [N][4], shifted in place by -V_core
  const void* acc;           // acc.w = potential of the K_nl-scaled coefficients (core pass)
  const uint8_t* mask;       // coefficient set of the centre iteration, or null
  const int* blk_prog;
  const int64_t* blk_begin;
  const int64_t* blk_end;
  int n_blocks, n_prog;
  int f32;                   // float4 (mixed) or double4 particles
  const double* b_prog;
  double alpha, inv_alpha, tol;
  double* part;              // [n_blocks][4] scratch
  double* state;             // [n_prog][16]: x_c(3), iterations, converged, r_core^2, V_core(3)
  double* com;               // [n_prog][6] or null: += (x_c, V_core)
};
// max_iter mean-shift iterations (converged progenitors skip), then x -= x_c.
cudaError_t scf_centre_launch(const RecentreArgs& a, int max_iter, cudaStream_t s);
// KA = K_nl A (every progenitor's [2 NC] row).
cudaError_t scf_scale_k_launch(const double* A, double* KA, int nmax, int lmax, int n_prog, double alpha,
                               cudaStream_t s);
// r_core and V_core from acc.w, com += (x_c, V_core), v -= V_core.
cudaError_t scf_core_launch(const RecentreArgs& a, cudaStream_t s);

// Basis scale at the maximum of the bi-orthonormal a_000 (scf_recentre.cu):
// kScaleRounds grids of kScalePoints values of ln b, b_prog updated in place.
constexpr int kScalePoints = 33;
constexpr int kScaleRounds = 3;
constexpr int kScaleNewton = 4;  // safeguarded Newton steps on d ln a_000 / d ln b = 0 after the grids
struct ScaleArgs {
  const void* pos;
  const uint8_t* mask;       // coefficient set, or null
  const int* blk_prog;
  const int64_t* blk_begin;
  const int64_t* blk_end;
  int n_blocks, n_prog;
  int f32;
  double* b_prog;            // [n_prog], read and updated
  double alpha, inv_alpha, span;
  double* part;              // [n_blocks][kScalePoints + 1] scratch
  double* state;             // [n_prog][4] scratch
};
cudaError_t scf_scale_a000_launch(const ScaleArgs& a, cudaStream_t s);
// Sums of the exponent search at (a.alpha, a.b_prog[p]) per progenitor into
// out[p][3] = (sum m g, sum m g d ln g / d alpha, sum m), g = (1 + (r/b)^(1/alpha))^-alpha.
cudaError_t scf_alpha_sums_launch(const ScaleArgs& a, double* out, cudaStream_t s);

struct ScfLaunchInfo {
  int threads;   // threads per block
  int tile;      // particles per tile (block ranges are whole tiles)
  size_t smem;   // dynamic shared memory per block
  int variant;   // kernel variant chosen by the prepare call (1: register-tiled single precision)
  int items;     // variant 1: TN x TM contraction items (output tiles) per particle sub-group
  int sub;       // variant 1: particle sub-groups per block
  int win;       // variant 1: windows per block (partial rows per block = sub * win)
  int win_tiles; // variant 1: tiles per window
};

void scf_make_norm(int nmax, int lmax, double* norm, double alpha = 1.0);
// Per-coefficient scale pairs (gscale[l][n], hscale[l][n-1]; 0 at n = 0) of the
// field kernel's scaled recurrences, as doubles ([NC][2]).
void scf_make_kscale(int nmax, int lmax, double* kscale, double alpha = 1.0);

cudaError_t scf_com_adj_launch(const ComAdjArgs& a, cudaStream_t s);
// Dual-number kernels of the adjoint (double precision).  Both loop over their
// block's particle range, so they run on the block maps of kernels 1 and 3
// whatever tile those were built for.
cudaError_t scf_k1_dual_prepare(int lmax, int nmax, ScfLaunchInfo* info, int* blocks_per_sm);
cudaError_t scf_k1_dual_launch(const K1Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s);
cudaError_t scf_k3_dual_prepare(int lmax, int nmax, ScfLaunchInfo* info, int* blocks_per_sm);
cudaError_t scf_k3_dual_launch(const K3Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s);

// Each kernel translation unit keeps its own copy of the constant tables.
cudaError_t scf_upload_const_coeffs(const ScfConst* t);
cudaError_t scf_upload_const_forces(const ScfConst* t);
cudaError_t scf_upload_const_adjoint(const ScfConst* t);

// Launch configuration (threads, dynamic shared memory) of each kernel for
// the given sizes; sets the shared-memory attribute of the instantiation.
// tp: kernel 1 particle tile (64, 128, 256); tb: kernel 3 block size (64, 128, 256).
cudaError_t scf_k1_prepare(int precision, int lmax, int nmax, int tp, ScfLaunchInfo* info, int* blocks_per_sm);
// Kernel 1 for the radial family of exponent alpha != 1 (K1Args::tab), 128-particle
// tiles; info->variant = 3.
cudaError_t scf_k1_gen_prepare(int precision, int lmax, int nmax, ScfLaunchInfo* info, int* blocks_per_sm);
// Register-tiled single-precision kernel 1 (info->variant = 1).
// gen: the radial family of exponent alpha != 1 (runtime steps from K1Args::tab,
// which the launch then requires).
cudaError_t scf_k1_tiled_prepare(int lmax, int nmax, ScfLaunchInfo* info, int* blocks_per_sm, bool gen = false);
// Windows per block of the register-tiled kernel for a block map whose
// longest block has the given number of particles.
int scf_k1_windows(int64_t max_particles_per_block, const ScfLaunchInfo& info);
cudaError_t scf_k3_prepare(int precision, int lmax, int nmax, int tb, ScfLaunchInfo* info, int* blocks_per_sm);
// Kernel 3 for the radial family of exponent alpha != 1 (K3Args::tab), 128-thread
// blocks; info->variant = 3.
cudaError_t scf_k3_gen_prepare(int precision, int lmax, int nmax, ScfLaunchInfo* info, int* blocks_per_sm);
// Float-float kernel 3 for double-precision handles (info->variant = 2; the
// same threads, tile and block map as the double kernel; modes COEFFS and STEP).
cudaError_t scf_k3_ff_prepare(int lmax, int nmax, int tb, ScfLaunchInfo* info, int* blocks_per_sm);
cudaError_t scf_k3_ff_launch(const K3Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s);
cudaError_t scf_upload_const_forces_ff(const ScfConst* t);
// Float-float kernel 1 for double-precision handles (info->variant = 2; 128-
// particle tiles; double partial rows as the native kernel).
cudaError_t scf_k1_ff_prepare(int lmax, int nmax, int tp, ScfLaunchInfo* info, int* blocks_per_sm);
cudaError_t scf_k1_ff_launch(const K1Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s);
cudaError_t scf_upload_const_coeffs_ff(const ScfConst* t);

cudaError_t scf_k1_launch(int precision, const K1Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s);
cudaError_t scf_k2_launch(const K2Args& a, cudaStream_t s);
cudaError_t scf_prep_launch(const PrepArgs& a, cudaStream_t s);
cudaError_t scf_k3_launch(int precision, const K3Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s);
