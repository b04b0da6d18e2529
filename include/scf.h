/*
 * scf.h — C ABI of the GB300 self-consistent-field (SCF) gravity step.
 *
 * The method is the basis-expansion N-body scheme of KRIOS II
 * (arXiv:2602.13385, Sec. 2): the cluster potential is expanded in a
 * bi-orthogonal basis (Eq. 1a-2), the expansion coefficients are a
 * mass-weighted sum over particles (Eq. 3b), every particle moves in the
 * expansion's field plus the tidal field of an analytic host galaxy (Sec. 2.1,
 * App. A), and the radial basis is the Zhao family of Eq. 4 (alpha = 1, the
 * Hernquist-Ostriker Gegenbauer basis, by default; any alpha in
 * SCF_ALPHA_MIN..SCF_ALPHA_MAX), in units with G given by the caller
 * (Henon units: G = 1).
 *
 * All compute runs in CUDA kernels on one GPU (sm_103a).  The library does not
 * fall back to the CPU: every call that cannot run on the device returns an
 * error code.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Coefficients.  Real form of the expansion:
 *   psi(x) = G sum_{n,l} Phi_nl(r) sum_{m=0..l} P_l^m(cos th) [S_nlm cos(m ph) + T_nlm sin(m ph)]
 *   Phi_nl(r) = -(1/b) s^l (1+s)^-(2l+1) C_n^(2l+3/2)((s-1)/(s+1)),  s = r/b,
 *   S_nlm, T_nlm = (2 - delta_m0)/I_nl N_lm^2 sum_k w_k m_k Phi_nl(r_k) P_l^m(cos th_k) {cos, sin}(m ph_k)
 * with P_l^m carrying the Condon-Shortley phase, N_lm^2 = (2l+1)/(4 pi)
 * (l-m)!/(l+m)! and I_nl = int r^2 rho_nl Phi_nl dr the Hernquist-Ostriker
 * normalisation.  This is Eq. 3b with the paper's bi-orthonormal basis
 * rescaled by sqrt|I_nl|; the potential is identical.
 * A coefficient vector is [S | T], each half NC = (nmax+1)(lmax+1)(lmax+2)/2
 * doubles, entry (n, l, m) at n*(lmax+1)(lmax+2)/2 + l(l+1)/2 + m.  T_nl0 = 0.
 * With several progenitors the vectors are stacked: [n_prog][2*NC].
 *
 * Particles.  Device pointers, 4 components per particle, 16-byte aligned,
 * particles of progenitor p at indices [offsets[p], offsets[p+1]):
 *   pos = (x, y, z, m) in the cluster frame (origin at the cluster centre R),
 *   vel = (vx, vy, vz, unused), velocities relative to the frame,
 *   acc = (ax, ay, az, psi_SCF) — acceleration incl. the tidal term; the 4th
 *         component is the expansion's potential only.
 * Element type: double for SCF_FP64, float for SCF_MIXED.
 *
 * Centre of mass.  com = [n_prog][6] doubles (R, V) in the host frame (device
 * pointer), always double precision.
 *
 * Streams and ownership.  Every call enqueues work on the stream given to
 * scf_init and returns without waiting, except those whose description says
 * they synchronise (scf_status, scf_free, scf_autotune, scf_set_option,
 * scf_set_mask, scf_evolve).  The
 * caller owns all particle, coefficient and centre buffers; the handle owns
 * its workspace (block partials, block maps, a coefficient buffer, the status
 * word), allocated once in scf_init.  No call allocates after scf_init.
 *
 * Errors.  Every entry point returns 0 (SCF_OK) or a negative SCF_ERR_* code;
 * scf_strerror gives a static description.  Device-side problems (non-finite
 * positions) set bits of a status word read by scf_status; kernels never trap.
 */
#ifndef SCF_GB300_H
#define SCF_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define SCF_OK 0
#define SCF_ERR_INVALID_ARG (-1)   /* a size, count, offset or option is out of range */
#define SCF_ERR_NULL_POINTER (-2)  /* a required pointer is NULL */
#define SCF_ERR_MISALIGNED (-3)    /* a particle pointer is not 16-byte aligned */
#define SCF_ERR_UNSUPPORTED (-4)   /* lmax/nmax beyond the compiled limits, alpha out of range, a variant with alpha != 1 */
#define SCF_ERR_CUDA (-5)          /* a CUDA runtime call or kernel launch failed */
#define SCF_ERR_OUT_OF_MEMORY (-6) /* workspace allocation failed in scf_init */
#define SCF_ERR_DEVICE_STATUS (-7) /* scf_status found device-side problems */
#define SCF_ERR_TOO_LARGE (-8)     /* the problem does not fit the static scratch of scf_coeffs_noalloc */
#define SCF_ERR_ADJOINT_FP64 (-9)  /* scf_adjoint_level called on a mixed-precision handle */

/* ---- device status bits (scf_status) ---- */
#define SCF_STATUS_NONFINITE_POS 1 /* a particle position was NaN/Inf; it was skipped */
#define SCF_STATUS_NONFINITE_ACC 2 /* an acceleration came out NaN/Inf */

/* ---- limits of the compiled kernels ---- */
#define SCF_MAX_LMAX 12
#define SCF_MAX_NMAX 40
#define SCF_MAX_HOST_COMPONENTS 8
#define SCF_ALPHA_MIN 0.1 /* range of the Zhao exponent alpha (Eq. 4) */
#define SCF_ALPHA_MAX 4.0

/* ---- precision (Sec. 2 leaves it open) ---- */
#define SCF_FP64 0  /* every step in double precision */
#define SCF_MIXED 1 /* basis and field in float; coefficient sums, centre orbit and tidal term in double */

/* ---- host components (App. A); parameters in the caller's units ---- */
#define SCF_HOST_HERNQUIST 1 /* M = total mass, a = scale radius:  psi = -G M / (r + a)            */
#define SCF_HOST_NFW 2       /* M = scale mass M_NFW, a = r_s:     psi = -G M ln(1 + r/r_s) / r     */
#define SCF_HOST_MN 3        /* M, a = scale length, b = height:   psi = -G M / sqrt(R^2 + (sqrt(z^2+b^2)+a)^2) */
#define SCF_HOST_POWCUT 4    /* M = total mass M_b, a = cut-off radius r_c, b = power-law index alpha (0 <= alpha < 2):
                              * rho ~ (r_c/r)^alpha exp(-(r/r_c)^2) (the MWPotential2014 bulge, App. A),
                              * psi = G M_b/Gamma(s) (gamma(1 - alpha/2, x)/r_c - gamma(s, x)/r),
                              * s = (3 - alpha)/2, x = (r/r_c)^2, gamma the lower incomplete gamma function.
                              * The adjoint (scf_adjoint_level) does not take this component. */

typedef struct scf_host_component {
  int kind;
  double M, a, b;
} scf_host_component;

typedef struct scf_config {
  int nmax;          /* radial truncation, 0 <= nmax <= SCF_MAX_NMAX */
  int lmax;          /* angular truncation, 0 <= lmax <= SCF_MAX_LMAX */
  double alpha;      /* Zhao exponent of Eq. 4, SCF_ALPHA_MIN..SCF_ALPHA_MAX: 1 = Hernquist-Ostriker
                      * basis (all kernels), 1/2 = Clutton-Brock; see "Radial family" below */
  double b;          /* basis scale length b of Eq. 4 (> 0); per-progenitor values may override */
  double G;          /* gravitational constant (1 in Henon units) */
  double dt;         /* leapfrog step for scf_step */
  int precision;     /* SCF_FP64 or SCF_MIXED */
  int n_host;        /* number of host components, 0 = isolated cluster (no tidal term) */
  scf_host_component host[SCF_MAX_HOST_COMPONENTS];
} scf_config;

typedef struct scf_handle scf_handle;

/* Radial family (Eq. 4; Zhao 1996).  With s = r/b, t = s^(1/alpha),
 * xi = (t-1)/(t+1), a_l = (2l+1) alpha and lambda_l = a_l + 1/2, the radial
 * functions are  U_nl(r) = -(1/b) s^l (1+t)^(-a_l) C_n^(lambda_l)(xi),  the
 * lowest one the U_00 ~ (1 + (r/b)^(1/alpha))^(-alpha) that Eq. 4 prints.
 * alpha = 1 runs every kernel and option.  Any other alpha runs the general
 * coefficient and field kernels (recurrence tables of the handle's alpha in
 * its workspace): SCF_OPT_K1_TILE accepts 128 and (SCF_MIXED, the default
 * there) 0, SCF_OPT_K3_BLOCK only 128, the
 * float-float variants and the adjoint return SCF_ERR_UNSUPPORTED, and
 * scf_coeffs_noalloc takes alpha = 1 only.  An alpha whose tables overflow
 * single precision at the handle's (nmax, lmax) returns SCF_ERR_UNSUPPORTED
 * from scf_init; alpha <= 0 or non-finite returns SCF_ERR_INVALID_ARG.  At
 * r = 0 the l = 0 radial force has no direction (for alpha > 1 it grows
 * without bound towards the centre) and is left out there. */

/* Creates a handle for n_prog progenitors (independent clusters sharing the
 * configuration) whose particles occupy [offsets[p], offsets[p+1]) of every
 * particle array.
 *   cfg        host pointer, copied.
 *   offsets    host pointer to n_prog+1 non-decreasing int64, offsets[0] = 0.
 *   b_per_prog host pointer to n_prog basis scales, or NULL to use cfg->b.
 *   stream     a cudaStream_t (NULL = legacy default stream) on the current device.
 * Allocates the workspace on the current device and writes the handle to *out.
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_INVALID_ARG, SCF_ERR_UNSUPPORTED,
 * SCF_ERR_OUT_OF_MEMORY, SCF_ERR_CUDA; *out is untouched on error. */
int scf_init(const scf_config* cfg, int n_prog, const int64_t* offsets, const double* b_per_prog, void* stream,
             scf_handle** out);

/* Expansion coefficients of Eq. 3b for every progenitor: the particle sum
 * (kernel 1: per-block partial sums) followed by a deterministic fixed-order
 * reduction and the normalisation (kernel 2).  Bitwise reproducible for a
 * given handle.
 *   pos   device, particle positions (see Particles).
 *   mask  device, one byte per particle, 0 = leave out of the sum; NULL = all.
 *   A_out device, [n_prog][2*NC] doubles.
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_MISALIGNED, SCF_ERR_CUDA. */
int scf_coeffs(scf_handle* h, const void* pos, const uint8_t* mask, double* A_out);

/* Acceleration -grad psi_SCF (Eq. 1a) at every particle from the given
 * coefficients, plus the tidal acceleration of the accelerating, non-rotating
 * cluster frame (Sec. 2.1) a_host(R + x) - a_host(R) when the configuration
 * has host components.
 *   pos  device positions; A device [n_prog][2*NC] doubles;
 *   com  device [n_prog][6] doubles (only R is read); may be NULL without host;
 *   acc  device output (see Particles).
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_MISALIGNED, SCF_ERR_CUDA. */
int scf_forces(scf_handle* h, const void* pos, const double* A, const double* com, void* acc);

/* nsteps kick-drift-kick leapfrog steps of size cfg->dt.  Each step: half
 * kick and drift of every particle, the same for the centre orbit R, V in
 * the host field (double precision), coefficients of the new positions
 * (all particles), accelerations at the new positions, half kick.
 *   pos, vel, acc device particle arrays, updated in place.  On entry acc
 *                 must hold the acceleration at pos (from scf_forces or the
 *                 previous scf_step); on return it holds the one at the new pos.
 *   com           device [n_prog][6] doubles, updated in place (may be NULL
 *                 without host components).
 * The coefficients of the last step can be read with scf_last_coeffs.
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_MISALIGNED, SCF_ERR_INVALID_ARG
 * (nsteps < 0), SCF_ERR_CUDA. */
int scf_step(scf_handle* h, void* pos, void* vel, void* acc, double* com, int nsteps);

/* One leapfrog step (as scf_step with nsteps = 1, same kernels and results)
 * for a caller whose state lives in host memory: on return (after the
 * handle's stream) the host arrays hold the stepped state.
 * When every host array is mapped page-locked memory (cudaHostAlloc, or
 * torch pin_memory, under unified addressing) the step's kernels read and
 * write the host arrays in place over the host link: the transfers happen
 * inside the kernels, overlapped with their arithmetic, and the device arrays
 * are not used (they may be NULL); in SCF_MIXED with the register-tiled
 * kernel 1 the drifted positions and half-kicked velocities between kernels
 * 1 and 3 are kept in a device copy owned by the handle (2 x 16 bytes per
 * particle, allocated by the first such call, freed by scf_free), so the
 * host link carries the state in once and out once.  Otherwise the state is staged through the
 * device arrays: copied in on a second stream of the handle, kernels 1 and 2,
 * then the positions and the centres copied back while kernel 3 runs, which
 * is launched in `chunks` pieces of its block map so that each piece's
 * velocities and accelerations go back while the next piece runs.  The copy
 * stream and its events are created by the first staged call and freed by
 * scf_free; the handle's stream waits for the copies, so a synchronisation of
 * the handle's stream covers the whole call.
 *   pos, vel, acc, com           device arrays as for scf_step (staged form only).
 *   host_pos, host_vel, host_acc host arrays of the same layout: read, then
 *                                overwritten with the new state (acc: the
 *                                acceleration at the new positions).
 *   host_com                     host [n_prog][6] doubles, read and updated
 *                                (NULL without host components).
 *   chunks                       1..SCF_STAGE_MAX_CHUNKS (staged form).
 * Host arrays must stay valid until the handle's stream has finished.
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_MISALIGNED, SCF_ERR_INVALID_ARG
 * (chunks out of range), SCF_ERR_OUT_OF_MEMORY (the device copy), SCF_ERR_CUDA. */
#define SCF_STAGE_MAX_CHUNKS 32
int scf_step_host(scf_handle* h, void* pos, void* vel, void* acc, double* com, void* host_pos, void* host_vel,
                  void* host_acc, double* host_com, int chunks);

/* Handle options.
 *   SCF_OPT_GRAPHS    1 (default) = scf_step replays a captured CUDA graph per
 *                     step where it can, 0 = plain kernel launches.
 *   SCF_OPT_K1_TILE   particles per tile (= threads per block) of the
 *                     coefficient kernel: 64, 128 (default) or 256.
 *   SCF_OPT_K3_BLOCK  threads per block of the field kernel: 64, 128
 *                     (default), 256, or (SCF_MIXED only, else
 *                     SCF_ERR_UNSUPPORTED) 320.
 *   SCF_OPT_K1_VARIANT 0 = the coefficient kernel with one thread per output
 *                     and SCF_OPT_K1_TILE particles per tile (the double-
 *                     precision default); 1 = the register-tiled kernel
 *                     (register output tiles per thread, 21 x 3 at
 *                     nmax = 20, 11 x 5 at nmax = 10, 7 x 8 otherwise, over 60-particle
 *                     tiles; SCF_MIXED only, its default); 2 = (SCF_FP64
 *                     only) the one-thread-per-output kernel in float-float
 *                     arithmetic on the single-precision pipe (128-particle
 *                     tiles only; partial sums within about 1e-13 of the
 *                     double kernel's).  Reading SCF_OPT_K1_TILE gives 0
 *                     while variant 1 is in use.
 *   SCF_OPT_K3_VARIANT 0 = the field kernel in the handle's precision (the
 *                     default); 1 = (SCF_FP64 only) the field kernel in
 *                     float-float arithmetic on the single-precision pipe:
 *                     the same results to about 1e-13 relative, the
 *                     per-particle set-up, tidal difference and kick in
 *                     double; 128-thread blocks only (other
 *                     SCF_OPT_K3_BLOCK values return SCF_ERR_UNSUPPORTED
 *                     while it is selected).  The adjoint always uses the
 *                     double kernel.  The autotuner keeps the variant.
 *   SCF_OPT_CENTRE_AHEAD 1 (default) = scf_step computes the next step's
 *                     centre kick-drift-kick (Sec. 2.1, the orbit of R) on a
 *                     second stream beside kernel 3, and kernel 2 of the next
 *                     step takes it when the state it steps is bitwise the
 *                     one that was stepped ahead (same dt); 0 = kernel 2
 *                     always computes it.  Either way the results are
 *                     bitwise the same.
 * Setting a tile or block size synchronises the stream and rewrites the block
 * maps in the workspace (sized in scf_init for every allowed value).
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_INVALID_ARG (unknown option or value),
 * SCF_ERR_UNSUPPORTED (the size does not fit this configuration), SCF_ERR_CUDA. */
#define SCF_OPT_GRAPHS 1
#define SCF_OPT_K1_TILE 2
#define SCF_OPT_K3_BLOCK 3
#define SCF_OPT_K1_VARIANT 4
#define SCF_OPT_K3_VARIANT 5
#define SCF_OPT_CENTRE_AHEAD 6
int scf_set_option(scf_handle* h, int option, int value);
int scf_get_option(const scf_handle* h, int option, int* value);

/* Autotuner: times every allowed SCF_OPT_K1_TILE with the coefficient pass
 * and every SCF_OPT_K3_BLOCK with the field pass of a step (its closing half
 * kick applied to acc, which stands in for the velocities) (2 warm-up + reps timed calls
 * each, CUDA events on the handle's stream) on the caller's particles, and
 * keeps the fastest of each (in SCF_MIXED the register-tiled kernel 1 is a
 * fourth candidate).  pos, com as for scf_forces; acc is overwritten.
 * ms_out (host, nullable) receives 8 average times in milliseconds
 * (tiles 64, 128, 256 of kernel 1, then blocks 64, 128, 256 of kernel 3, then
 * the register-tiled kernel 1, then blocks of 320 of kernel 3; 0 for a shape
 * that does not fit or apply).  Synchronises the stream; creates CUDA events.
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_MISALIGNED, SCF_ERR_INVALID_ARG
 * (reps < 1), SCF_ERR_CUDA. */
int scf_autotune(scf_handle* h, const void* pos, const double* com, void* acc, int reps, double* ms_out);

/* One level of the reverse (adjoint) sweep through scf_step, in double
 * precision.  Differentiates the kick-drift-kick of Sec. 2.1, with
 *   a_k(x, R) = f(x_k; A(x)) + a_host(R + x_k) - a_host(R),
 * A(x) the coefficients of Eq. 3b (every particle's mass m_k = pos.w
 * counted, no mask) and the centre (R, V) stepped by the host alone.
 * Let a forward run hold states x_t, com_t (t = 0..T, after t calls of
 * scf_step with one step each).  Reverse sweep, for t = T down to 0:
 *   scf_adjoint_level(h, x_t, com_t, w_t, t > 0, xbar, vbar, combar, thetabar)
 * with w_T = w_0 = dt/2 and w_t = dt otherwise (a(x_t) enters the closing
 * kick of step t and the opening kick of step t+1).  Before the first call
 * xbar, vbar, combar hold dL/dx_T, dL/dv_T, dL/d(R_T, V_T) and thetabar 0;
 * after the last call they hold dL/dx_0, dL/dv_0, dL/d(R_0, V_0) and
 * dL/d(GM_c, a_c).  One call does, with d_k = w_t vbar_k:
 *   xbar_k += (da_k/dx_k)^T d_k      (Hessian of the expansion potential at
 *                                     fixed coefficients, plus T(R + x_k) d_k),
 *   xbar_k += m_k f(x_k; A^J),  A^J = sum_i (dB(x_i)/dx_i) d_i   (through A),
 *   Rbar += sum_k (T(R + x_k) - T(R)) d_k + w_t T(R) Vbar,
 *   thetabar += the same pull-back through the host parameters,
 * then, if drift != 0, undoes the drift: vbar += dt xbar, Vbar += dt Rbar.
 * T is the host's tidal tensor (the Jacobian of a_host).
 *   pos       device [N][4] doubles, x_t with masses (as for scf_step).
 *   com       device [n_prog][6], (R_t, V_t); NULL allowed without host.
 *   weight    w_t;  drift  0 at t = 0, else 1.
 *   xbar, vbar  device [N][4] doubles, updated (4th component untouched).
 *   combar    device [n_prog][6] doubles (Rbar, Vbar), updated.
 *   thetabar  device [n_prog][2*n_host] doubles, per progenitor and host
 *             component c: (dL/dGM_c, dL/da_c) accumulated, with GM_c = G M_c
 *             and a_c the scale length of App. A (NFW r_s, Hernquist a,
 *             Miyamoto-Nagai a); summing over progenitors is the caller's.
 * Derivatives are exact up to rounding (dual numbers in the kernels); at a
 * particle exactly at r = 0 the own-position term of l = 1 is taken as 0.
 * Overwrites the handle's coefficient buffer (scf_last_coeffs) and the
 * captured step graph.  Launches 6 kernels (5 without host components).
 * Errors: SCF_ERR_ADJOINT_FP64, SCF_ERR_NULL_POINTER, SCF_ERR_MISALIGNED,
 * SCF_ERR_INVALID_ARG (weight not finite), SCF_ERR_UNSUPPORTED, SCF_ERR_CUDA. */
int scf_adjoint_level(scf_handle* h, const void* pos, const double* com, double weight, int drift, void* xbar,
                      void* vbar, double* combar, double* thetabar);

/* Energy diagnostic of every progenitor in its accelerating, non-rotating
 * frame (Sec. 2.1), in double precision whatever the handle's precision:
 *   E_out[p][0] = K = sum_k 1/2 m_k |v_k|^2
 *   E_out[p][1] = W = 1/2 sum_k m_k psi_SCF(x_k), psi_SCF read from acc.w
 *   E_out[p][2] = U = sum_k m_k [psi_host(R + x_k) - psi_host(R) + x_k . a_host(R)]
 *                 (the potential of the frame's tidal acceleration; 0 without host)
 *   E_out[p][3] = K + W + U
 * pos, vel, acc are the state layouts of scf_step (element type of the
 * precision); acc must hold the accelerations and potential at pos, as
 * scf_step and scf_forces leave them.  com as for scf_step (NULL allowed
 * without host components).  E_out is a device [n_prog][4] doubles.  The sums
 * run in a fixed order, so repeated calls give the same bits.  For an
 * isolated cluster K + W is the energy the self-consistent system conserves.
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_MISALIGNED, SCF_ERR_CUDA. */
int scf_energy(scf_handle* h, const void* pos, const void* vel, const void* acc, const double* com, double* E_out);

/* ---- Escape physics (Sec. 2.2; Sec. 3.1 footnote on the tidal radius) ---- */

/* Boundedness of every particle and the coefficient set of Eq. 3b.
 * Particle i of progenitor p is bound when its cluster-frame energy
 *   E_i = kin |v_i|^2 - sum_{j != i, j in p} G m_j / |x_i - x_j|
 * is negative (unsoftened direct summation over all particles of p; pairs at
 * zero separation and pairs with a non-finite separation add nothing, so a
 * particle with a non-finite position is never bound).  The footnote of
 * Sec. 2.2 prints kin = 1; kin = 1/2 is the standard specific energy.
 * r_x is the energy-based Lagrange radius: the k-th smallest cluster-frame
 * radius among p's bound particles, k = ceil(frac n_bound) (r_x = 0 when none
 * is bound); the coefficient set is r <= r_x (frac = 0.999 in the paper).
 * Radii are compared as r^2 = (x x + y y) + z z in double precision.
 * In double precision the pair terms are evaluated in float-float arithmetic
 * (each coordinate and mass split into two floats, 48 bits; a term's
 * relative error is about 1e-14 + 2^-48 |x| / r_ij) and blocks of 64 of them
 * are added in double.  In mixed precision each pair term and blocks of 64
 * of them are float (1/r the hardware approximation), added in double.  In
 * both, pairs whose r^2 lies outside the normal float range
 * [1.18e-38, 3.40e38] add nothing.
 *   pos, vel   device [N][4] in the handle's element type (16-byte aligned)
 *   kin        > 0 and finite;  frac in (0, 1]
 *   E_out      device [N] doubles (E_i), or NULL
 *   bound_out  device [N] bytes, 1 = bound (required when N > 0)
 *   mask_out   device [N] bytes, 1 = r <= r_x, or NULL
 *   stats_out  device [n_prog][4] doubles: n_bound, bound mass, r_x, size of the set
 * All sums have a fixed order (bitwise reproducible).  Cost O(sum_p N_p^2).
 * The workspace for it (8 (S+1) N bytes, S <= 16 pair-sum segments) is
 * reserved by scf_init.
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_MISALIGNED, SCF_ERR_INVALID_ARG, SCF_ERR_CUDA. */
int scf_bound(scf_handle* h, const void* pos, const void* vel, double kin, double frac, double* E_out,
              uint8_t* bound_out, uint8_t* mask_out, double* stats_out);

/* Tidal scales of every progenitor at its centre R = com[p][0..2] (Sec. 2.2):
 *   out[p][0..8]  T_ij = -d^2 psi_host / dx_i dx_j (row-major), from the host components
 *   out[p][9..11] eigenvalues l1 >= l2 >= l3 of T
 *   out[p][12]    |T|_F (Frobenius norm)
 *   out[p][13]    l1e = l1 - (l2 + l3)/2
 *   out[p][14]    r_t = (G M_c[p] / l1e)^(1/3) (Sec. 3.1 footnote); +inf when l1e <= 0;
 *                 0 when M_c is NULL
 *   out[p][15]    dt_int = sqrt(eta) (|T|_F^2 / 6)^(-1/4); +inf without host
 * com: device [n_prog][6] (NULL allowed without host components: R = 0);
 * M_c: device [n_prog] cluster masses or NULL; eta > 0 (1/400 in the paper);
 * out: device [n_prog][16] doubles.
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_INVALID_ARG, SCF_ERR_CUDA. */
int scf_tidal(scf_handle* h, const double* com, const double* M_c, double eta, double* out);

/* Sets the coefficient set used by scf_step's coefficient pass: a device
 * [N] byte mask (1 = the particle enters Eq. 3b), or NULL for all particles
 * (the default).  The handle keeps the pointer, not the bytes; the caller
 * keeps the buffer alive and may rewrite it between calls.  Changing the
 * pointer synchronises the stream and drops the captured step. */
int scf_set_mask(scf_handle* h, const uint8_t* mask);

typedef struct scf_escape_params {
  double kin;        /* kinetic factor of the boundedness test (0.5, or 1 as printed) */
  double frac;       /* the coefficient set is r <= r_x of this fraction (0.999) */
  double eta;        /* integration-timestep parameter (1/400) */
  int max_steps;     /* most leapfrog steps per integration timestep (>= 1) */
  int retune_every;  /* complete refresh every this many integration timesteps, the
                        first included (the paper: 5); 0 = never.  It sets each
                        progenitor's b (alpha fixed) so that the lowest-order density
                        of the family, whose enclosed mass is (t/(1+t))^(alpha+1),
                        has half its mass inside r_50, the energy-based Lagrange
                        radius of half the bound stars: b = r_50 (2^(1/(alpha+1)) - 1)^alpha
                        (r_50 / (1 + sqrt 2) at alpha = 1) */
  int recentre;      /* 1: at each complete refresh, first scf_recentre (the SCF centre
                        and core velocity, 100 iterations at most, step tolerance
                        1e-12 b) with the current coefficient set, then scf_bound again
                        in the new frame; 0: the frame stays on the centre orbit */
  int retune_rule;   /* b at a complete refresh: 0 = the half-mass rule above,
                        1 = scf_retune_a000 (the maximum of a_000) over the coefficient set,
                        2 = scf_retune_alpha: alpha (shared) and b at the joint maximum of
                        a_000 over the coefficient set, alpha in [alpha_lo, alpha_hi] */
  double alpha_lo, alpha_hi; /* the exponent range of retune_rule 2 */
} scf_escape_params;

/* Basis scale of each progenitor at the maximum of a_000 in the bi-orthonormal
 * normalisation of Eq. 3a (Sec. 2: b tuned so that the lowest mode
 * approximates the cluster; alpha and the centre fixed).  With the lowest pair
 * scaled to unit self-energy, a_000(b) = Y_00 / sqrt(|I_00(1)| b) *
 * sum_k m_k g(r_k / b) over the coefficient set (mask; NULL = all),
 * g(s) = (1 + s^(1/alpha))^-alpha.  Search in ln b: 3 grids of 33 values, the
 * first over [b/8, 8b], each next over one step either side of the previous
 * best (the first best in grid order), the last best moved to the vertex of
 * the parabola through it and its neighbours; then 4 safeguarded Newton steps
 * on d ln a_000 / d ln b = 0 inside the last grid's bracket, so b is the
 * maximiser to rounding.  An empty set keeps b.  Updates the handle's scales
 * (scf_get_scales) on its stream; double-precision sums in a fixed order.
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_MISALIGNED, SCF_ERR_CUDA. */
int scf_retune_a000(scf_handle* h, const void* pos, const uint8_t* mask);

/* Exponent alpha of the radial family (Eq. 4) and every progenitor's b at the
 * joint maximum of a_000 (a complete refresh retunes both, Sec. 2.2): one
 * alpha for the handle, maximising the product of the progenitors' a_000,
 * each at its own maximising b_p(alpha) (the search of scf_retune_a000).  The
 * bi-orthonormal a_000 carries |I_00(alpha)|^(-1/2), I_00 = -(alpha + 1)
 * Gamma(2 alpha + 1) / (2^(4 alpha + 3) (alpha + 1/2) Gamma(alpha + 1/2)^2).
 * 17 values of ln alpha over [alpha_lo, alpha_hi] bracket the maximum; inside
 * the bracket the root of d/d alpha sum_p ln a_000,p (envelope theorem: the
 * partial derivative at b_p(alpha)) is found by the Illinois method.  The
 * handle then moves to that alpha: recurrence tables, normalisation and
 * field scales rebuilt, the general kernels selected for alpha != 1 (default
 * shapes, no float-float variants; the captured step is dropped), b_p set.
 * Synchronises the stream once per trial alpha (about 25).  Progenitors with an
 * empty set keep their b and take no part; with no set at all nothing
 * changes.  alpha_out (host, may be NULL) receives the exponent.
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_MISALIGNED, SCF_ERR_INVALID_ARG
 * (range empty or not positive), SCF_ERR_UNSUPPORTED (range outside
 * SCF_ALPHA_MIN..SCF_ALPHA_MAX, or tables of the found alpha not finite at
 * the handle's (nmax, lmax): the handle keeps its exponent), SCF_ERR_CUDA. */
int scf_retune_alpha(scf_handle* h, const void* pos, const uint8_t* mask, double alpha_lo, double alpha_hi,
                     double* alpha_out);

/* The handle's current exponent alpha of the radial family (changed by
 * scf_retune_alpha and by scf_evolve with retune_rule 2) into *alpha (host).
 * Errors: SCF_ERR_NULL_POINTER. */
int scf_get_alpha(const scf_handle* h, double* alpha);

/* Re-centring of the cluster frame (Sec. 2.1).  For every progenitor:
 * 1. the SCF centre x_c, where a_000 of the expansion about x_c (alpha, b fixed)
 *    is largest: a_000 is a positive multiple of sum_k m_k g(|x_k - x_c|/b),
 *    g(s) = (1 + s^(1/alpha))^-alpha, summed over the coefficient set (mask;
 *    NULL = all particles), and x_c is reached by the fixed-point (mean-shift)
 *    iteration x_c += sum m w (x_k - x_c) / sum m w, w = t (1+t)^(-alpha-1) / s^2,
 *    t = s^(1/alpha), from x_c = 0, until the step is <= tol * b or after
 *    max_iter steps; every particle is then shifted by -x_c;
 * 2. the core radius r_core^2 = sum_i rho_i^2 r_i^2 / sum_i rho_i^2 over all
 *    particles (rho_i the density of the set's expansion about x_c, Eq. 1b;
 *    particles at r = 0 left out) and the core velocity V_core = the
 *    mass-weighted mean velocity of the particles with r < r_core; every
 *    velocity is then shifted by -V_core;
 * 3. com (nullable) += (x_c, V_core), so host-frame positions and velocities
 *    are unchanged and the centre orbit continues from the new centre.
 *   pos, vel  device particles, shifted in place;  acc  device [N][4], used as
 *             scratch (overwritten; recompute the field before the next step);
 *   mask      device, one byte per particle, or NULL;
 *   max_iter  1..1000;  tol >= 0 (relative to b);
 *   out       host [n_prog][8] = (x_c, V_core, r_core, iterations), or NULL
 *             (then nothing is synchronised).
 * Sums in double precision in a fixed order (weights in the handle's
 * precision): reproducible bit for bit.  The handle's coefficients (scf_last_coeffs)
 * are those of the set about the new centre.
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_MISALIGNED, SCF_ERR_INVALID_ARG, SCF_ERR_CUDA. */
int scf_recentre(scf_handle* h, void* pos, void* vel, void* acc, double* com, const uint8_t* mask, int max_iter,
                 double tol, double* out);

/* nsteps leapfrog steps with the escape physics of Sec. 2.2.  At the start of
 * every integration timestep: scf_bound (bound flags, the mask r <= r_x and
 * stats, into the caller's buffers), the mask becomes the step's coefficient
 * set (scf_set_mask), at a complete refresh (retune_every) each progenitor's
 * b is retuned (scf_get_scales reads it), acc is recomputed at the current
 * positions from that set, and the next integration timestep is the smallest dt_int of scf_tidal
 * at the current centres with M_c = the bound mass; it runs
 * clamp(floor(dt_int / dt), 1, max_steps) steps of scf_step (fewer at the
 * end; max_steps without host components).  Reads dt_int back once per
 * integration timestep (a stream synchronisation).  On return the step mask
 * stays set to `mask`, bound/mask/stats describe the state at the start of
 * the last integration timestep, and *n_refresh (if not NULL) is the number
 * of integration timesteps.  Buffers as for scf_step and scf_bound.
 * Errors: those of scf_step and scf_bound; SCF_ERR_INVALID_ARG for a bad
 * parameter or dt <= 0. */
int scf_evolve(scf_handle* h, void* pos, void* vel, void* acc, double* com, int nsteps, const scf_escape_params* ep,
               uint8_t* bound, uint8_t* mask, double* stats, int* n_refresh);

/* Copies the basis scale b of every progenitor (device [n_prog] doubles, on
 * the handle's stream) into b_out: the value given to scf_init, or the last
 * one a complete refresh of scf_evolve set.
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_CUDA. */
int scf_get_scales(scf_handle* h, double* b_out);

/* Copies (device to device, on the handle's stream) the coefficients used by
 * the last force evaluation of scf_step into A_out ([n_prog][2*NC] doubles). */
int scf_last_coeffs(scf_handle* h, double* A_out);

/* Synchronises the handle's stream, writes the accumulated device status bits
 * (SCF_STATUS_*) to *status (may be NULL) and clears them.  Returns
 * SCF_ERR_DEVICE_STATUS if any bit was set, SCF_ERR_CUDA if the stream
 * reported an error, else SCF_OK. */
int scf_status(scf_handle* h, int* status);

/* Number of kernel launches one call of each entry point makes (for
 * accounting): which = 0 coeffs, 1 forces, 2 one step. */
int scf_launches_per_call(const scf_handle* h, int which);

/* Kernel timing with CUDA events recorded on the handle's stream around each
 * launch (the tracing of the three kernels).  scf_profile(h, 1) creates a
 * pool of event pairs (up to 4096 launches) and starts recording;
 * scf_profile(h, 0) stops recording and releases the pool.  Call it outside
 * the sections being timed: it creates CUDA events.
 * scf_profile_read synchronises the stream, writes the summed device time
 * in milliseconds and the number of recorded launches of kernel 1, 2 and 3
 * into ms[3] and launches[3] (host pointers; either may be NULL) and clears
 * the record.  Errors: SCF_ERR_NULL_POINTER, SCF_ERR_CUDA. */
int scf_profile(scf_handle* h, int enable);
int scf_profile_read(scf_handle* h, double* ms, int64_t* launches);

/* Coefficients of one cluster (same result as scf_coeffs with n_prog = 1)
 * for callers that cannot allocate device memory: code running inside an
 * arena or pool it must not grow, on a path where cudaMalloc is not allowed
 * or would synchronise the device, or a plugin handed device pointers but no
 * allocator.  The paper has no counterpart; this entry point only changes
 * where the scratch lives.
 *   cfg    host pointer; nmax, lmax, alpha (= 1), b and precision are used.
 *   n      number of particles (>= 0); pos device [n][4] (16-byte aligned,
 *          double for SCF_FP64, float for SCF_MIXED); mask device or NULL;
 *   A_out  device [2*NC] doubles;  stream  a cudaStream_t (NULL = default).
 * Allocates nothing: the block partial sums, block map and normalisation live
 * in one file-scope __device__ array of fixed size (SCF_NOALLOC_MAX_BLOCKS x
 * SCF_NOALLOC_MAX_COEFS doubles of partials, about 10.5 MiB in all) that every
 * GPU loading the library holds until the process exits.  The first call on
 * a device looks up that array's address (cudaGetSymbolAddress) and uploads
 * the recurrence tables, so make it before any stream capture.  Every call
 * rewrites all scratch it reads, but calls share the array: calls that
 * overlap on the GPU race and must be serialised by the caller.
 * Errors: SCF_ERR_TOO_LARGE when 2*NC > SCF_NOALLOC_MAX_COEFS (e.g. nmax = 40,
 * lmax = 12); SCF_ERR_NULL_POINTER, SCF_ERR_INVALID_ARG, SCF_ERR_UNSUPPORTED,
 * SCF_ERR_MISALIGNED, SCF_ERR_CUDA. */
#define SCF_NOALLOC_MAX_BLOCKS 320
#define SCF_NOALLOC_MAX_COEFS 4096
int scf_coeffs_noalloc(const scf_config* cfg, int64_t n, const void* pos, const uint8_t* mask, double* A_out,
                       void* stream);

/* Status of the last scf_coeffs_noalloc call on the current device: a
 * particle whose position or mass is NaN or infinite is left out of the sums
 * (the kernel never traps) and sets SCF_STATUS_NONFINITE_POS in the status
 * word of the static scratch; each call clears the word first.  This call
 * copies the word into *status (host, may be NULL) on `stream` and
 * synchronises that stream, allocating nothing; it reads whatever the last
 * call left, so calls of scf_coeffs_noalloc queued on other streams race
 * with it.  Before the first scf_coeffs_noalloc call on the device it
 * reports 0.  No counterpart in the paper.
 * Returns SCF_ERR_DEVICE_STATUS if a bit is set, SCF_ERR_CUDA on a CUDA
 * error, else SCF_OK. */
int scf_noalloc_status(void* stream, int* status);

/* Measured rate of independent FMA chains (8 per thread, 2048 threads per
 * SM) on the double-precision (SCF_FP64) or single-precision (SCF_MIXED)
 * pipe: the measured counterpart of the nominal non-tensor peak that the
 * roofline fractions of the coefficient and field kernels refer to.  No
 * counterpart in the paper (a measurement utility).  Synchronises the stream.
 *   iters      loop trips (16 x 8 FMAs per thread each); a few ms of work is
 *              about 1e4 (single) or 2e2 (double) on a GB300.
 *   stream     a cudaStream_t on the current device.
 *   flops_out  host, FLOP/s (FMA = 2) of the best of three launches.
 *   ms_out     host, duration of that launch (may be NULL).
 * Errors: SCF_ERR_NULL_POINTER, SCF_ERR_INVALID_ARG, SCF_ERR_CUDA. */
int scf_fma_peak(int precision, int iters, void* stream, double* flops_out, double* ms_out);

/* Releases the workspace (synchronising the stream first) and the handle.
 * NULL is accepted. */
int scf_free(scf_handle* h);

/* Static description of a return code. */
const char* scf_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* SCF_GB300_H */
