// Internal interfaces between the C ABI layer (scf_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "scf_device.cuh"

enum ScfMode { SCF_MODE_COEFFS = 0, SCF_MODE_STEP = 1 };

// Kernel 1: per-block partial sums of the coefficients (optionally after the
// half kick + drift of a leapfrog step).
struct K1Args {
  void* pos;          // [N][4] float or double (read; written in step mode)
  void* vel;          // [N][4] (step mode)
  const void* acc;    // [N][4] (step mode)
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
  // of the field kernel's element type, and a_host(R) per progenitor
  void* F_out;              // [n_prog][NC] float2 (f32) or double2, or null
  int f32;                  // element type of F_out
  const double* b_prog;
  double G;
  double* aR_out;           // [n_prog][4], or null
};

// Force coefficients and a_host(R) from given coefficients (scf_forces).
struct PrepArgs {
  const double* A;          // [n_prog][2*NC]
  const double* com;        // [n_prog][6] or null
  void* F_out;
  int f32;
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
  const void* F;            // [n_prog][NC] (cos, sin) force-coefficient pairs
  const double* com;        // [n_prog][6] or null (R is read)
  const double* aR;         // [n_prog][4] a_host(R)
  const int* blk_prog;
  const int64_t* blk_begin;
  const int64_t* blk_end;
  const double* b_prog;
  int nmax, lmax, nc, nlm;
  int mode;
  double G, dt;
  ScfHostParams host;
  unsigned* status;
};

struct ScfLaunchInfo {
  int threads;   // threads per block
  int tile;      // particles per tile (block ranges are whole tiles)
  size_t smem;   // dynamic shared memory per block
  int variant;   // kernel variant chosen by the prepare call
};

void scf_make_norm(int nmax, int lmax, double* norm);

// Each kernel translation unit keeps its own copy of the constant tables.
cudaError_t scf_upload_const_coeffs(const ScfConst* t);
cudaError_t scf_upload_const_forces(const ScfConst* t);

// Launch configuration (threads, dynamic shared memory) of each kernel for
// the given sizes; sets the shared-memory attribute of the instantiation.
// tp: kernel 1 particle tile (64, 128, 256); tb: kernel 3 block size (64, 128, 256).
cudaError_t scf_k1_prepare(int precision, int lmax, int nmax, int tp, ScfLaunchInfo* info, int* blocks_per_sm);
cudaError_t scf_k3_prepare(int precision, int lmax, int nmax, int tb, ScfLaunchInfo* info, int* blocks_per_sm);

cudaError_t scf_k1_launch(int precision, const K1Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s);
cudaError_t scf_k2_launch(const K2Args& a, cudaStream_t s);
cudaError_t scf_prep_launch(const PrepArgs& a, cudaStream_t s);
cudaError_t scf_k3_launch(int precision, const K3Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s);
