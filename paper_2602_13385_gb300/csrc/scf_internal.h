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
  int nc, n_prog;
  int mode;
  double dt;
  double* com;              // [n_prog][6] (step mode with host)
  ScfHostParams host;
};

// Kernel 3: acceleration (+ tidal term) and, in step mode, the closing half kick.
struct K3Args {
  const void* pos;
  void* vel;
  void* acc;
  const double* A;          // [n_prog][2*NC]
  const double* com;        // [n_prog][6] or null
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
  int threads;
  size_t smem;
};

void scf_make_norm(int nmax, int lmax, double* norm);

// Each kernel translation unit keeps its own copy of the constant tables.
cudaError_t scf_upload_const_coeffs(const ScfConst* t);
cudaError_t scf_upload_const_forces(const ScfConst* t);

// Launch configuration (threads, dynamic shared memory) of each kernel for
// the given sizes; sets the shared-memory attribute of the instantiation.
cudaError_t scf_k1_prepare(int precision, int lmax, int nmax, ScfLaunchInfo* info, int* blocks_per_sm);
cudaError_t scf_k3_prepare(int precision, int lmax, int nmax, ScfLaunchInfo* info, int* blocks_per_sm);

cudaError_t scf_k1_launch(int precision, const K1Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s);
cudaError_t scf_k2_launch(const K2Args& a, cudaStream_t s);
cudaError_t scf_k3_launch(int precision, const K3Args& a, int blocks, const ScfLaunchInfo& info, cudaStream_t s);
