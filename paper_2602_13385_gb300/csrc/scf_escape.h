// Internal interface of the escape-physics kernels (scf_escape.cu): the
// boundedness test, the energy-based Lagrange radius with its coefficient-set
// mask, and the tidal scales at the cluster centre (Sec. 2.2).  Not part of
// the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "scf_device.cuh"

// Upper bound on the number of j-segments the pair kernel splits each
// progenitor into (more blocks when the progenitors are small).
constexpr int kBoundMaxSplit = 16;

struct BoundArgs {
  const void* pos;             // [N][4] float (mixed) or double
  const void* vel;             // [N][4]
  const int64_t* prog_off;     // [n_prog + 1] particle offsets
  int n_prog;
  int64_t n_total;
  int f32;                     // particle arrays are float4
  int split;                   // j-segments per progenitor
  double G, kin, frac;
  double* part;                // [split][N] partial sums of m_j / r_ij
  unsigned long long* key;     // [N] bits of r^2
  double* E_out;               // [N] energies, or null
  uint8_t* bound;              // [N] 1 = bound
  uint8_t* mask;               // [N] 1 = r <= r_x, or null
  double* stats;               // [n_prog][4] = (n_bound, M_bound, r_x, n_in_set)
};

struct TidalArgs {
  const double* com;           // [n_prog][6] centre (R, V), or null (R = 0)
  const double* M_c;           // cluster masses with stride M_stride, or null (r_t = 0)
  int M_stride;
  int n_prog;
  double G, eta;
  ScfHostParams host;
  double* out;                 // [n_prog][16]
};

// j-segments per progenitor for a block map of i_chunks blocks in total.
int scf_bound_split(int64_t i_chunks, int n_sm);
// i-particles per block of the pair kernel (f32: single-precision particles).
int64_t scf_bound_chunk(int f32);
// max_chunks: i-blocks of the largest progenitor.
cudaError_t scf_bound_launch(const BoundArgs& a, int64_t max_chunks, cudaStream_t s);
cudaError_t scf_tidal_launch(const TidalArgs& a, cudaStream_t s);
// The selection alone (bound flags and radius keys from a previous
// scf_bound_launch; mask may be null).
cudaError_t scf_select_launch(const BoundArgs& a, cudaStream_t s);
// b_prog[p] = r_x / scf_half_mass_divisor(alpha) from the stats of a selection at
// frac = 0.5: r_x / (1 + sqrt 2) at alpha = 1, r_x (2^(1/(alpha+1)) - 1)^alpha otherwise.
double scf_half_mass_divisor(double alpha);
cudaError_t scf_retune_b_launch(const double* stats, double* b_prog, int n_prog, double alpha, cudaStream_t s);
