// Float-float ("double-single") arithmetic: a value carried as the unevaluated
// sum h + l of two floats with |l| <= ulp(h)/2, about 48 significant bits.
// GB300 retires 64 single-precision FMAs for each double-precision one, so a
// double-accuracy computation written with these operations (each 3-12
// single-precision instructions) runs several times faster than in native
// double precision.
//
// The error-free transformations (Knuth's TwoSum, Dekker's FastTwoSum, the
// FMA-based exact product) are written with the _rn intrinsics, which the
// compiler never contracts into FMAs (a contraction would break them).
// Relative error of one operation: about 2^-44 (add) and 2^-45 (multiply).
#pragma once

#include <cuda_runtime.h>

struct FF {
  float h, l;
};

__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// |a| >= |b| (or a = 0)
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ FF ff_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ FF ff_from(float x) { return {x, 0.f}; }

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ FF ff_neg(FF a) { return {-a.h, -a.l}; }

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const FF s = ff_two_sum(a.h, b.h);
  return ff_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return ff_fast_two_sum(p, e);
}

__device__ __forceinline__ FF ff_mul(FF a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = fmaf(a.h, b, -p);
  e = fmaf(a.l, b, e);
  return ff_fast_two_sum(p, e);
}

// a b + c
__device__ __forceinline__ FF ff_fma(FF a, FF b, FF c) { return ff_add(ff_mul(a, b), c); }

// An unnormalised accumulator for long sums of products: the high part is
// carried with TwoSum, every rounding error and low-order product term goes
// to the low part; ff_acc_done renormalises.
__device__ __forceinline__ void ff_acc_prod(FF& acc, FF a, FF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const FF s = ff_two_sum(acc.h, p);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
}

__device__ __forceinline__ FF ff_acc_done(FF acc) { return ff_two_sum(acc.h, acc.l); }
