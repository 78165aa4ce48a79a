// Float-float ("double-float") arithmetic on the float32 pipes.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  On this GPU float64 arithmetic runs at ~1/56 of
// the float32 rate, so the float64-accurate parts of the mixed-precision path
// (refinement residuals, mass and Hamiltonian applies, Gram matrices and the
// rotation) are evaluated in this arithmetic instead.  The building blocks are
// the exact transformations of Dekker and Knuth: the exact product error of a
// fused multiply-add, fma(a, b, -a*b), and the error-free TwoSum.  Every step
// uses the _rn intrinsics so the compiler cannot contract a rounded product
// into a later addition (which would break the exactness the error terms need).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace paro {

struct FF {
  float hi, lo;
};

// Split of a float64 into hi + lo: hi is x rounded to the nearest float, lo the
// remainder x - hi (exact in float64: at most 29 significant bits) rounded to a
// float, so hi + lo carries ~48 bits of x and |lo| <= ulp(hi)/2.  Rounding hi
// to nearest (not toward zero) keeps it unbiased: kernels that use hi alone
// (the tensor-core Grams) then see rounding errors of either sign, which
// average out over a sum instead of shrinking every product by ~2^-24.
__device__ __forceinline__ FF ff_split(double x) {
  FF r;
  r.hi = __double2float_rn(x);
  r.lo = __double2float_rn(__dsub_rn(x, static_cast<double>(r.hi)));
  return r;
}

__device__ __forceinline__ FF ff_from_float(float x) { return FF{x, 0.0f}; }

// hi + lo in float64 (exact: the two significands do not overlap).
__device__ __forceinline__ double ff_to_double(FF a) { return static_cast<double>(a.hi) + static_cast<double>(a.lo); }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s += x * w (both float-float).  The product's hi*hi part is split exactly,
// the cross terms hi*lo and lo*hi are added in float32, lo*lo is dropped.
__device__ __forceinline__ void ff_mac(FF& s, FF x, FF w) {
  const float p = __fmul_rn(x.hi, w.hi);
  float e = __fmaf_rn(x.hi, w.hi, -p);
  e = __fmaf_rn(x.hi, w.lo, e);
  e = __fmaf_rn(x.lo, w.hi, e);
  float t, err;
  two_sum(s.hi, p, t, err);
  s.hi = t;
  s.lo = __fadd_rn(s.lo, __fadd_rn(err, e));
}

// s += x (float-float).
__device__ __forceinline__ void ff_add(FF& s, FF x) {
  float t, err;
  two_sum(s.hi, x.hi, t, err);
  s.hi = t;
  s.lo = __fadd_rn(s.lo, __fadd_rn(err, x.lo));
}

__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }

// Renormalise so that |lo| <= ulp(hi)/2 (Fast2Sum).
__device__ __forceinline__ FF ff_norm(FF a) {
  const float s = __fadd_rn(a.hi, a.lo);
  return FF{s, __fsub_rn(a.lo, __fsub_rn(s, a.hi))};
}

// Host: split a float64 constant the same way (hi rounded to nearest).
inline FF ff_split_host(double x) {
  FF r;
  r.hi = static_cast<float>(x);
  r.lo = static_cast<float>(x - static_cast<double>(r.hi));
  return r;
}

}  // namespace paro
