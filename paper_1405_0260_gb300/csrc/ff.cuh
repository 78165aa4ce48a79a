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
//
// For 2^-100 <= |x| < 2^88 (and zero) the split is taken from the bits with
// 32-bit integer operations: hi = the top 24 bits of the 53-bit significand,
// rounded to nearest even on the 29 bits below; lo = that 29-bit remainder less
// the rounding increment, a signed integer converted to float (one rounding)
// and scaled by 2^(E-52) in two exact power-of-two steps.  The result is
// bit-identical to rounding x and x - hi in float64, without a float64
// instruction (those run at ~1/64 of the float32 rate on this GPU).  Other
// values take the float64 form.
__device__ __forceinline__ FF ff_split(double x) {
  const unsigned bh = (unsigned)__double2hiint(x), bl = (unsigned)__double2loint(x);
  const unsigned sgn = bh >> 31;
  const int E = (int)((bh >> 20) & 0x7FFu) - 1023;
  FF r;
  if (E >= -100 && E <= 87) {
    unsigned H = (((bh & 0xFFFFFu) | 0x100000u) << 3) | (bl >> 29);
    const int R = (int)(bl & 0x1FFFFFFFu);
    const bool up = R > 0x10000000 || (R == 0x10000000 && (H & 1u));
    int L = up ? R - 0x20000000 : R;  // x - hi in units of 2^(E-52), |L| <= 2^28
    H += up ? 1u : 0u;
    int Eh = E;
    if (H == 0x1000000u) {  // rounded up to the next power of two
      H = 0x800000u;
      ++Eh;
    }
    r.hi = __uint_as_float((sgn << 31) | ((unsigned)(Eh + 127) << 23) | (H & 0x7FFFFFu));
    if (sgn) L = -L;
    r.lo = __fmul_rn(__fmul_rn(__int2float_rn(L), __uint_as_float((unsigned)(E + 139) << 23)), 0x1p-64f);
    return r;
  }
  if (((bh << 1) | bl) == 0u) return FF{__uint_as_float(sgn << 31), 0.0f};  // +-0
  r.hi = __double2float_rn(x);
  r.lo = __double2float_rn(__dsub_rn(x, static_cast<double>(r.hi)));
  return r;
}

// A float as a float64, exactly, from its bits (zero, normal); other values
// (subnormal, infinite, NaN) by conversion.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xFFu;
  if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  if (ex == 0u || ex == 0xFFu) return static_cast<double>(f);
  return __hiloint2double((int)((u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7FFFFFu) >> 3)), (int)(u << 29));
}

__device__ __forceinline__ FF ff_from_float(float x) { return FF{x, 0.0f}; }

// hi + lo rounded to float64 (one float64 addition; the conversions are exact).
__device__ __forceinline__ double ff_to_double(FF a) { return f2d_exact(a.hi) + f2d_exact(a.lo); }

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
