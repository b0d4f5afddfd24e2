// Double-float ("df64") arithmetic: a value is hi + lo with two FP32 words,
// |lo| <= ulp(hi)/2, giving a 48-bit significand that runs entirely on the FP32
// pipes.  GB300 executes FP64 at a small fraction of its FP32 rate, so the
// FP64-class quantities of the hot path (positions, velocities, spins,
// tangential springs, smoothing fields) use this type.
//
// Algorithms: Knuth's TwoSum, Dekker's Fast2Sum (quick_two_sum) and the
// FMA-based TwoProd, as described by Dekker (1971), Knuth (TAOCP vol. 2,
// Sec. 4.2.2) and Hida, Li & Bailey (2001).  The __f*_rn intrinsics keep the
// compiler from fusing or reassociating the error-free steps.
#pragma once
#include <cuda_runtime.h>

struct dd {
  float hi, lo;
};

__host__ __device__ inline dd dd_make(float hi, float lo) { return dd{hi, lo}; }

#ifdef __CUDACC__

__device__ __forceinline__ dd two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dd{s, e};
}

__device__ __forceinline__ dd quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return dd{s, e};
}

__device__ __forceinline__ dd two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return dd{p, e};
}

__device__ __forceinline__ dd dd_from_float(float a) { return dd{a, 0.0f}; }

__device__ __forceinline__ float dd_to_float(dd a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dd dd_from_double(double a) {
  float hi = __double2float_rn(a);
  float lo = __double2float_rn(a - (double)hi);
  return dd{hi, lo};
}

__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }

// Accurate addition (both error terms kept).
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  float e = __fadd_rn(s.lo, t.hi);
  dd u = quick_two_sum(s.hi, e);
  e = __fadd_rn(t.lo, u.lo);
  return quick_two_sum(u.hi, e);
}

__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

// Cheaper addition: one TwoSum on the high words, low words added plainly.  Its
// error is about 2^-44 of |a| + |b| (not of the result), which the contact
// geometry tolerates: the overlap s^2 - d^2 keeps ~1e-11 relative accuracy.
__device__ __forceinline__ dd dd_add_fast(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, e);
}

__device__ __forceinline__ dd dd_sub_fast(dd a, dd b) { return dd_add_fast(a, dd_neg(b)); }

__device__ __forceinline__ dd dd_add_f(dd a, float b) {
  dd s = two_sum(a.hi, b);
  float e = __fadd_rn(s.lo, a.lo);
  return quick_two_sum(s.hi, e);
}

__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, e);
}

__device__ __forceinline__ dd dd_mul_f(dd a, float b) {
  dd p = two_prod(a.hi, b);
  float e = __fmaf_rn(a.lo, b, p.lo);
  return quick_two_sum(p.hi, e);
}

// a + b * c with the product formed exactly.
__device__ __forceinline__ dd dd_fma_ff(dd a, float b, float c) {
  dd p = two_prod(b, c);
  return dd_add(a, p);
}

#endif  // __CUDACC__
