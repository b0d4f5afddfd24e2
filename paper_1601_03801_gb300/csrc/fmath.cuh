// Overloads of the few math functions the generic kernels use, for FP32 and FP64
// force words (CUDA's own correctly rounded sqrt and its pow/floor).
#pragma once
#include <cuda_runtime.h>

namespace sedi {
__device__ __forceinline__ float xsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double xsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float xpow(float a, float b) { return powf(a, b); }
__device__ __forceinline__ double xpow(double a, double b) { return pow(a, b); }
// Power for the drag correlation in the FP32 forms: CUDA's fast __powf (2^(b log2 a) with
// hardware approximations; relative error ~1e-6 for a in [0.1, 1], b <= 4.14).
__device__ __forceinline__ float xpow_drag(float a, float b) { return __powf(a, b); }
__device__ __forceinline__ double xpow_drag(double a, double b) { return pow(a, b); }
// Quotient and reciprocal square root in the force word.  FP32: CUDA's fast forms
// (__fdividef, rsqrtf: ~2 ulp, so ~2e-7 relative, far inside the 1e-5 force tolerance;
// __fdividef returns 0 for |b| > 2^126, far outside any value here).  FP64: correctly
// rounded, for the parity form.
__device__ __forceinline__ float xdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double xdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float xrsqrt(float a) { return rsqrtf(a); }
__device__ __forceinline__ double xrsqrt(double a) { return 1.0 / sqrt(a); }
// Square root of a positive argument in the force word.  FP32: a * rsqrtf(a) (a few
// ulp, ~3e-7 relative, inside the 1e-5 force tolerance), with the argument raised to
// the smallest normal number so that a denormal overlap cannot meet a flushed
// reciprocal; FP64: correctly rounded.
__device__ __forceinline__ float xsqrt_pos(float a) {
  a = fmaxf(a, 1.17549435e-38f);
  return a * rsqrtf(a);
}
__device__ __forceinline__ double xsqrt_pos(double a) { return sqrt(a); }
__device__ __forceinline__ float xlog(float a) { return logf(a); }
__device__ __forceinline__ double xlog(double a) { return log(a); }
__device__ __forceinline__ float xfloor(float a) { return floorf(a); }
__device__ __forceinline__ double xfloor(double a) { return floor(a); }
// a * b + c with a single rounding, written out so that the result does not depend
// on the compiler's contraction choices (which can change with register budgets)
__device__ __forceinline__ float xfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double xfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float xabs(float a) { return fabsf(a); }
__device__ __forceinline__ double xabs(double a) { return fabs(a); }
__device__ __forceinline__ bool xisfinite(float a) { return isfinite(a); }
__device__ __forceinline__ bool xisfinite(double a) { return isfinite(a); }
}  // namespace sedi
