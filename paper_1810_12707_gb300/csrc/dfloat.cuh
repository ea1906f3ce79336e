// dfloat.cuh -- double-float arithmetic on the FP32 pipe: a real value is carried as the
// unevaluated sum hi + lo of two FP32 numbers (a 48-bit significand, about 3.6e-15 relative).
//
// On GB300 the FP32 pipe executes 72 times as many lane operations per second as the FP64 pipe,
// and a conversion between FP64 and FP32 costs as much as an FP64 operation, so a transform that
// must meet an FP64-level tolerance is cheaper in double-float arithmetic kept end to end (data
// stored as float pairs between passes) than in FP64.
//
// Published error-free transformations used (all operations round to nearest):
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b), v = fl(s - a),
//                                       e = fl(fl(a - fl(s - v)) + fl(b - v)),  a + b = s + e.
//   Fast2Sum (Dekker 1971), |a| >= |b|: s = fl(a + b), e = fl(b - fl(s - a)),    a + b = s + e.
//   TwoProd with a fused multiply-add:   p = fl(a b),   e = fma(a, b, -p),        a b = p + e.
// The sum and the product are "lazy": they return (hi, lo) without renormalising, so |lo| may
// exceed half an ulp of hi by a small factor; the error this adds is of the order of 2^-24 |lo|,
// i.e. a few units of 2^-48 of the operands' magnitudes, which is what an FFT's norm-wise error
// bound is measured against.  dfr_norm (Fast2Sum) renormalises before values are stored to global
// memory.  Every operation is written with the _rn intrinsics, which the compiler never merges
// into fused multiply-adds: a contraction would change the rounded results the error terms are
// computed from.
#pragma once

#include <cuda_runtime.h>

namespace mhd {

struct dfr {
  float hi, lo;
};

__host__ __device__ constexpr dfr dfr_const(double x) {
  return dfr{(float)x, (float)(x - (double)(float)x)};
}

// a + b, lazy: TwoSum of the high parts, the low parts and the rounding error summed in FP32
__device__ __forceinline__ dfr operator+(dfr a, dfr b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  return dfr{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}

__device__ __forceinline__ dfr operator-(dfr a) { return dfr{-a.hi, -a.lo}; }

__device__ __forceinline__ dfr operator-(dfr a, dfr b) { return a + (-b); }

// a * b, lazy: TwoProd of the high parts plus the cross terms (a.lo b.lo, about 2^-48 of the
// product, is dropped)
__device__ __forceinline__ dfr operator*(dfr a, dfr b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dfr{p, e};
}

// k * a for an FP32 number k (small integer wavenumbers, powers of two)
__device__ __forceinline__ dfr operator*(float k, dfr a) {
  const float p = __fmul_rn(a.hi, k);
  float e = __fmaf_rn(a.hi, k, -p);
  e = __fmaf_rn(a.lo, k, e);
  return dfr{p, e};
}

// exact scaling by a power of two
__device__ __forceinline__ dfr dfr_scale2(dfr a, float p2) { return dfr{__fmul_rn(a.hi, p2), __fmul_rn(a.lo, p2)}; }

// Renormalise: hi = fl(hi + lo), lo = the rest (Fast2Sum).
__device__ __forceinline__ dfr dfr_norm(dfr a) {
  const float s = __fadd_rn(a.hi, a.lo);
  return dfr{s, __fsub_rn(a.lo, __fsub_rn(s, a.hi))};
}

// 1 / a: the FP32 reciprocal r0 of the high part refined by one Newton step carried in
// double-float, r = r0 + r0 (1 - a r0); 1 - a r0 is formed exactly to first order from the
// TwoProd of the high parts.
__device__ __forceinline__ dfr dfr_rcp(dfr a) {
  const float r0 = __frcp_rn(a.hi);
  const float p = __fmul_rn(a.hi, r0);
  const float pe = __fmaf_rn(a.hi, r0, -p);
  // 1 - a r0 = (1 - p) - pe - a.lo r0, with 1 - p exact (p is within an ulp of 1)
  const float d = __fmaf_rn(-a.lo, r0, __fsub_rn(__fsub_rn(1.0f, p), pe));
  return dfr{r0, __fmul_rn(r0, d)};
}

__device__ __forceinline__ double dfr_to_double(dfr a) { return (double)a.hi + (double)a.lo; }

// Split of an FP64 value (FP64 work: only where the state enters or leaves the double-float form).
__device__ __forceinline__ dfr dfr_from_double(double x) {
  const float h = (float)x;
  return dfr{h, (float)(x - (double)h)};
}

// Complex double-float value, 16 bytes: (re.hi, re.lo, im.hi, im.lo).  Same size as an FP64
// complex, so buffers and shared-memory pencils are laid out exactly as in the FP64 passes.
struct alignas(16) cdf {
  using value_type = dfr;
  dfr re, im;
};

__device__ __forceinline__ cdf cdf_norm(cdf a) { return cdf{dfr_norm(a.re), dfr_norm(a.im)}; }

__device__ __forceinline__ cdf cdf_from_c64(double re, double im) {
  return cdf{dfr_from_double(re), dfr_from_double(im)};
}

}  // namespace mhd
