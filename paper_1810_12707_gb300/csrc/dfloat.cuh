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
// bound is measured against.  Renormalisation (Fast2Sum) happens before values are stored to
// global memory and where a value's sign matters (squares).  Every operation is written with the
// _rn intrinsics, which the compiler never merges into fused multiply-adds: a contraction would
// change the rounded results the error terms are computed from.
//
// Two double-float numbers -- the real and imaginary parts of a complex value, or the values of
// two grid rows -- are carried together as `cdf` {hi = (x.hi, y.hi), lo = (x.lo, y.lo)} and
// operated on with the packed two-lane FP32 instructions of sm_100 and later (__fadd2_rn,
// __fmul2_rn, __ffma2_rn): the same lane operations as two scalar sequences, in half the
// instructions.
#pragma once

#include <cuda_runtime.h>

namespace mhd {

// ---- scalar double-float ----
struct dfr {
  float hi, lo;
};

__host__ __device__ constexpr dfr dfr_const(double x) {
  return dfr{(float)x, (float)(x - (double)(float)x)};
}

__device__ __forceinline__ double dfr_to_double(dfr a) { return (double)a.hi + (double)a.lo; }

// Split of an FP64 value (FP64 work: only where the state enters or leaves the double-float form).
__device__ __forceinline__ dfr dfr_from_double(double x) {
  const float h = (float)x;
  return dfr{h, (float)(x - (double)h)};
}

// Renormalise: hi = fl(hi + lo), lo = the rest (Fast2Sum).
__device__ __forceinline__ dfr dfr_norm(dfr a) {
  const float s = __fadd_rn(a.hi, a.lo);
  return dfr{s, __fsub_rn(a.lo, __fsub_rn(s, a.hi))};
}

// ---- packed pairs of double-float numbers ----
struct alignas(16) cdf {
  using value_type = dfr;  // one lane
  float2 hi, lo;
};

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2swap(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float2 f2bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, f2neg(b)); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__host__ __device__ constexpr cdf cdf_const(double x, double y) {
  return cdf{{(float)x, (float)y}, {(float)(x - (double)(float)x), (float)(y - (double)(float)y)}};
}
__device__ __forceinline__ cdf cdf_zero() { return cdf{{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ dfr cdf_x(cdf a) { return dfr{a.hi.x, a.lo.x}; }
__device__ __forceinline__ dfr cdf_y(cdf a) { return dfr{a.hi.y, a.lo.y}; }
__device__ __forceinline__ cdf cdf_make(dfr x, dfr y) { return cdf{{x.hi, y.hi}, {x.lo, y.lo}}; }
// (s, s) from a double-float scalar
__device__ __forceinline__ cdf cdf_bc(dfr s) { return cdf{f2bc(s.hi), f2bc(s.lo)}; }

// lane-wise a + b, lazy: TwoSum of the high parts, the low parts and the rounding error summed
__device__ __forceinline__ cdf operator+(cdf a, cdf b) {
  const float2 s = f2add(a.hi, b.hi);
  const float2 v = f2sub(s, a.hi);
  const float2 e = f2add(f2sub(a.hi, f2sub(s, v)), f2sub(b.hi, v));
  return cdf{s, f2add(e, f2add(a.lo, b.lo))};
}
__device__ __forceinline__ cdf operator-(cdf a) { return cdf{f2neg(a.hi), f2neg(a.lo)}; }
__device__ __forceinline__ cdf operator-(cdf a, cdf b) { return a + (-b); }

// lane-wise a * b, lazy: TwoProd of the high parts plus the cross terms (a.lo b.lo, about 2^-48
// of the product, is dropped)
__device__ __forceinline__ cdf operator*(cdf a, cdf b) {
  const float2 p = f2mul(a.hi, b.hi);
  float2 e = f2fma(a.hi, b.hi, f2neg(p));
  e = f2fma(a.hi, b.lo, e);
  e = f2fma(a.lo, b.hi, e);
  return cdf{p, e};
}

// k * a, lane-wise, for an FP32 number k (small integer wavenumbers, powers of two)
__device__ __forceinline__ cdf operator*(float k, cdf a) {
  const float2 kk = f2bc(k);
  const float2 p = f2mul(a.hi, kk);
  float2 e = f2fma(a.hi, kk, f2neg(p));
  e = f2fma(a.lo, kk, e);
  return cdf{p, e};
}

// s * a, lane-wise, for a double-float scalar s
__device__ __forceinline__ cdf operator*(dfr s, cdf a) { return cdf_bc(s) * a; }

// exact scaling by a power of two
__device__ __forceinline__ cdf cdf_scale2(cdf a, float p2) { return cdf{f2mul(a.hi, f2bc(p2)), f2mul(a.lo, f2bc(p2))}; }

// lane-wise Fast2Sum renormalisation
__device__ __forceinline__ cdf cdf_norm(cdf a) {
  const float2 s = f2add(a.hi, a.lo);
  return cdf{s, f2sub(a.lo, f2sub(s, a.hi))};
}

// lane-wise 1 / a: the FP32 reciprocal r0 of the high part refined by one Newton step carried in
// double-float, r = r0 + r0 (1 - a r0); 1 - a r0 is formed to first order from the TwoProd of the
// high parts (1 - p is exact: p is within an ulp of 1).
__device__ __forceinline__ cdf cdf_rcp(cdf a) {
  const float2 r0 = make_float2(__frcp_rn(a.hi.x), __frcp_rn(a.hi.y));
  const float2 p = f2mul(a.hi, r0);
  const float2 pe = f2fma(a.hi, r0, f2neg(p));
  const float2 d = f2fma(f2neg(a.lo), r0, f2sub(f2sub(f2bc(1.0f), p), pe));
  return cdf{r0, f2mul(r0, d)};
}

// ---- complex double-float values: x = real part, y = imaginary part ----

// i a
__device__ __forceinline__ cdf cdf_mul_i(cdf a) {
  return cdf{make_float2(-a.hi.y, a.hi.x), make_float2(-a.lo.y, a.lo.x)};
}
// -i a
__device__ __forceinline__ cdf cdf_mul_negi(cdf a) {
  return cdf{make_float2(a.hi.y, -a.hi.x), make_float2(a.lo.y, -a.lo.x)};
}
// conj(a)
__device__ __forceinline__ cdf cdf_conj(cdf a) {
  return cdf{make_float2(a.hi.x, -a.hi.y), make_float2(a.lo.x, -a.lo.y)};
}
// (a.y, a.x)
__device__ __forceinline__ cdf cdf_swap(cdf a) { return cdf{f2swap(a.hi), f2swap(a.lo)}; }

// Complex product a w with the twiddle given as wr = (Re w, Re w) and wi = (-Im w, Im w):
// a w = a (Re w) + swap(a) (-Im w, Im w).
__device__ __forceinline__ cdf cdf_cmul(cdf a, cdf wr, cdf wi) { return a * wr + cdf_swap(a) * wi; }

__device__ __forceinline__ cdf cdf_from_c64(double re, double im) {
  const dfr x = dfr_from_double(re), y = dfr_from_double(im);
  return cdf_make(x, y);
}

}  // namespace mhd
