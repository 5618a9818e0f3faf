// Float-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits carried by FP32
// operations only (the double-length technique of Dekker, "A floating-point
// technique for extending the available precision", 1971; its GPU form after
// Thall, "Extended-precision floating-point numbers for GPU computation",
// 2006).  Used on paths that need more than FP32 but would otherwise run as
// long serial chains of FP64 operations, which are slow on this GPU; the
// exponent range is FP32's.
#pragma once

namespace ff {

struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 make(float a) { return {a, 0.f}; }

// s + e == a + b exactly (Knuth's two-sum).
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

// s + e == a + b exactly when |a| >= |b| (or a == 0).
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

// p + e == a * b exactly (the FMA gives the rounding error of the product).
__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ F2 add(F2 a, F2 b) {
  F2 s = two_sum(a.hi, b.hi);
  const F2 t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ F2 neg(F2 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ F2 mul(F2 a, F2 b) {
  F2 p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}

// a - b * c
__device__ __forceinline__ F2 sub_mul(F2 a, F2 b, F2 c) { return add(a, neg(mul(b, c))); }

// 1 / a for a != 0: the FP32 quotient x0 and one Newton step,
// x1 = x0 + x0 (1 - a x0), with the residual 1 - a x0 formed in float-float.
__device__ __forceinline__ F2 recip(F2 a) {
  const float x0 = 1.0f / a.hi;
  const F2 ax = mul(a, make(x0));
  const F2 e = add(make(1.0f), neg(ax));
  return fast_two_sum(x0, x0 * e.hi);
}

__device__ __forceinline__ double to_double(F2 a) { return (double)a.hi + (double)a.lo; }

}  // namespace ff
