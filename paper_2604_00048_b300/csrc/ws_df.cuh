// Double-word arithmetic from error-free transformations (Knuth's TwoSum, the
// FMA-based TwoProduct): a value is carried as an unevaluated sum hi + lo of two
// working-precision numbers. Used where the refinement residual needs more than the
// working precision; B300's FP64 rate is far too low to do this in double.
#pragma once

namespace ws {

template <typename F>
struct DW {
  F hi, lo;
};

// s + e == a + b exactly (Knuth).
template <typename F>
__device__ __forceinline__ DW<F> two_sum(F a, F b) {
  const F s = a + b;
  const F bb = s - a;
  const F e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

// p + e == a * b exactly (one FMA).
template <typename F>
__device__ __forceinline__ DW<F> two_prod(F a, F b) {
  const F p = a * b;
  return {p, fma(a, b, -p)};
}

template <typename F>
__device__ __forceinline__ DW<F> dw_add(DW<F> a, DW<F> b) {
  DW<F> s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  const F h = s.hi + s.lo;
  return {h, s.lo - (h - s.hi)};
}

// (a.hi + a.lo) * c with c a working-precision scalar.
template <typename F>
__device__ __forceinline__ DW<F> dw_scale(DW<F> a, F c) {
  DW<F> p = two_prod(a.hi, c);
  p.lo = fma(a.lo, c, p.lo);
  const F h = p.hi + p.lo;
  return {h, p.lo - (h - p.hi)};
}

// acc + r * s with r a working-precision scalar: error ~ u^2 (|acc| + |r s|) (the
// sloppy double-word sum; enough where the terms' magnitudes, not the result's, set the
// scale, as in a linear recursion).
template <typename F>
__device__ __forceinline__ DW<F> dw_fma(DW<F> acc, F r, DW<F> s) {
  DW<F> p = two_prod(r, s.hi);
  p.lo = fma(r, s.lo, p.lo);
  DW<F> t = two_sum(acc.hi, p.hi);
  t.lo += acc.lo + p.lo;
  const F h = t.hi + t.lo;
  return {h, t.lo - (h - t.hi)};
}

// Double-float number type for the ragged path's high-precision re-solve: normalised
// hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits, from FP32 operations only
// (B300 issues FP64 at a small fraction of its FP32 rate). Addition is the accurate
// two-TwoSum form and multiplication the FMA form analysed by Joldes, Muller and Popescu
// (ACM TOMS 2017: relative errors about 3u^2 and 5u^2 with u = 2^-24); the reciprocal
// square root is one Newton step in double-float from the rounded FP32 value.
__device__ __forceinline__ DW<float> fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

struct dwf {
  float hi, lo;
  __device__ __forceinline__ dwf() : hi(0.f), lo(0.f) {}
  __device__ __forceinline__ dwf(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ dwf(float v) : hi(v), lo(0.f) {}
  __device__ __forceinline__ explicit dwf(int v) : hi((float)v), lo(0.f) {}
  __device__ __forceinline__ float to_float() const { return hi + lo; }
};

__device__ __forceinline__ dwf operator-(dwf a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dwf operator+(dwf a, dwf b) {
  const DW<float> s = two_sum(a.hi, b.hi);
  const DW<float> t = two_sum(a.lo, b.lo);
  DW<float> v = fast_two_sum(s.hi, s.lo + t.hi);
  v = fast_two_sum(v.hi, v.lo + t.lo);
  return {v.hi, v.lo};
}

__device__ __forceinline__ dwf operator-(dwf a, dwf b) { return a + (-b); }

__device__ __forceinline__ dwf operator*(dwf a, dwf b) {
  DW<float> p = two_prod(a.hi, b.hi);
  const float t = fmaf(a.lo, b.hi, a.hi * b.lo);
  p = fast_two_sum(p.hi, p.lo + t);
  return {p.hi, p.lo};
}

__device__ __forceinline__ bool operator>(dwf a, dwf b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// fma overloads in this namespace (a declaration here hides the global ones)
__device__ __forceinline__ dwf fma(dwf a, dwf b, dwf c) { return a * b + c; }
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }

// a * b + c with a * b >= 0 and c >= 0 (sums of squares): the same-sign ("sloppy") double-word
// addition, one TwoSum and one FastTwoSum, whose relative error stays about 2u^2 when the
// terms cannot cancel (Joldes, Muller and Popescu, 2017).
__device__ __forceinline__ dwf fma_pos(dwf a, dwf b, dwf c) {
  const dwf p = a * b;
  DW<float> s = two_sum(p.hi, c.hi);
  s.lo += p.lo + c.lo;
  const DW<float> v = fast_two_sum(s.hi, s.lo);
  return {v.hi, v.lo};
}

// 1/sqrt(x) for x > 0: r0 from the hardware reciprocal square root (one MUFU op, relative
// error below 2^-22.9), then one Newton step in double-float, r = r0 + r0 (1 - x r0^2) / 2,
// which squares the relative error (about 1.5 * 2^-45.8, at the level of the double-float
// operations' own rounding).
__device__ __forceinline__ dwf rsqrt_(dwf x) {
  float r0;
  asm("rsqrt.approx.f32 %0, %1;" : "=f"(r0) : "f"(x.hi));  // subnormal inputs kept (no .ftz)
  const dwf e = dwf(1.0f) - x * dwf(two_prod(r0, r0).hi, two_prod(r0, r0).lo);
  return dwf(r0) + dwf(0.5f * r0) * e;
}

__device__ __forceinline__ dwf sqrt_(dwf x) { return x.hi > 0.f ? x * rsqrt_(x) : dwf(0.f); }

}  // namespace ws
