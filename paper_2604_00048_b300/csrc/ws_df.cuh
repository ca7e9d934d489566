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

}  // namespace ws
