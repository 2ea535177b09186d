// Double-float arithmetic (pairs of FP32 values, hi + lo) for the
// double-float redo (element_df.cuh): error-free transformations two_sum
// (Knuth) and fast_two_sum (Dekker, |a| >= |b|), the accurate double-word
// sum (relative error <= 3 u^2 / (1 - 4 u) of the exact sum, u = 2^-24;
// Joldes, Muller & Popescu 2017), the product with hi*hi kept exactly by an
// FMA and the two cross terms added (<= 5 u^2), exact sign tests against an
// FP32 threshold and the order of normalised pairs.  Host and device: the
// host build (plain C++, no FMA contraction) is what the CPU tests check
// against exact rationals.
#pragma once

#ifndef __CUDACC__
#include <cmath>
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace hexval {

struct DF {
  float hi, lo;
  DF() = default;
  __host__ __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ explicit DF(int v) : hi(static_cast<float>(v)), lo(0.f) {}
};

__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__host__ __device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
__host__ __device__ __forceinline__ DF operator+(const DF& x, const DF& y) {
  float s, t, u, v;
  two_sum(x.hi, y.hi, s, t);
  two_sum(x.lo, y.lo, u, v);
  t += u;
  fast_two_sum(s, t, s, t);
  t += v;
  fast_two_sum(s, t, s, t);
  return DF(s, t);
}
__host__ __device__ __forceinline__ DF operator-(const DF& x) { return DF(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ DF operator-(const DF& x, const DF& y) { return x + (-y); }
__host__ __device__ __forceinline__ DF operator*(const DF& x, const DF& y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  float s, t;
  fast_two_sum(p, e, s, t);
  return DF(s, t);
}
__host__ __device__ __forceinline__ DF fma(const DF& a, const DF& b, const DF& c) { return a * b + c; }

// Ordering of normalised pairs (hi = the rounding of hi + lo, as every
// operation above returns them): rounding is monotone, so hi1 < hi2 implies
// hi1 + lo1 <= hi2 + lo2, and equal his compare by lo.
__host__ __device__ __forceinline__ bool df_less(const DF& a, const DF& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__host__ __device__ __forceinline__ DF df_min(const DF& a, const DF& b) { return df_less(b, a) ? b : a; }
__host__ __device__ __forceinline__ DF df_max(const DF& a, const DF& b) { return df_less(a, b) ? b : a; }

// Exact sign test v - t > 0 for a float t.  two_sum gives hi - t = s + r
// exactly; when hi is within a factor 2 of t, r = 0 (Sterbenz) and the sign
// of the rounded s + lo is the sign of the exact s + lo; otherwise |s| is far
// above |r + lo| and decides alone.
__host__ __device__ __forceinline__ bool df_gt(const DF& v, float t) {
  float s, r;
  two_sum(v.hi, -t, s, r);
  return s + (r + v.lo) > 0.f;
}
__host__ __device__ __forceinline__ bool df_le(const DF& v, float t) { return !df_gt(v, t); }

}  // namespace hexval
