// The samples and coefficients of one element in double-float arithmetic
// (pairs of FP32 values, hi + lo), for the redo of the FP32 form's
// escalations before FP64: on this GPU FP32 arithmetic is 64 times faster than FP64, and
// a double-float operation costs 2 to 20 FP32 instructions, so the redo runs
// several times faster while keeping about 44 bits.
//
// Primitives (error-free transformations): two_sum (Knuth), fast_two_sum
// (Dekker, |a| >= |b|), two_prod (FMA).  A double-float sum is the accurate
// double-word addition (relative error <= 3 u^2 / (1 - 4 u) of the exact sum,
// u = 2^-24, Joldes, Muller & Popescu 2017), a product keeps hi*hi exactly and
// the two cross terms (relative error <= 5 u^2).  Every operation is thus
// within u_df = 2^-44 (relative) of its exact result on the computed
// operands, and the forward-error analysis of the FP64 kernels applies with u
// replaced by u_df and each FMA counted as a product and a sum.
//
// Inputs: each FP64 coordinate x is split into hi = x rounded to FP32 and lo
// = (x - hi) rounded to FP32, |x - (hi + lo)| <= 2^-48 |x| + 2^-149; x - hi
// is formed exactly on the integer pipe from the low mantissa bits of x.
// Parts that fall below the FP32 normal range add at most 2^-149 per
// operation, far below E >= 2^-121 (L >= 2^-30).
//
// Bound (unscaled coefficients; the classes scale as in the FP32 form):
// E = (2^-31 L + 2^-38 X) L^2 with L the largest |component| of the computed
// edge vectors and X >= |coordinates|: the evaluation contributes at most
// 4096 u_df L^3 (the FP64 constant 930, doubled for the FMA split, with
// margin) and the input split 256 eps L^2 with eps = 2^-47 X + u_df L.
// Elements with L outside [2^-30, 2^30] or X > 2^60 are not handled here.
#pragma once

#include "element32.cuh"
// after the FP64 code above: its fma calls must not see the double-float fma
#include "df_arith.cuh"

namespace hexval {

__device__ __forceinline__ DF det3(const V3<DF>& A, const V3<DF>& B, const V3<DF>& C) {
  const DF cx = B.y * C.z - B.z * C.y;
  const DF cy = B.z * C.x - B.x * C.z;
  const DF cz = B.x * C.y - B.y * C.x;
  return A.x * cx + A.y * cy + A.z * cz;
}

// x = hi + lo as above; `bad` when x is outside the FP32 range.
__device__ __forceinline__ DF split_df(double x, bool& bad) {
  const float hi = d2f_int(x, bad);
  const long long bits = __double_as_longlong(x);
  const uint32_t h = static_cast<uint32_t>(bits >> 32), l = static_cast<uint32_t>(bits);
  const int e = static_cast<int>((h >> 20) & 0x7ffu);
  // x - hi = (-1)^s 2^(e - 1075) (m29 - c 2^29): m29 = the 29 mantissa bits
  // below hi's, c = 1 when hi was rounded up
  const int m29 = static_cast<int>(l & 0x1fffffffu);
  const int c = static_cast<int>((l >> 28) & 1u);
  float r = __int2float_rn(m29 - (c << 29));  // |m29 - c 2^29| <= 2^29: rounds to 24 bits
  r = ldexpf(r, e - 1075);
  if (h >> 31) r = -r;
  return DF(hi, ((h << 1) | l) == 0u ? 0.f : r);
}

// Scaled coefficients of element g in double-float and their bound E (on the
// unscaled coefficients, as float); false when the element is outside this
// path's range (or a connectivity entry is out of range).
__device__ __forceinline__ bool df_root(const Batch& p, int64_t g, Scaled<DF>& s, float& E) {
  V3<double> X[8];
  if (!load_element(p, g, X)) return false;
  bool bad = false;
  V3<DF> Y[8];
  float Xm = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    Y[k] = {split_df(X[k].x, bad), split_df(X[k].y, bad), split_df(X[k].z, bad)};
    Xm = fmaxf(Xm, fmaxf(fabsf(Y[k].x.hi), fmaxf(fabsf(Y[k].y.hi), fabsf(Y[k].z.hi))));
  }
  V3<DF> a[4], b[4], gg[4];
  edges_from_nodes(Y, a, b, gg);
  float L = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    L = fmaxf(L, fmaxf(fabsf(a[q].x.hi), fmaxf(fabsf(a[q].y.hi), fabsf(a[q].z.hi))));
    L = fmaxf(L, fmaxf(fabsf(b[q].x.hi), fmaxf(fabsf(b[q].y.hi), fabsf(b[q].z.hi))));
    L = fmaxf(L, fmaxf(fabsf(gg[q].x.hi), fmaxf(fabsf(gg[q].y.hi), fabsf(gg[q].z.hi))));
  }
  L *= 1.0001f;  // the hi parts may round |component| down
  bad |= !(L >= 0x1p-30f) || !(L <= 0x1p30f) || !(Xm <= 0x1p60f);
  if (bad) return false;
  E = fmaf(0x1p-31f, L, 0x1p-38f * Xm * 1.0001f) * (L * L) * 1.001f;
  coefficients_from_edges(a, b, gg, s);
  return true;
}

// Depth-0 decision from the double-float coefficients and their bound E
// (outcomes as fp32_classify: 0 invalid, 1 valid, 2 refine, 3 undecided);
// lo / hi = min / max of the 27 unscaled coefficients.
__device__ __forceinline__ int df_classify(const Scaled<DF>& s, float E, double& lo, double& hi) {
  DF mnC = s.corner[0], mxC = s.corner[0];
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    mnC = df_min(mnC, s.corner[k]);
    mxC = df_max(mxC, s.corner[k]);
  }
  DF mnS = s.edgeC[0];
#pragma unroll
  for (int e = 1; e < 12; ++e) mnS = df_min(mnS, s.edgeC[e]);
  DF mnE = s.edge[0], mxE = s.edge[0];
#pragma unroll
  for (int e = 1; e < 12; ++e) {
    mnE = df_min(mnE, s.edge[e]);
    mxE = df_max(mxE, s.edge[e]);
  }
  DF mnF = s.face[0], mxF = s.face[0];
#pragma unroll
  for (int f = 1; f < 6; ++f) {
    mnF = df_min(mnF, s.face[f]);
    mxF = df_max(mxF, s.face[f]);
  }
  const DF c8 = s.centre;
  // unscaled extremes (the scales are powers of 2, exact on both parts)
  const DF lo2 = df_min(df_min(mnC, DF(mnE.hi * 0.5f, mnE.lo * 0.5f)),
                        df_min(DF(mnF.hi * 0.25f, mnF.lo * 0.25f), DF(c8.hi * 0.125f, c8.lo * 0.125f)));
  const DF hi2 = df_max(df_max(mxC, DF(mxE.hi * 0.5f, mxE.lo * 0.5f)),
                        df_max(DF(mxF.hi * 0.25f, mxF.lo * 0.25f), DF(c8.hi * 0.125f, c8.lo * 0.125f)));
  lo = f2d_int(lo2.hi) + f2d_int(lo2.lo);
  hi = f2d_int(hi2.hi) + f2d_int(hi2.lo);
  const bool invalid = df_le(mnC, -E) | df_le(mnS, -4.f * E);
  const bool samples = df_gt(mnC, E) & df_gt(mnS, 4.f * E);
  const bool certified = samples & df_gt(mnE, 2.f * E) & df_gt(mnF, 4.f * E) & df_gt(c8, 8.f * E);
  const bool refine = samples & (df_le(mnE, -2.f * E) | df_le(mnF, -4.f * E) | df_le(c8, -8.f * E));
  return invalid ? 0 : (certified ? 1 : (refine ? 2 : 3));
}

}  // namespace hexval
