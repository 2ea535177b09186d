// The FP32 form of one element: 20 samples and 27 coefficients (Sec. 4-5,
// Table t:Tsmall) in FP32 with a certified error bound, and the depth-0
// decision of Sec. 6 that FP32 can certify.
//
// FP32 error bound, u = 2^-24: with eps the per-component error of the
// computed edge vectors (input rounding included) and L the largest
// |component| among them, every unscaled sample and coefficient is within
// 200 eps L^2 + 740 u L^3 of its exact value; the kernels use
// E = (256 eps L^2 + 1024 u L^3) 1.0001 with eps = 2^-23 X + 2^-24 L,
// X >= |coordinates|.  The scaled class values (corner c, edge sample C =
// 4 J, edge 2 b, face 4 b, centre 8 b) are within E times their scale.
#pragma once

#include "hexval_internal.cuh"

namespace hexval {

// FP64 -> FP32 on the integer pipe, rounding the magnitude to nearest (ties
// up): |result - x| <= 2^-24 |x|.  Sets `bad` when x is outside the exponent
// range [2^-126, 2^125) (zero is fine), including NaN and infinities.
__device__ __forceinline__ float d2f_int(double x, bool& bad) {
  long long bits = __double_as_longlong(x);
  uint32_t hi = static_cast<uint32_t>(bits >> 32), lo = static_cast<uint32_t>(bits);
  uint32_t e = (hi >> 20) & 0x7ffu;
  bool zero = ((hi << 1) | lo) == 0u;
  uint32_t f = __funnelshift_l(lo, hi, 3);
  f = (f & 0x7fffffffu) ^ 0x40000000u;  // exponent field e - 896 for e in [897, 1149]
  f += (lo >> 28) & 1u;                 // rounding (a carry moves into the exponent)
  f |= hi & 0x80000000u;
  bad |= !zero && (e - 897u > 252u);
  return zero ? __uint_as_float(hi & 0x80000000u) : __uint_as_float(f);
}

// FP32 -> FP64 on the integer pipe (exact for normal numbers; FP32
// subnormals, below 2^-126, become signed zeros).
__device__ __forceinline__ double f2d_int(float v) {
  uint32_t b = __float_as_uint(v);
  uint32_t sgn = b & 0x80000000u;
  bool tiny = (b & 0x7f800000u) == 0u;
  uint32_t hi = tiny ? sgn : (sgn | (((b & 0x7fffffffu) >> 3) + (896u << 20)));
  uint32_t lo = tiny ? 0u : (b << 29);
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

__device__ __forceinline__ float fabsmax3(float m, const V3<float>& v) {
  return fmaxf(m, fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.z))));
}

// Samples and coefficients of one element from its 8 nodes in FP32, and
// their bound E.  X bounds |coordinate| (indexed: |node 1| only, completed
// here with 3 L).  Returns false when the bound cannot be formed in FP32
// (then the element goes to FP64).
template <bool INDEXED>
__device__ __forceinline__ bool fp32_root(const V3<float> Y[8], float X, bool bad,
                                          Scaled<float>& s, float& E) {
  V3<float> a[4], b[4], gg[4];
  edges_from_nodes(Y, a, b, gg);
  float L = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    L = fabsmax3(L, a[q]);
    L = fabsmax3(L, b[q]);
    L = fabsmax3(L, gg[q]);
  }
  if (INDEXED) X = fmaf(3.f, L, X);  // every node is within 3 edges of node 1
  const float eps = fmaf(0x1p-24f, L, 0x1p-23f * X);
  const float L2 = L * L;
  E = fmaf(256.f * eps, L2, 1024.f * 0x1p-24f * (L2 * L)) * 1.0001f;
  // too small (underflow) or too large (overflow) for the FP32 bound
  bad |= !(L >= 0x1p-30f) || !(E < 0x1p100f);
  if (bad) return false;
  coefficients_from_edges(a, b, gg, s);
  return true;
}

// Depth-0 decision from the scaled coefficients: 0 invalid (a sample
// certainly <= 0), 1 valid (all 27 certainly > 0), 2 refine (all samples
// certainly > 0 and a coefficient certainly <= 0), 3 escalate (a sign FP32
// cannot settle); lo / hi = min / max of the 27 unscaled coefficients.
__device__ __forceinline__ int fp32_classify(const Scaled<float>& s, float E, float& lo,
                                             float& hi) {
  float mnC = s.corner[0], mxC = s.corner[0];
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    mnC = fminf(mnC, s.corner[k]);
    mxC = fmaxf(mxC, s.corner[k]);
  }
  float mnS = s.edgeC[0];
#pragma unroll
  for (int e = 1; e < 12; ++e) mnS = fminf(mnS, s.edgeC[e]);
  float mnE = s.edge[0], mxE = s.edge[0];
#pragma unroll
  for (int e = 1; e < 12; ++e) {
    mnE = fminf(mnE, s.edge[e]);
    mxE = fmaxf(mxE, s.edge[e]);
  }
  float mnF = s.face[0], mxF = s.face[0];
#pragma unroll
  for (int f = 1; f < 6; ++f) {
    mnF = fminf(mnF, s.face[f]);
    mxF = fmaxf(mxF, s.face[f]);
  }
  lo = fminf(fminf(mnC, mnE * 0.5f), fminf(mnF * 0.25f, s.centre * 0.125f));
  hi = fmaxf(fmaxf(mxC, mxE * 0.5f), fmaxf(mxF * 0.25f, s.centre * 0.125f));
  // Step 2: a sample certainly <= 0; Step 4: all 27 certainly > 0
  const bool invalid = (mnC <= -E) | (mnS <= -4.f * E);
  const bool samples = (mnC > E) & (mnS > 4.f * E);
  const bool certified = samples & (mnE > 2.f * E) & (mnF > 4.f * E) & (s.centre > 8.f * E);
  const bool refine = samples & ((mnE <= -2.f * E) | (mnF <= -4.f * E) | (s.centre <= -8.f * E));
  return invalid ? 0 : (certified ? 1 : (refine ? 2 : 3));
}

// The FP32 decision of one element (outcomes as fp32_classify).
template <bool INDEXED>
__device__ __forceinline__ int fp32_decide(const V3<float> Y[8], float X, bool bad, float& lo,
                                           float& hi) {
  Scaled<float> s;
  float E;
  if (!fp32_root<INDEXED>(Y, X, bad, s, E)) return 3;
  return fp32_classify(s, E, lo, hi);
}

// Node records of element g for the FP32 form: FP32 coordinates, the bound X
// on |coordinate| as the FP32 pass forms it, and whether a coordinate is
// outside the FP32 range.  Returns false for a connectivity entry out of
// range.
__device__ __forceinline__ bool load_element32(const Batch& p, int64_t g, V3<float> Y[8],
                                               float& X, bool& bad) {
  bad = false;
  if (!p.indexed) {
    X = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      Y[k].x = d2f_int(__ldg(p.soa + (3 * k + 0) * p.stride + g), bad);
      Y[k].y = d2f_int(__ldg(p.soa + (3 * k + 1) * p.stride + g), bad);
      Y[k].z = d2f_int(__ldg(p.soa + (3 * k + 2) * p.stride + g), bad);
      X = fabsmax3(X, Y[k]);
    }
    return true;
  }
  const int4* c4 = reinterpret_cast<const int4*>(p.conn + 8 * g);
  const int4 c0 = __ldg(c4), c1 = __ldg(c4 + 1);
  const int id[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 8; ++k) ok &= static_cast<uint32_t>(id[k]) < static_cast<uint64_t>(p.n_nodes);
  if (!ok) return false;
  const float4* N = reinterpret_cast<const float4*>(p.s.node32);
  float badw = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 h = __ldg(N + id[k]);
    Y[k] = {h.x, h.y, h.z};
    badw += h.w;
  }
  bad = badw != 0.f;
  X = fabsmax3(0.f, Y[0]);  // completed with 3 L by fp32_root
  return true;
}

}  // namespace hexval
