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
//
// Where the constants come from.  Rounding a coordinate to FP32 errs by at
// most 2^-24 X, so a computed edge component differs from the exact edge by
// at most two input roundings and the subtraction's own: eps = 2^-23 X +
// 2^-24 L; a sum of two parallel edges by at most 2 eps + 2^-23 L.  A triple
// product is linear in each column: columns perturbed by at most (dA, dB,
// dC) per component (magnitudes at most mA, mB, mC) move it by at most
// 6 (dA mB mC + mA dB mC + mA mB dC) to first order, and its evaluation adds
// at most 5 roundings to each of its 6 terms (6 gamma_5 mA mB mC).  A corner
// sample (columns L, L, L) is thus within 18 eps L^2 + 30 u L^3 (+ higher
// order) and an edge sample C (columns L, 2L, 2L) within 72 eps L^2 +
// 168 u L^3.  Each class of Table t:Tsmall is a signed sum of these samples
// with small integer weights and power-of-two scalings (the centre, the
// largest: 12 edge samples and 5 times the 8 corners, over 8: 198 eps L^2 +
// 402 u L^3), and its partial sums form a tree in which every term passes
// through at most 5 roundings, adding gamma_5 times the sum of the absolute
// terms (12 * 24 L^3 + 40 * 6 L^3, over 8: 330 u L^3).  That gives the
// totals above; the constants 256 and 1024 exceed them with a margin for
// the second-order terms.
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

// Three-operand minimum / maximum (one instruction on sm_100 and later).  A
// NaN operand is ignored, as by fminf / fmaxf; the result is NaN only when
// all three are.
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Largest |component| of the 12 edge vectors (seeded with 0).
__device__ __forceinline__ float edge_magnitude(const V3<float> a[4], const V3<float> b[4],
                                                const V3<float> g[4]) {
  float L = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    L = max3f(L, fabsf(a[q].x), fabsf(a[q].y));
    L = max3f(L, fabsf(a[q].z), fabsf(b[q].x));
    L = max3f(L, fabsf(b[q].y), fabsf(b[q].z));
    L = max3f(L, fabsf(g[q].x), fabsf(g[q].y));
    L = fmaxf(L, fabsf(g[q].z));
  }
  return L;
}

// Largest |coordinate| of the 8 nodes (seeded with 0).
__device__ __forceinline__ float node_magnitude(const V3<float> Y[8]) {
  float X = 0.f;
#pragma unroll
  for (int k = 0; k < 8; k += 2) {
    X = max3f(X, fabsf(Y[k].x), fabsf(Y[k].y));
    X = max3f(X, fabsf(Y[k].z), fabsf(Y[k + 1].x));
    X = max3f(X, fabsf(Y[k + 1].y), fabsf(Y[k + 1].z));
  }
  return X;
}

// Largest |coordinate| of one node.
__device__ __forceinline__ float fabsmax3(const V3<float>& v) {
  return max3f(fabsf(v.x), fabsf(v.y), fabsf(v.z));
}

// Minimum and maximum of n values (n >= 2) with three-operand steps.
template <int N>
__device__ __forceinline__ float min_of(const float* v) {
  float m = fminf(v[0], v[1]);
  int i = 2;
#pragma unroll
  for (; i + 1 < N; i += 2) m = min3f(m, v[i], v[i + 1]);
  if (i < N) m = fminf(m, v[i]);
  return m;
}
template <int N>
__device__ __forceinline__ float max_of(const float* v) {
  float m = fmaxf(v[0], v[1]);
  int i = 2;
#pragma unroll
  for (; i + 1 < N; i += 2) m = max3f(m, v[i], v[i + 1]);
  if (i < N) m = fmaxf(m, v[i]);
  return m;
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
  const float L = edge_magnitude(a, b, gg);
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
  const float mnC = min_of<8>(s.corner), mxC = max_of<8>(s.corner);
  const float mnS = min_of<12>(s.edgeC);
  const float mnE = min_of<12>(s.edge), mxE = max_of<12>(s.edge);
  const float mnF = min_of<6>(s.face), mxF = max_of<6>(s.face);
  lo = fminf(min3f(mnC, mnE * 0.5f, mnF * 0.25f), s.centre * 0.125f);
  hi = fmaxf(max3f(mxC, mxE * 0.5f, mxF * 0.25f), s.centre * 0.125f);
  // Step 2: a sample certainly <= 0; Step 4: all 27 certainly > 0
  const bool invalid = (mnC <= -E) | (mnS <= -4.f * E);
  const bool samples = (mnC > E) & (mnS > 4.f * E);
  const bool certified = samples & (mnE > 2.f * E) & (mnF > 4.f * E) & (s.centre > 8.f * E);
  const bool refine = samples & ((mnE <= -2.f * E) | (mnF <= -4.f * E) | (s.centre <= -8.f * E));
  return invalid ? 0 : (certified ? 1 : (refine ? 2 : 3));
}

// What FP32 leaves unsettled in an element it escalates (fp32_classify
// outcome 3), for the FP64 redo of just those signs (fp64_partial,
// element64.cuh): bits 0-7 the corner samples, 8-19 the edge samples, 20-31
// the edge coefficients that are not certainly positive (the samples of an
// escalated element are never certainly <= 0); bit 32: a face or the centre
// not certainly positive, or an edge coefficient certainly <= 0.
__device__ __forceinline__ uint64_t fp32_unsettled(const Scaled<float>& s, float E) {
  uint64_t m = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (!(s.corner[k] > E)) m |= 1ull << k;
#pragma unroll
  for (int e = 0; e < 12; ++e)
    if (!(s.edgeC[e] > 4.f * E)) m |= 1ull << (8 + e);
  bool other = false;
#pragma unroll
  for (int e = 0; e < 12; ++e) {
    if (s.edge[e] <= -2.f * E) other = true;
    else if (!(s.edge[e] > 2.f * E)) m |= 1ull << (20 + e);
  }
#pragma unroll
  for (int f = 0; f < 6; ++f) other |= !(s.face[f] > 4.f * E);
  other |= !(s.centre > 8.f * E);
  return other ? m | (1ull << 32) : m;
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

// FP32 node records of the indexed form: float4 {x, y, z, w} per node.  A
// node with a coordinate outside the FP32 range gets x = y = z = +inf and
// w = 1.  An element touching such a node is escalated by its bound alone,
// whatever w: with some of its nodes finite, an edge joins a finite node to
// an infinite one (the 12 edges connect the 8 nodes), so L = inf and E is not
// finite; with all 8 infinite, every edge component is NaN and L stays 0.
// Either way fp32_root reports the element as not decidable in FP32.
//
// True when the 8 connectivity entries of a row are in [0, n_nodes)
// (n_nodes < 2^31: negative entries compare as large unsigned values).
__device__ __forceinline__ bool ids_in_range(const int4& c0, const int4& c1, int64_t n_nodes) {
  uint32_t m = __vimax3_u32(c0.x, c0.y, c0.z);
  m = __vimax3_u32(m, c0.w, c1.x);
  m = __vimax3_u32(m, c1.y, c1.z);
  m = max(m, static_cast<uint32_t>(c1.w));
  return m < static_cast<uint32_t>(n_nodes);
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
    }
    X = node_magnitude(Y);
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
  X = fabsmax3(Y[0]);  // completed with 3 L by fp32_root
  return true;
}

}  // namespace hexval
