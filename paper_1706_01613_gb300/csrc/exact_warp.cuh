// Exact tier, depth 0, by a whole warp with the integers in registers and
// shared memory.
//
// Most elements that reach the exact tier are decided at depth 0 (a sample
// whose FP64 value is within rounding of zero, an element that is barely
// valid).  For them the full tier (exact.cuh: one thread, integers in global
// memory, widths sized for the deepest refinement) is needlessly slow.  Here
// the 24 coordinates are scaled to integers as in exact.cuh (all of B bits
// for B <= 120), lane t < 20 computes sample t (Sec. 5) as an exact 384-bit
// integer, and lanes 8..26 form the sign of their Table t:Tsmall
// combination (scaled as in the FP64 kernels: edge 2b = C - c_a - c_b,
// face 4b = sum of 4 C - 3 x sum of 4 c, centre 8b = sum of 12 C - 5 x sum
// of 8 c, with c the corner samples and C = 4 J the edge samples).  The
// verdict is that of Steps 2-4 of Sec. 6: INVALID at depth 0 if a sample is
// <= 0, VALID at depth 0 if all 27 coefficients are > 0.  Anything else
// (refinement needed, or B > 120) is left to the full tier.
//
// Widths: coordinates < 2^120; edge vectors < 2^121; sums of two edges
// < 2^122 (all in 4 limbs of 32 bits, two's complement); a triple product
// of such columns < 6 * 2^365 < 2^368; the combinations < 52 * 2^368 <
// 2^374: every value fits 12 limbs (384 bits) with its sign, so the
// arithmetic modulo 2^384 is exact.
#pragma once

#include "exact.cuh"
#include "warp_items.cuh"

namespace hexval {
namespace exact_tier {

constexpr int kFastBits = 120;
constexpr int kFastWords = 24 * 4 + 20 * 12;  // shared words per warp

template <int K>
struct Wide {
  uint32_t v[K];
};

template <int K>
__device__ __forceinline__ Wide<K> wneg(const Wide<K>& a) {
  Wide<K> r;
  unsigned long long c = 1;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    c += static_cast<uint32_t>(~a.v[i]);
    r.v[i] = static_cast<uint32_t>(c);
    c >>= 32;
  }
  return r;
}

template <int K>
__device__ __forceinline__ Wide<K> wadd(const Wide<K>& a, const Wide<K>& b) {
  Wide<K> r;
  unsigned long long c = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    c += static_cast<unsigned long long>(a.v[i]) + b.v[i];
    r.v[i] = static_cast<uint32_t>(c);
    c >>= 32;
  }
  return r;
}

template <int K>
__device__ __forceinline__ Wide<K> wsub(const Wide<K>& a, const Wide<K>& b) {
  Wide<K> r;
  unsigned long long c = 1;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    c += static_cast<unsigned long long>(a.v[i]) + static_cast<uint32_t>(~b.v[i]);
    r.v[i] = static_cast<uint32_t>(c);
    c >>= 32;
  }
  return r;
}

template <int K>
__device__ __forceinline__ bool wnegative(const Wide<K>& a) {
  return (a.v[K - 1] >> 31) != 0u;
}

template <int K>
__device__ __forceinline__ bool wpositive(const Wide<K>& a) {
  uint32_t any = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) any |= a.v[i];
  return !wnegative(a) && any != 0u;
}

// Signed product (operands far from the most negative value).
template <int KA, int KB>
__device__ __forceinline__ Wide<KA + KB> wmul(const Wide<KA>& a, const Wide<KB>& b) {
  const bool na = wnegative(a), nb = wnegative(b);
  const Wide<KA> ma = na ? wneg(a) : a;
  const Wide<KB> mb = nb ? wneg(b) : b;
  Wide<KA + KB> r;
#pragma unroll
  for (int i = 0; i < KA + KB; ++i) r.v[i] = 0u;
#pragma unroll
  for (int i = 0; i < KA; ++i) {
    unsigned long long c = 0;
#pragma unroll
    for (int j = 0; j < KB; ++j) {
      unsigned long long t = static_cast<unsigned long long>(ma.v[i]) * mb.v[j] + r.v[i + j] + c;
      r.v[i + j] = static_cast<uint32_t>(t);
      c = t >> 32;
    }
    r.v[i + KB] = static_cast<uint32_t>(c);
  }
  return na != nb ? wneg(r) : r;
}

template <int KO, int K>
__device__ __forceinline__ Wide<KO> wext(const Wide<K>& a) {
  Wide<KO> r;
  const uint32_t fill = wnegative(a) ? 0xffffffffu : 0u;
#pragma unroll
  for (int i = 0; i < KO; ++i) r.v[i] = i < K ? a.v[i] : fill;
  return r;
}

__device__ __forceinline__ Wide<4> load4(const uint32_t* s) {
  Wide<4> r;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.v[i] = s[i];
  return r;
}

// Component d of vector `id` (0-11 edge vectors, 12-23 sums of two parallel
// edges, ids as in warp_items.cuh) from the integer coordinates X (4 words
// per coordinate, [3 node + d]).
__device__ __forceinline__ Wide<4> column(const uint32_t* X, int id, int d) {
  if (id < 12) {
    int lo, hi;
    edge_nodes(id, lo, hi);
    return wsub(load4(X + 4 * (3 * hi + d)), load4(X + 4 * (3 * lo + d)));
  }
  int e0, e1;
  sum_parts(id - 12, e0, e1);
  int l0, h0, l1, h1;
  edge_nodes(e0, l0, h0);
  edge_nodes(e1, l1, h1);
  return wadd(wsub(load4(X + 4 * (3 * h0 + d)), load4(X + 4 * (3 * l0 + d))),
              wsub(load4(X + 4 * (3 * h1 + d)), load4(X + 4 * (3 * l1 + d))));
}

// Weight of sample t (0-7 corners by node id, 8-19 edge samples) in the
// scaled coefficient of lane L (8-19 edges, 20-25 faces, 26 centre), as in
// fp64_element_warp.
__device__ __forceinline__ int q_weight(int L, int t) {
  if (L < 8 || L > 26) return 0;
  if (L < 20) {
    const int ed = L - 8, u = ed & 1, v = (ed & 3) >> 1;
    int n0, n1;
    if (ed < 4) { n0 = node_at(0, u, v); n1 = node_at(1, u, v); }
    else if (ed < 8) { n0 = node_at(u, 0, v); n1 = node_at(u, 1, v); }
    else { n0 = node_at(u, v, 0); n1 = node_at(u, v, 1); }
    if (t == L) return 1;
    return (t == n0 || t == n1) ? -1 : 0;
  }
  if (L == 26) return t < 8 ? -5 : 1;
  const int f = L - 20, u = f & 1;
  if (t < 8) {  // corners of the face
    const int x = (t == 1 || t == 2 || t == 5 || t == 6), y = (t == 2 || t == 3 || t == 6 || t == 7),
              z = t >= 4;
    const bool on = f < 2 ? z == u : (f < 4 ? y == u : x == u);
    return on ? -3 : 0;
  }
  const int c = t - 8;  // edge samples of the face (indices into C)
  bool on;
  if (f < 2) on = c == 0 + 2 * u || c == 1 + 2 * u || c == 4 + 2 * u || c == 5 + 2 * u;
  else if (f < 4) on = c == u || c == u + 2 || c == 8 + 2 * u || c == 9 + 2 * u;
  else on = c == 4 + u || c == 6 + u || c == 8 + u || c == 10 + u;
  return on ? 1 : 0;
}

// The 20 samples of element e as exact integers (Sec. 5), by the whole warp:
// coordinates scaled to integers (sm[0, 96): 24 x 4 words), sample t in
// sm[96 + 12 t, +12) (lanes t < 20 compute them).  Returns false when the
// coordinates span more than kFastBits bits (then nothing is written).  All
// 32 lanes call it; `sm` holds kFastWords words.
__device__ __forceinline__ bool fast_samples_warp(const Batch& p, uint32_t e, uint32_t* sm) {
  const int lane = threadIdx.x & 31;
  const int64_t g = p.base + e;
  // coordinate of this lane (lanes 0-23: node lane / 3, axis lane % 3)
  double v = 0.0;
  if (!p.indexed) {
    if (lane < 24) v = __ldg(p.soa + lane * p.stride + g);
  } else {
    int id = lane < 8 ? __ldg(p.conn + 8 * g + lane) : 0;
    int nid = __shfl_sync(kFull, id, (lane < 24 ? lane : 0) / 3);
    if (lane < 24) v = __ldg(p.nodes + 3 * static_cast<int64_t>(nid) + lane % 3);
  }
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  const int ex = static_cast<int>((bits >> 52) & 0x7ff);
  unsigned long long m = bits & 0xfffffffffffffull;
  if (ex) m |= 1ull << 52;
  int q = (ex ? ex : 1) - 1075;
  if (lane >= 24) m = 0;
  int qlo = 1 << 20, qhi = -(1 << 20);
  if (m) {
    const int tz = __ffsll(static_cast<long long>(m)) - 1;
    m >>= tz;
    q += tz;
    qlo = q;
    qhi = q + 63 - __clzll(static_cast<long long>(m));
  }
  const int qmin = __reduce_min_sync(kFull, qlo), top = __reduce_max_sync(kFull, qhi);
  const int B = top >= qmin ? top - qmin + 1 : 0;
  if (B > kFastBits) return false;
  uint32_t* Xs = sm;        // 24 coordinates x 4 words
  uint32_t* Ss = sm + 96;   // 20 samples x 12 words
  if (lane < 24) {
    Wide<4> x;
    const int sh = m ? q - qmin : 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int lo = 32 * i - sh;  // bit of m that lands at bit 0 of word i
      unsigned long long w = 0;
      if (lo >= 0) w = lo < 64 ? (m >> lo) : 0ull;
      else if (lo > -64) w = m << (-lo);
      x.v[i] = static_cast<uint32_t>(w);
    }
    if (bits >> 63) x = wneg(x);
#pragma unroll
    for (int i = 0; i < 4; ++i) Xs[4 * lane + i] = x.v[i];
  }
  __syncwarp();
  if (lane < 20) {  // sample `lane`: det(A, B, C) = A . (B x C)
    int ia, ib, ic;
    sample_columns(lane, ia, ib, ic);
    Wide<4> A[3], Bv[3], C[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      A[d] = column(Xs, ia, d);
      Bv[d] = column(Xs, ib, d);
      C[d] = column(Xs, ic, d);
    }
    Wide<12> acc;
#pragma unroll
    for (int i = 0; i < 12; ++i) acc.v[i] = 0u;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
      const Wide<8> cr = wsub(wmul(Bv[d1], C[d2]), wmul(Bv[d2], C[d1]));
      acc = wadd(acc, wmul(A[d], cr));
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) Ss[12 * lane + i] = acc.v[i];
  }
  __syncwarp();
  return true;
}

// Scaled Table t:Tsmall coefficient of class lane L (0-7 corners, 8-19 edges,
// 20-25 faces, 26 centre; as in fp64_element_warp) from the samples in Ss,
// modulo 2^384.
__device__ __forceinline__ Wide<12> class_value(const uint32_t* Ss, int L) {
  Wide<12> acc;
  if (L < 8) {
#pragma unroll
    for (int i = 0; i < 12; ++i) acc.v[i] = Ss[12 * L + i];
    return acc;
  }
#pragma unroll
  for (int i = 0; i < 12; ++i) acc.v[i] = 0u;
  for (int t = 0; t < 20; ++t) {
    const int wgt = q_weight(L, t);
    if (wgt == 0) continue;
    const unsigned int a = static_cast<unsigned int>(wgt < 0 ? -wgt : wgt);
    Wide<12> term;
    unsigned long long c = 0;
#pragma unroll
    for (int i = 0; i < 12; ++i) {  // a x sample t, modulo 2^384
      c += static_cast<unsigned long long>(a) * Ss[12 * t + i];
      term.v[i] = static_cast<uint32_t>(c);
      c >>= 32;
    }
    acc = wgt < 0 ? wsub(acc, term) : wadd(acc, term);
  }
  return acc;
}

// Flag byte (without the exact bit) of element e if it is decided at depth
// 0; -1 when it needs refinement (every sample > 0, a coefficient <= 0); -2
// when its coordinates are outside the fast range.  All 32 lanes call it;
// `sm` holds kFastWords words.
static __device__ __noinline__ int exact_depth0_warp(const Batch& p, uint32_t e, uint32_t* sm) {
  const int lane = threadIdx.x & 31;
  if (!fast_samples_warp(p, e, sm)) return -2;
  const uint32_t* Ss = sm + 96;
  bool pos = true;
  if (lane < 20) {
    Wide<12> acc;
#pragma unroll
    for (int i = 0; i < 12; ++i) acc.v[i] = Ss[12 * lane + i];
    pos = wpositive(acc);
  }
  if (__any_sync(kFull, !pos)) return make_flag(kVInvalid, 0, 0);  // Step 2
  bool cpos = true;  // corners (lanes 0-7) are the positive samples
  if (lane >= 8 && lane < 27) cpos = wpositive(class_value(Ss, lane));
  if (__all_sync(kFull, cpos)) return make_flag(kVValid, 0, 0);  // Step 4
  return -1;
}

// Exact signs of the coefficients of one box of the refinement: the box of
// depth `level` at dyadic position (x, y, z) = pos (16 bits each) of element
// e.  The root coefficients b (Table t:Tsmall) as integers scaled by 8 (and
// by the coordinate scaling, a positive power of 2) in 480-bit words; then,
// along xi, eta and zeta in turn, the Bernstein coefficients of the quadratic
// on [s/n, (s+1)/n] (n = 2^level) scaled by n^2, exactly what `level`
// halvings by de Casteljau give, up to that positive factor:
//   n^2 c0 = (n-s)^2 b0 + 2 s (n-s) b1 + s^2 b2
//   n^2 c1 = (n-s)(n-s-1) b0 + ((n-s)(s+1) + s(n-s-1)) b1 + s(s+1) b2
//   n^2 c2 = (n-s-1)^2 b0 + 2 (s+1)(n-s-1) b1 + (s+1)^2 b2.
// Widths: |8 b| < 2^377, every pass multiplies the magnitude by at most n^2 <=
// 2^30, so the values stay below 2^467 < 2^479.  Returns 0 (a corner
// coefficient <= 0), 1 (all 27 > 0), 2 (corners > 0, another <= 0), or -1
// when the coordinates are outside the fast tier's range.  All 32 lanes call
// it; `sm` holds at least 27 x 15 and kFastWords words.
constexpr int kBoxWords = 15;
static __device__ __noinline__ int exact_box_warp(const Batch& p, uint32_t e, int level,
                                                  uint64_t pos, uint32_t* sm) {
  const int lane = threadIdx.x & 31;
  if (!fast_samples_warp(p, e, sm)) return -1;
  Wide<kBoxWords> c;
  int t = 0;  // tensor position i + 3 j + 9 k of this lane's coefficient
  if (lane < 27) {
    const Wide<12> v = class_value(sm + 96, lane);
    // unscaled x 8: corners c x 8, edges 2b x 4, faces 4b x 2, centre 8b
    const int sh = lane < 8 ? 3 : (lane < 20 ? 2 : (lane < 26 ? 1 : 0));
    c = wext<kBoxWords>(v);
    for (int r = 0; r < sh; ++r) c = wadd(c, c);
    t = lane < 8 ? corner_t(lane)
                 : (lane < 20 ? edge_t(lane - 8) : (lane < 26 ? face_t(lane - 20) : tix(1, 1, 1)));
  }
  __syncwarp();
  uint32_t* W = sm;  // [27][kBoxWords], over the samples (read above)
  if (lane < 27)
#pragma unroll
    for (int i = 0; i < kBoxWords; ++i) W[kBoxWords * t + i] = c.v[i];
  __syncwarp();
  const unsigned int n = 1u << level;
  const int ti = lane % 3, tj = (lane / 3) % 3, tk = lane / 9;  // lane = tensor position now
  for (int axis = 0; axis < 3; ++axis) {
    const unsigned int s = static_cast<unsigned int>((pos >> (16 * axis)) & 0xffffu);
    const int r = axis == 0 ? ti : (axis == 1 ? tj : tk);  // output index along the axis
    const unsigned int a = n - s, b = s + 1, am = n - s - 1;
    unsigned int w[3];
    if (r == 0) { w[0] = a * a; w[1] = 2u * s * a; w[2] = s * s; }
    else if (r == 1) { w[0] = a * am; w[1] = a * b + s * am; w[2] = s * b; }
    else { w[0] = am * am; w[1] = 2u * b * am; w[2] = b * b; }
    Wide<kBoxWords> acc;
#pragma unroll
    for (int i = 0; i < kBoxWords; ++i) acc.v[i] = 0u;
    if (lane < 27) {
      const int stride = axis == 0 ? 1 : (axis == 1 ? 3 : 9);
      const int base = lane - r * stride;
      for (int m = 0; m < 3; ++m) {
        const uint32_t* src = W + kBoxWords * (base + m * stride);
        Wide<kBoxWords> term;
        unsigned long long cy = 0;
#pragma unroll
        for (int i = 0; i < kBoxWords; ++i) {  // w[m] x coefficient, modulo 2^480
          cy += static_cast<unsigned long long>(w[m]) * src[i];
          term.v[i] = static_cast<uint32_t>(cy);
          cy >>= 32;
        }
        acc = wadd(acc, term);
      }
    }
    __syncwarp();
    if (lane < 27)
#pragma unroll
      for (int i = 0; i < kBoxWords; ++i) W[kBoxWords * lane + i] = acc.v[i];
    __syncwarp();
    c = acc;
  }
  const bool corner = lane < 27 && ti != 1 && tj != 1 && tk != 1;
  const bool positive = lane < 27 && wpositive(c);
  if (__any_sync(kFull, corner && !positive)) return 0;
  if (__all_sync(kFull, lane >= 27 || positive)) return 1;
  return 2;
}

}  // namespace exact_tier
}  // namespace hexval
