// Exact tier: elements whose verdict depends on a sign that the FP64 error
// bound cannot settle are recomputed in exact integer arithmetic.
//
// Every FP64 coordinate is M * 2^q with an integer M; scaling all 24 by
// 2^-qmin (qmin the lowest set bit among them) makes them integers of at most
// B bits.  The 20 samples of J (Sec. 5) are then integers, the scaled Bezier
// coefficients 8 b (Table t:Tsmall) are integers, and a de Casteljau split
// with every output scaled by 4 stays integral, so the whole decision of
// Sec. 6 runs on integers.  Values are two's-complement multi-limb integers
// of W = 32 NL bits computed modulo 2^W; W is chosen per element so that
// every intermediate (at most 3B + 13 + 6 D bits plus sign) fits, which makes
// the modular results exact.
//
// The refinement is a depth-first walk that evaluates the same order-free
// verdict as the breadth-first kernels: INVALID at the shallowest level
// holding a non-positive corner coefficient, else UNDECIDED if an uncertified
// box reached the cap, else VALID at the deepest certified box.  Boxes at or
// below the best INVALID level found so far are not expanded.
//
// Working storage: per worker thread, 592 integers of up to 32 limbs in the
// handle's scratch, interleaved across workers (limb w of worker t at
// w * n_workers + t) so that a warp's accesses coalesce.
#pragma once

#include "hexval_internal.cuh"

namespace hexval {

namespace exact_tier {

constexpr int kLimbsMax = 32;
constexpr int kWorkers = 512;  // threads that may work on the exact list at once
constexpr int kStackInts = (kMaxDepth + 1) * 27;
constexpr int kTempInts = 160;
constexpr int kInts = kStackInts + kTempInts;
constexpr unsigned long long kMaxBoxes = 1ull << 22;  // work bound per element

struct Ws {
  uint32_t* base;
  uint32_t t;
  __device__ __forceinline__ uint32_t& w(uint32_t int_id, uint32_t limb) const {
    return base[(static_cast<uint64_t>(int_id) * kLimbsMax + limb) * kWorkers + t];
  }
};

template <int NL>
struct Big {
  const Ws& ws;
  __device__ void zero(uint32_t r) const {
#pragma unroll 1
    for (int i = 0; i < NL; ++i) ws.w(r, i) = 0u;
  }
  // r = +-(m << sh), m < 2^53
  __device__ void set(uint32_t r, unsigned long long m, int sh, bool neg) const {
    #pragma unroll 1
    for (int i = 0; i < NL; ++i) {
      int lo = 32 * i - sh;  // bit of m that lands at limb i, bit 0
      unsigned long long v = 0;
      if (lo >= 0) {
        v = lo < 64 ? (m >> lo) : 0ull;
      } else if (lo > -64) {
        v = m << (-lo);
      }
      ws.w(r, i) = static_cast<uint32_t>(v);
    }
    if (neg) negate(r);
  }
  __device__ void negate(uint32_t r) const {
    unsigned long long c = 1;
    #pragma unroll 1
    for (int i = 0; i < NL; ++i) {
      c += static_cast<uint32_t>(~ws.w(r, i));
      ws.w(r, i) = static_cast<uint32_t>(c);
      c >>= 32;
    }
  }
  // r = a + b  (r may alias)
  __device__ void add(uint32_t r, uint32_t a, uint32_t b) const {
    unsigned long long c = 0;
    #pragma unroll 1
    for (int i = 0; i < NL; ++i) {
      c += static_cast<unsigned long long>(ws.w(a, i)) + ws.w(b, i);
      ws.w(r, i) = static_cast<uint32_t>(c);
      c >>= 32;
    }
  }
  // r = a - b
  __device__ void sub(uint32_t r, uint32_t a, uint32_t b) const {
    unsigned long long c = 1;
    #pragma unroll 1
    for (int i = 0; i < NL; ++i) {
      c += static_cast<unsigned long long>(ws.w(a, i)) + static_cast<uint32_t>(~ws.w(b, i));
      ws.w(r, i) = static_cast<uint32_t>(c);
      c >>= 32;
    }
  }
  // r = wa a + wb b + wc c  with small non-negative weights (mod 2^W)
  __device__ void lin3(uint32_t r, uint32_t a, uint32_t wa, uint32_t b, uint32_t wb, uint32_t c,
                       uint32_t wc) const {
    unsigned long long carry = 0;
    #pragma unroll 1
    for (int i = 0; i < NL; ++i) {
      unsigned long long acc = carry + static_cast<unsigned long long>(wa) * ws.w(a, i) +
                               static_cast<unsigned long long>(wb) * ws.w(b, i) +
                               static_cast<unsigned long long>(wc) * ws.w(c, i);
      ws.w(r, i) = static_cast<uint32_t>(acc);
      carry = acc >> 32;
    }
  }
  // r = a * b mod 2^W (r must not alias a or b)
  __device__ void mul(uint32_t r, uint32_t a, uint32_t b) const {
    zero(r);
    #pragma unroll 1
    for (int i = 0; i < NL; ++i) {
      unsigned long long ai = ws.w(a, i);
      if (!ai) continue;
      unsigned long long carry = 0;
#pragma unroll 1
      for (int j = 0; i + j < NL; ++j) {
        unsigned long long t = ai * ws.w(b, j) + ws.w(r, i + j) + carry;
        ws.w(r, i + j) = static_cast<uint32_t>(t);
        carry = t >> 32;
      }
    }
  }
  // -1, 0, +1
  __device__ int sign(uint32_t a) const {
    if (ws.w(a, NL - 1) >> 31) return -1;
#pragma unroll 1
    for (int i = 0; i < NL; ++i)
      if (ws.w(a, i)) return 1;
    return 0;
  }
};

// temp integer ids
constexpr uint32_t T0 = kStackInts;  // 24 coordinates: T0 + 3k + d
constexpr uint32_t TE = T0 + 24;     // 12 edge vectors a[4], b[4], g[4]: TE + 3q + d
constexpr uint32_t TS = TE + 36;     // 12 sums: TS + 3q + d
constexpr uint32_t TC = TS + 36;     // 8 corner samples
constexpr uint32_t TCE = TC + 8;     // 12 edge samples (4 J)
constexpr uint32_t TX = TCE + 12;    // scratch for products and sums (>= 12)
constexpr uint32_t TP = TX + 16;     // 27 pass buffer
static_assert(TP + 27 <= kInts, "temp region too small");

template <int NL>
struct Exact {
  Big<NL> B;

  // det(A, B, C) = A . (B x C) into r (uses TX..TX+5)
  __device__ void det(uint32_t r, uint32_t A, uint32_t Bv, uint32_t C) const {
    const uint32_t t0 = TX, t1 = TX + 1, cr = TX + 2, acc = TX + 5;
    // cross components into cr..cr+2
    for (int d = 0; d < 3; ++d) {
      int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
      B.mul(t0, Bv + d1, C + d2);
      B.mul(t1, Bv + d2, C + d1);
      B.sub(cr + d, t0, t1);
    }
    B.zero(acc);
    for (int d = 0; d < 3; ++d) {
      B.mul(t0, A + d, cr + d);
      B.add(acc, acc, t0);
    }
#pragma unroll 1
    for (int i = 0; i < NL; ++i) B.ws.w(r, i) = B.ws.w(acc, i);
  }

  // one de Casteljau pass (scaled by 4) along `axis` taking half `side`
  // from integers src (27, tensor order) into dst
  __device__ void pass(uint32_t src, uint32_t dst, int axis, int side) const {
    const int step = axis == 0 ? 1 : (axis == 1 ? 3 : 9);
    for (int u = 0; u < 3; ++u)
      for (int v = 0; v < 3; ++v) {
        int o = axis == 0 ? (3 * u + 9 * v) : (axis == 1 ? (u + 9 * v) : (u + 3 * v));
        uint32_t p0 = src + o, p1 = src + o + step, p2 = src + o + 2 * step;
        uint32_t q0 = dst + o, q1 = dst + o + step, q2 = dst + o + 2 * step;
        if (side == 0) {  // (4 p0, 2 p0 + 2 p1, p0 + 2 p1 + p2)
          B.lin3(q2, p0, 1, p1, 2, p2, 1);
          B.lin3(q1, p0, 2, p1, 2, p2, 0);
          B.lin3(q0, p0, 4, p1, 0, p2, 0);
        } else {          // (p0 + 2 p1 + p2, 2 p1 + 2 p2, 4 p2)
          B.lin3(q0, p0, 1, p1, 2, p2, 1);
          B.lin3(q1, p0, 0, p1, 2, p2, 2);
          B.lin3(q2, p0, 0, p1, 0, p2, 4);
        }
      }
  }

  // classification of the box at `lv`: 0 INVALID corner, 1 certified, 2 refine
  __device__ int classify(uint32_t lv) const {
    const uint32_t b0 = lv * 27;
    for (int k = 0; k < 3; k += 2)
      for (int j = 0; j < 3; j += 2)
        for (int i = 0; i < 3; i += 2)
          if (B.sign(b0 + tix(i, j, k)) <= 0) return 0;
    for (int t = 0; t < 27; ++t) {
      int i = t % 3, j = (t / 3) % 3, k = t / 9;
      if (i == 1 || j == 1 || k == 1)
        if (B.sign(b0 + t) <= 0) return 2;
    }
    return 1;
  }

  // Returns the flag byte (without the exact bit), or -1 if the work bound
  // was exceeded.
  __device__ int run(const unsigned long long M[24], const int sh[24], const bool neg[24],
                     int max_depth) const {
    for (int q = 0; q < 24; ++q) B.set(T0 + q, M[q], sh[q], neg[q]);
    // edge vectors (Sec. 5): a along xi, b along eta, g along zeta
    for (int z = 0; z < 2; ++z)
      for (int y = 0; y < 2; ++y)
        for (int d = 0; d < 3; ++d)
          B.sub(TE + 3 * (y + 2 * z) + d, T0 + 3 * node_at(1, y, z) + d, T0 + 3 * node_at(0, y, z) + d);
    for (int z = 0; z < 2; ++z)
      for (int x = 0; x < 2; ++x)
        for (int d = 0; d < 3; ++d)
          B.sub(TE + 12 + 3 * (x + 2 * z) + d, T0 + 3 * node_at(x, 1, z) + d,
                T0 + 3 * node_at(x, 0, z) + d);
    for (int y = 0; y < 2; ++y)
      for (int x = 0; x < 2; ++x)
        for (int d = 0; d < 3; ++d)
          B.sub(TE + 24 + 3 * (x + 2 * y) + d, T0 + 3 * node_at(x, y, 1) + d,
                T0 + 3 * node_at(x, y, 0) + d);
    auto A_ = [](int q) { return TE + 3 * q; };
    auto B_ = [](int q) { return TE + 12 + 3 * q; };
    auto G_ = [](int q) { return TE + 24 + 3 * q; };
    // sums of parallel edges: sb[u], sg[u], sa[u], sg2[u], sa2[u], sb2[u]
    for (int u = 0; u < 2; ++u)
      for (int d = 0; d < 3; ++d) {
        B.add(TS + 3 * (0 + u) + d, B_(0 + 2 * u) + d, B_(1 + 2 * u) + d);
        B.add(TS + 3 * (2 + u) + d, G_(0 + 2 * u) + d, G_(1 + 2 * u) + d);
        B.add(TS + 3 * (4 + u) + d, A_(0 + 2 * u) + d, A_(1 + 2 * u) + d);
        B.add(TS + 3 * (6 + u) + d, G_(u) + d, G_(u + 2) + d);
        B.add(TS + 3 * (8 + u) + d, A_(u) + d, A_(u + 2) + d);
        B.add(TS + 3 * (10 + u) + d, B_(u) + d, B_(u + 2) + d);
      }
    auto S_ = [](int q) { return TS + 3 * q; };
    // samples: corners c, edge midpoints C = 4 J
    for (int z = 0; z < 2; ++z)
      for (int y = 0; y < 2; ++y)
        for (int x = 0; x < 2; ++x)
          det(TC + node_at(x, y, z), A_(y + 2 * z), B_(x + 2 * z), G_(x + 2 * y));
    for (int z = 0; z < 2; ++z)
      for (int y = 0; y < 2; ++y) det(TCE + y + 2 * z, A_(y + 2 * z), S_(0 + z), S_(2 + y));
    for (int z = 0; z < 2; ++z)
      for (int x = 0; x < 2; ++x) det(TCE + 4 + x + 2 * z, S_(4 + z), B_(x + 2 * z), S_(6 + x));
    for (int y = 0; y < 2; ++y)
      for (int x = 0; x < 2; ++x) det(TCE + 8 + x + 2 * y, S_(8 + y), S_(10 + x), G_(x + 2 * y));
    // Step 2: a non-positive sample -> INVALID at depth 0
    for (int k = 0; k < 8; ++k)
      if (B.sign(TC + k) <= 0) return make_flag(kVInvalid, 0, 0);
    for (int e = 0; e < 12; ++e)
      if (B.sign(TCE + e) <= 0) return make_flag(kVInvalid, 0, 0);
    // Step 3: 8 b in tensor order at stack level 0
    const uint32_t sc = TX + 8, sC = TX + 9, tmp = TX + 10;
    for (int k = 0; k < 8; ++k) B.lin3(corner_t(k), TC + k, 8, TC + k, 0, TC + k, 0);
    for (int e = 0; e < 12; ++e) {
      int x0, y0, z0, x1, y1, z1;
      if (e < 4) { x0 = 0; x1 = 1; y0 = y1 = e & 1; z0 = z1 = e >> 1; }
      else if (e < 8) { x0 = x1 = e & 1; y0 = 0; y1 = 1; z0 = z1 = (e - 4) >> 1; }
      else { x0 = x1 = e & 1; y0 = y1 = (e - 8) >> 1; z0 = 0; z1 = 1; }
      B.sub(tmp, TCE + e, TC + node_at(x0, y0, z0));
      B.sub(tmp, tmp, TC + node_at(x1, y1, z1));
      B.lin3(edge_t(e), tmp, 4, tmp, 0, tmp, 0);
    }
    // faces: 2 (sum of its 4 edge samples - 3 sum of its 4 corners)
    const int fe[6][4] = {{0, 1, 4, 5}, {2, 3, 6, 7}, {0, 2, 8, 9},
                          {1, 3, 10, 11}, {4, 6, 8, 10}, {5, 7, 9, 11}};
    for (int f = 0; f < 6; ++f) {
      B.zero(sc);
      B.zero(sC);
      for (int q = 0; q < 4; ++q) B.add(sC, sC, TCE + fe[f][q]);
      for (int z = 0; z < 2; ++z)
        for (int y = 0; y < 2; ++y)
          for (int x = 0; x < 2; ++x) {
            bool on = f == 0 ? z == 0 : f == 1 ? z == 1 : f == 2 ? y == 0
                    : f == 3 ? y == 1 : f == 4 ? x == 0 : x == 1;
            if (on) B.add(sc, sc, TC + node_at(x, y, z));
          }
      B.lin3(tmp, sc, 3, sc, 0, sc, 0);
      B.sub(tmp, sC, tmp);
      B.lin3(face_t(f), tmp, 2, tmp, 0, tmp, 0);
    }
    B.zero(sc);
    B.zero(sC);
    for (int e = 0; e < 12; ++e) B.add(sC, sC, TCE + e);
    for (int k = 0; k < 8; ++k) B.add(sc, sc, TC + k);
    B.lin3(tmp, sc, 5, sc, 0, sc, 0);
    B.sub(tix(1, 1, 1), sC, tmp);
    // Step 4
    bool cert = true;
    for (int t = 0; t < 27; ++t) cert &= B.sign(t) > 0;
    if (cert) return make_flag(kVValid, 0, 0);
    if (max_depth == 0) return make_flag(kVUndecided, 0, 0);
    // Step 5: depth-first walk
    int best = max_depth + 1, deepest = 0;
    bool cap = false;
    int child[kMaxDepth + 1];
    int depth = 0;
    child[0] = 0;
    unsigned long long boxes = 0;
    while (depth >= 0) {
      if (child[depth] == 8 || depth + 1 >= best) {
        --depth;
        continue;
      }
      int o = child[depth]++;
      if (++boxes > kMaxBoxes) return -1;
      const uint32_t par = depth * 27, kid = (depth + 1) * 27;
      pass(par, kid, 0, o & 1);
      pass(kid, TP, 1, (o >> 1) & 1);
      pass(TP, kid, 2, o >> 2);
      int d1 = depth + 1;
      int c = classify(d1);
      if (c == 0) {
        best = min(best, d1);
      } else if (c == 1) {
        deepest = max(deepest, d1);
      } else if (d1 >= max_depth) {
        cap = true;
      } else {
        depth = d1;
        child[depth] = 0;
      }
    }
    if (best <= max_depth) return make_flag(kVInvalid, best, 0);
    if (cap) return make_flag(kVUndecided, max_depth, 0);
    return make_flag(kVValid, deepest, 0);
  }
};

// Decides element e of the batch exactly and writes its flag (exact bit
// set).  `worker` < kWorkers selects the working storage.
static __device__ __noinline__ void exact_element(const Batch& p, uint32_t e, uint32_t worker) {
  const Scratch& S = p.s;
  Ws ws{S.exact_work, worker};
  int64_t g = p.base + e;
  V3<double> X[8];
  if (!load_element(p, g, X)) return;  // cannot happen: checked by the bulk pass
  unsigned long long M[24];
  int q[24];
  bool neg[24];
  int qmin = 1 << 20, top = -(1 << 20);
  for (int k = 0; k < 8; ++k)
    for (int d = 0; d < 3; ++d) {
      double v = d == 0 ? X[k].x : (d == 1 ? X[k].y : X[k].z);
      unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
      int ex = static_cast<int>((bits >> 52) & 0x7ff);
      unsigned long long m = bits & 0xfffffffffffffull;
      if (ex) m |= 1ull << 52;
      int qq = (ex ? ex : 1) - 1075;
      int idx = 3 * k + d;
      neg[idx] = bits >> 63;
      if (m) {
        int tz = __ffsll(static_cast<long long>(m)) - 1;
        m >>= tz;
        qq += tz;
        qmin = min(qmin, qq);
        top = max(top, qq + 63 - __clzll(static_cast<long long>(m)));
      }
      M[idx] = m;
      q[idx] = qq;
    }
  int Bbits = top >= qmin ? top - qmin + 1 : 0;
  int sh[24];
  for (int k = 0; k < 24; ++k) sh[k] = M[k] ? q[k] - qmin : 0;
  int need = 3 * Bbits + 17 + 6 * p.max_depth;
  int flag;
  if (need <= 256)
    flag = Exact<8>{Big<8>{ws}}.run(M, sh, neg, p.max_depth);
  else if (need <= 512)
    flag = Exact<16>{Big<16>{ws}}.run(M, sh, neg, p.max_depth);
  else if (need <= 1024)
    flag = Exact<32>{Big<32>{ws}}.run(M, sh, neg, p.max_depth);
  else
    flag = -1;
  if (flag < 0) {
    set_status(S.status, kSbRange);
    flag = make_flag(kVUndecided, p.max_depth, 0);
  }
  p.flags[g] = static_cast<uint8_t>(flag | 0x80);
}

}  // namespace exact_tier
}  // namespace hexval
