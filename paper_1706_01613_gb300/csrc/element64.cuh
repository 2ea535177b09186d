// FP64 element routine of the bulk pass (Sec. 6, Steps 1-4), shared by the
// FP64 bulk kernel and by the tail kernel that redoes the elements escalated
// by the FP32 pass.
//
// Error bound (u = 2^-53, L = largest |component| of the 12 computed edge
// vectors): every sample and coefficient is within 930 u L^3 of its exact
// value; E = 2^(3 e_L - 3107) >= 2^-42 L^3 with e_L the biased exponent of L.
#pragma once

#include "hexval_internal.cuh"

namespace hexval {

// The escalation keys of the scaled classes: x2 edge coefficients, x4 face
// coefficients and edge samples (C = 4 J), x8 centre.
struct Keys {
  uint32_t k1, k2, k4, k8;
};
__device__ __forceinline__ Keys keys_d(double E) {
  uint32_t k = dhi(E);
  return {k, k + (1u << 20), k + (2u << 20), k + (3u << 20)};
}
__device__ __forceinline__ Keys keys_f(float E) {
  uint32_t k = fbits(E);
  return {k, k + (1u << 23), k + (2u << 23), k + (3u << 23)};
}

__device__ __forceinline__ Sign3 sign_k(double v, uint32_t k) { return sign_d(v, k); }
__device__ __forceinline__ Sign3 sign_k(float v, uint32_t k) { return sign_f(v, k); }

// Depth-0 classification of the scaled coefficients (Sec. 6, Steps 2 and 4).
// Returns 0 invalid, 1 valid, 2 refine, 3 ambiguous.
template <typename T>
__device__ __forceinline__ int classify_root(const Scaled<T>& s, const Keys& K) {
  bool nonpos = false, amb = false;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    Sign3 q = sign_k(s.corner[k], K.k1);
    nonpos |= q.nonpos;
    amb |= !(q.nonpos | q.pos);
  }
#pragma unroll
  for (int e = 0; e < 12; ++e) {
    Sign3 q = sign_k(s.edgeC[e], K.k4);
    nonpos |= q.nonpos;
    amb |= !(q.nonpos | q.pos);
  }
  if (nonpos) return 0;
  if (amb) return 3;
  bool notcert = false;
  amb = false;
#pragma unroll
  for (int e = 0; e < 12; ++e) {
    Sign3 q = sign_k(s.edge[e], K.k2);
    notcert |= q.nonpos;
    amb |= !(q.nonpos | q.pos);
  }
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    Sign3 q = sign_k(s.face[f], K.k4);
    notcert |= q.nonpos;
    amb |= !(q.nonpos | q.pos);
  }
  {
    Sign3 q = sign_k(s.centre, K.k8);
    notcert |= q.nonpos;
    amb |= !(q.nonpos | q.pos);
  }
  if (notcert) return 2;
  if (amb) return 3;
  return 1;
}

// min / max of the 27 unscaled coefficients, FP64 (integer keys per class,
// then the class extremes are unscaled exactly).
__device__ __forceinline__ void minmax_d(const Scaled<double>& s, double& lo, double& hi) {
  long long mn[4], mx[4];
  mn[0] = mx[0] = dkey(s.corner[0]);
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    long long q = dkey(s.corner[k]);
    mn[0] = min(mn[0], q);
    mx[0] = max(mx[0], q);
  }
  mn[1] = mx[1] = dkey(s.edge[0]);
#pragma unroll
  for (int e = 1; e < 12; ++e) {
    long long q = dkey(s.edge[e]);
    mn[1] = min(mn[1], q);
    mx[1] = max(mx[1], q);
  }
  mn[2] = mx[2] = dkey(s.face[0]);
#pragma unroll
  for (int f = 1; f < 6; ++f) {
    long long q = dkey(s.face[f]);
    mn[2] = min(mn[2], q);
    mx[2] = max(mx[2], q);
  }
  mn[3] = mx[3] = dkey(s.centre);
  long long a = min(min(mn[0], dkey(dunkey(mn[1]) * 0.5)),
                    min(dkey(dunkey(mn[2]) * 0.25), dkey(dunkey(mn[3]) * 0.125)));
  long long b = max(max(mx[0], dkey(dunkey(mx[1]) * 0.5)),
                    max(dkey(dunkey(mx[2]) * 0.25), dkey(dunkey(mx[3]) * 0.125)));
  lo = dunkey(a);
  hi = dunkey(b);
}

__device__ __forceinline__ bool nonfinite_d(const V3<double> X[8]) {
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    acc |= ((dhi(X[k].x) & 0x7ff00000u) == 0x7ff00000u);
    acc |= ((dhi(X[k].y) & 0x7ff00000u) == 0x7ff00000u);
    acc |= ((dhi(X[k].z) & 0x7ff00000u) == 0x7ff00000u);
  }
  return acc != 0;
}

// Stores everything a refined element needs and its root box (level 0).
__device__ __forceinline__ void push_root(const Batch& p, unsigned int slot, uint32_t e,
                                          const Scaled<double>& s, double E, double M) {
  const Scratch& S = p.s;
  S.slot_elem[slot] = e;
  S.slot_state[slot] = 0u;
  S.slot_lev[slot] = 0u;
  S.slot_e0[slot] = E;
  S.slot_m0[slot] = M;
  S.qslot[0][slot] = slot;
  if (S.qpos[0]) S.qpos[0][slot] = 0ull;
  double t[27];
  store_tensor(s, t);
#pragma unroll
  for (int q = 0; q < 27; ++q) S.qcoef[0][q * S.qcap + slot] = t[q];
}

// Processes element e of the batch in FP64 (act = false: idle lane, which
// still takes part in the warp-aggregated appends).  Writes the verdict when
// it is decided at depth 0; otherwise appends the element to level 0 of the
// refinement queue or to the exact list.  Must be called by all 32 lanes.
__device__ __forceinline__ void fp64_element(const Batch& p, bool act, uint32_t e) {
  const Scratch& S = p.s;
  int64_t g = p.base + e;
  V3<double> X[8];
  int outcome = -1;  // 0 inv, 1 valid, 2 refine, 3 exact, 4 nonfinite, 5 bad index, 6 cap
  Scaled<double> s;
  double E = 0.0, lo = 0.0, hi = 0.0;
  if (act) {
    if (!load_element(p, g, X)) {
      outcome = 5;
    } else if (nonfinite_d(X)) {
      outcome = 4;
    } else {
      V3<double> a[4], b[4], gg[4];
      edges_from_nodes(X, a, b, gg);
      coefficients_from_edges(a, b, gg, s);
      int emax = max_exponent_d(a, b, gg);
      E = pow2d(min(3 * emax - 3107, 1000));
      outcome = classify_root(s, keys_d(E));
      minmax_d(s, lo, hi);
      if (outcome == 2 && p.max_depth == 0) outcome = 6;  // cap at the root
    }
  }
  bool want_q = act && outcome == 2;
  unsigned int slot = warp_append(&S.cnt->level_count[0], want_q);
  bool overflow = want_q && slot >= S.qcap;
  if (want_q && !overflow) {
    double M = fmax(fabs(lo), fabs(hi)) + E;
    push_root(p, slot, e, s, E, M);
  }
  bool want_x = act && (outcome == 3 || overflow);
  unsigned int xpos = warp_append(&S.cnt->exact_count, want_x);
  if (!act) return;
  uint8_t flag = 0;
  bool write = true;
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  switch (outcome) {
    case 0: flag = make_flag(kVInvalid, 0, 0); break;
    case 1: flag = make_flag(kVValid, 0, 0); break;
    case 4: flag = make_flag(kVNonfinite, 0, 0); lo = hi = qnan; break;
    case 5: flag = make_flag(kVUndecided, 0, 0); lo = hi = qnan; set_status(S.status, kSbIndex); break;
    case 6: flag = make_flag(kVUndecided, 0, 0); break;
    default: write = false; break;
  }
  if (want_x) {
    if (xpos < S.exact_cap) {
      S.exact_list[xpos] = e;
    } else {
      flag = make_flag(kVUndecided, 0, 0);
      write = true;
      set_status(S.status, kSbQueue);
    }
  }
  if (overflow) set_status(S.status, kSbQueue);
  if (write) p.flags[g] = flag;
  if (p.bmin) p.bmin[g] = lo;
  if (p.bmax) p.bmax[g] = hi;
}

// ------------------------------------------ redo of the unsettled signs ----
// FP64 sample q of an element from its edge vectors (q < 8: corner node q;
// otherwise the sample of edge q - 8, C = 4 J at its midpoint), with the
// operations coefficients_from_edges uses for it, so within its FP64 bound.
static __device__ __noinline__ double sample64(const V3<double>* a, const V3<double>* b,
                                               const V3<double>* g, int q) {
  switch (q) {
    case 0: return det3(a[0], b[0], g[0]);
    case 1: return det3(a[0], b[1], g[1]);
    case 2: return det3(a[1], b[1], g[3]);
    case 3: return det3(a[1], b[0], g[2]);
    case 4: return det3(a[2], b[2], g[0]);
    case 5: return det3(a[2], b[3], g[1]);
    case 6: return det3(a[3], b[3], g[3]);
    case 7: return det3(a[3], b[2], g[2]);
    case 8: return det3(a[0], vadd(b[0], b[1]), vadd(g[0], g[1]));
    case 9: return det3(a[1], vadd(b[0], b[1]), vadd(g[2], g[3]));
    case 10: return det3(a[2], vadd(b[2], b[3]), vadd(g[0], g[1]));
    case 11: return det3(a[3], vadd(b[2], b[3]), vadd(g[2], g[3]));
    case 12: return det3(vadd(a[0], a[1]), b[0], vadd(g[0], g[2]));
    case 13: return det3(vadd(a[0], a[1]), b[1], vadd(g[1], g[3]));
    case 14: return det3(vadd(a[2], a[3]), b[2], vadd(g[0], g[2]));
    case 15: return det3(vadd(a[2], a[3]), b[3], vadd(g[1], g[3]));
    case 16: return det3(vadd(a[0], a[2]), vadd(b[0], b[2]), g[0]);
    case 17: return det3(vadd(a[0], a[2]), vadd(b[1], b[3]), g[1]);
    case 18: return det3(vadd(a[1], a[3]), vadd(b[0], b[2]), g[2]);
    case 19: return det3(vadd(a[1], a[3]), vadd(b[1], b[3]), g[3]);
    default: return 0.0;
  }
}

// FP64 edge coefficient e (scaled by 2, as Scaled::edge): the edge sample
// less the corner samples of the edge's two end nodes, as
// coefficients_from_edges forms it.
static __device__ __noinline__ double edge64(const V3<double>* a, const V3<double>* b,
                                             const V3<double>* g, int e) {
  int ca, cb;
  if (e < 4) {  // xi-edge at (eta, zeta) = (e & 1, e >> 1)
    ca = node_at(0, e & 1, e >> 1);
    cb = node_at(1, e & 1, e >> 1);
  } else if (e < 8) {  // eta-edge at (xi, zeta)
    ca = node_at((e - 4) & 1, 0, (e - 4) >> 1);
    cb = node_at((e - 4) & 1, 1, (e - 4) >> 1);
  } else {  // zeta-edge at (xi, eta)
    ca = node_at((e - 8) & 1, (e - 8) >> 1, 0);
    cb = node_at((e - 8) & 1, (e - 8) >> 1, 1);
  }
  return sample64(a, b, g, 8 + e) - sample64(a, b, g, ca) - sample64(a, b, g, cb);
}

// Depth-0 decision of an element the FP32 pass escalated, redoing in FP64
// only the signs FP32 left unsettled (mask: fp32_unsettled), each with the
// bound of the full FP64 evaluation (fp64_element: the same E from the same
// FP64 edge vectors).  A redone sample certainly <= 0 makes the element
// INVALID (Sec. 6, Step 2); all samples and all 27 coefficients certainly
// positive -- those FP32 certified and those redone -- make it VALID (Step 4).
// X: the element's nodes.  Returns 0 (INVALID@0), 1 (VALID@0), or -1 when
// the full FP64 evaluation is needed (a sign still unsettled, a face or
// centre coefficient, a coefficient certainly <= 0, non-finite coordinates).
__device__ __forceinline__ int fp64_partial(const V3<double> X[8], uint64_t mask) {
  if (nonfinite_d(X)) return -1;
  V3<double> a[4], b[4], gg[4];
  edges_from_nodes(X, a, b, gg);
  const Keys K = keys_d(pow2d(min(3 * max_exponent_d(a, b, gg) - 3107, 1000)));
  bool open = false;
  for (uint32_t m = static_cast<uint32_t>(mask) & 0xfffffu; m; m &= m - 1) {
    const int q = __ffs(m) - 1;
    const Sign3 c = sign_d(sample64(a, b, gg, q), q < 8 ? K.k1 : K.k4);
    if (c.nonpos) return 0;
    open |= !c.pos;
  }
  if (open || (mask >> 32)) return -1;
  for (uint32_t m = static_cast<uint32_t>(mask >> 20) & 0xfffu; m; m &= m - 1)
    if (!sign_d(edge64(a, b, gg, __ffs(m) - 1), K.k2).pos) return -1;
  return 1;
}

}  // namespace hexval
