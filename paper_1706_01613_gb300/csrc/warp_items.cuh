// Warp-cooperative versions of the two FP64 work items of the tail kernel,
// for steps with few items.
//
// On this GPU a warp can issue an FP64 instruction only about every 64
// cycles, whatever the number of active lanes, so one thread working through
// the ~300 FP64 instructions of an element or of a box costs ~10 us of
// latency.  Here the 32 lanes of a warp share one item: the 24 coordinates,
// 36 edge components, 36 edge sums, 20 triple products and the Table
// t:Tsmall combinations of an element are spread over the lanes (about 30
// FP64 instructions per warp), and so are the 9 + 15 + 25 rows of the three
// de Casteljau passes of a box (18 FP64 instructions per warp).  Same
// arithmetic, same rounding per value and the same error bounds as the
// thread-per-item routines (element64.cuh and refine_box), hence the same
// results.  Each warp uses kWarpScratch doubles of shared memory.
#pragma once

#include "element64.cuh"

namespace hexval {

constexpr int kWarpScratch = 272;  // doubles per warp (box: 27 + 45 + 75 + 125)
// doubles per warp that fp64_element_warp needs: 116 for the element itself,
// the full kWarpScratch when it refines the element in-warp (refine_in_warp)
constexpr int kElemScratch = kWarpScratch;
constexpr unsigned int kFull = 0xffffffffu;

__device__ __forceinline__ double shfl_d(double v, int src) {
  return __shfl_sync(kFull, v, src);
}

// Corner node of the ends of edge vector q (0-3 along xi, 4-7 eta, 8-11 zeta).
__device__ __forceinline__ void edge_nodes(int q, int& lo, int& hi) {
  int u = q & 3;
  if (q < 4) {  // a[eta + 2 zeta]
    lo = node_at(0, u & 1, u >> 1);
    hi = node_at(1, u & 1, u >> 1);
  } else if (q < 8) {  // b[xi + 2 zeta]
    lo = node_at(u & 1, 0, u >> 1);
    hi = node_at(u & 1, 1, u >> 1);
  } else {  // g[xi + 2 eta]
    lo = node_at(u & 1, u >> 1, 0);
    hi = node_at(u & 1, u >> 1, 1);
  }
}

// The two edge vectors added by sum vector s (order of coefficients_from_edges:
// sb[0..1], sg[0..1], sa[0..1], sg2[0..1], sa2[0..1], sb2[0..1]); edge
// vector ids as in edge_nodes.
__device__ __forceinline__ void sum_parts(int s, int& e0, int& e1) {
  int u = s & 1;
  switch (s >> 1) {
    case 0: e0 = 4 + 2 * u; e1 = 5 + 2 * u; break;   // b[0+2u] + b[1+2u]
    case 1: e0 = 8 + 2 * u; e1 = 9 + 2 * u; break;   // g[0+2u] + g[1+2u]
    case 2: e0 = 0 + 2 * u; e1 = 1 + 2 * u; break;   // a[0+2u] + a[1+2u]
    case 3: e0 = 8 + u; e1 = 10 + u; break;          // g[u] + g[u+2]
    case 4: e0 = 0 + u; e1 = 2 + u; break;           // a[u] + a[u+2]
    default: e0 = 4 + u; e1 = 6 + u; break;          // b[u] + b[u+2]
  }
}

// Columns (vector ids: 0-11 edge vectors, 12-23 sums) of sample t
// (0-7 corners by node id, 8-19 edge midpoints in edgeC order).
__device__ __forceinline__ void sample_columns(int t, int& A, int& B, int& C) {
  if (t < 8) {
    int x = (t == 1 || t == 2 || t == 5 || t == 6), y = (t == 2 || t == 3 || t == 6 || t == 7),
        z = t >= 4;
    A = y + 2 * z;
    B = 4 + x + 2 * z;
    C = 8 + x + 2 * y;
    return;
  }
  int e = t - 8, u = e & 1, v = (e & 3) >> 1;
  if (e < 4) {  // xi-edge (eta=u, zeta=v): det(a[u+2v], sb[v], sg[u])
    A = u + 2 * v;
    B = 12 + 0 + v;
    C = 12 + 2 + u;
  } else if (e < 8) {  // eta-edge (xi=u, zeta=v): det(sa[v], b[u+2v], sg2[u])
    A = 12 + 4 + v;
    B = 4 + u + 2 * v;
    C = 12 + 6 + u;
  } else {  // zeta-edge (xi=u, eta=v): det(sa2[v], sb2[u], g[u+2v])
    A = 12 + 8 + v;
    B = 12 + 10 + u;
    C = 8 + u + 2 * v;
  }
}

// The 20 samples and 27 scaled coefficients of element g in FP64 by the
// whole warp (all 32 lanes), on `sm` (116 doubles): lane t < 20
// gets sample t (smp, scaled as in Scaled<>), lane L < 27 the scaled
// coefficient of class slot L (coef: 0-7 corners, 8-19 edges (2 b), 20-25
// faces (4 b), 26 centre (8 b)), and every lane the bound E of the unscaled
// coefficients (2^(3 e_L - 3107) >= 2^-42 L^3, as element64.cuh).  Returns
// 0, or 1 for a connectivity entry out of range, 2 for a non-finite
// coordinate (nothing else is then computed).
__device__ __forceinline__ int warp_root64(const Batch& p, int64_t g, double* sm, double& smp,
                                           double& coef, double& E) {
  const int lane = threadIdx.x & 31;
  double* Xs = sm;           // 24 coordinates [node][d]
  double* V = sm + 24;       // 24 vectors x 3 (0-11 edges, 12-23 sums)
  double* Sm = sm + 96;      // 20 samples (scaled as in Scaled<>)
  // coordinates
  bool bad = false;
  if (!p.indexed) {
    if (lane < 24) Xs[lane] = __ldg(p.soa + lane * p.stride + g);
  } else {
    int id = lane < 8 ? __ldg(p.conn + 8 * g + lane) : 0;
    bad = __any_sync(kFull, lane < 8 && !(id >= 0 && static_cast<int64_t>(id) < p.n_nodes));
    int nid = __shfl_sync(kFull, id, (lane < 24 ? lane : 0) / 3);
    if (!bad && lane < 24) Xs[lane] = __ldg(p.nodes + 3 * static_cast<int64_t>(nid) + lane % 3);
  }
  __syncwarp();
  if (bad) return 1;
  if (__any_sync(kFull, lane < 24 && (dhi(Xs[lane]) & 0x7ff00000u) == 0x7ff00000u)) return 2;
  // 12 edge vectors (36 components) and the bound's exponent
  uint32_t m = 0;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    int c = lane + 32 * r;
    if (c < 36) {
      int q = c / 3, d = c % 3, lo, hi;
      edge_nodes(q, lo, hi);
      double v = Xs[3 * hi + d] - Xs[3 * lo + d];
      V[c] = v;
      m = max(m, dhi(v) & 0x7fffffffu);
    }
  }
  m = __reduce_max_sync(kFull, m);
  __syncwarp();
  // 12 sums of parallel edges
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    int c = lane + 32 * r;
    if (c < 36) {
      int s = c / 3, d = c % 3, e0, e1;
      sum_parts(s, e0, e1);
      V[36 + c] = V[3 * e0 + d] + V[3 * e1 + d];
    }
  }
  __syncwarp();
  // 20 samples: lane t computes det of its three columns
  smp = 0.0;
  if (lane < 20) {
    int A, B, C;
    sample_columns(lane, A, B, C);
    V3<double> a{V[3 * A], V[3 * A + 1], V[3 * A + 2]};
    V3<double> b{V[3 * B], V[3 * B + 1], V[3 * B + 2]};
    V3<double> c{V[3 * C], V[3 * C + 1], V[3 * C + 2]};
    smp = det3(a, b, c);
    Sm[lane] = smp;
  }
  __syncwarp();
  // scaled Table t:Tsmall (same expressions as coefficients_from_edges)
  coef = 0.0;  // lanes 0-7 corners, 8-19 edges (2b), 20-25 faces (4b), 26 centre (8b)
  if (lane < 8) {
    coef = smp;
  } else if (lane < 20) {
    int ed = lane - 8, u = ed & 1, v = (ed & 3) >> 1, n0, n1;
    if (ed < 4) { n0 = node_at(0, u, v); n1 = node_at(1, u, v); }
    else if (ed < 8) { n0 = node_at(u, 0, v); n1 = node_at(u, 1, v); }
    else { n0 = node_at(u, v, 0); n1 = node_at(u, v, 1); }
    coef = Sm[lane] - Sm[n0] - Sm[n1];
  } else if (lane < 26) {
    int f = lane - 20, u = f & 1;
    double cs, es;
    const double* c = Sm;
    const double* C = Sm + 8;
    if (f < 2) {
      cs = (c[node_at(0, 0, u)] + c[node_at(1, 0, u)]) + (c[node_at(0, 1, u)] + c[node_at(1, 1, u)]);
      es = (C[0 + 2 * u] + C[1 + 2 * u]) + (C[4 + 2 * u] + C[5 + 2 * u]);
    } else if (f < 4) {
      cs = (c[node_at(0, u, 0)] + c[node_at(1, u, 0)]) + (c[node_at(0, u, 1)] + c[node_at(1, u, 1)]);
      es = (C[u] + C[u + 2]) + (C[8 + 2 * u] + C[9 + 2 * u]);
    } else {
      cs = (c[node_at(u, 0, 0)] + c[node_at(u, 1, 0)]) + (c[node_at(u, 0, 1)] + c[node_at(u, 1, 1)]);
      es = (C[4 + u] + C[6 + u]) + (C[8 + u] + C[10 + u]);
    }
    coef = fma(-3.0, cs, es);
  } else if (lane == 26) {
    const double* c = Sm;
    const double* C = Sm + 8;
    double ez0 = (C[0] + C[1]) + (C[4] + C[5]), ez1 = (C[2] + C[3]) + (C[6] + C[7]);
    double cz0 = (c[node_at(0, 0, 0)] + c[node_at(1, 0, 0)]) + (c[node_at(0, 1, 0)] + c[node_at(1, 1, 0)]);
    double cz1 = (c[node_at(0, 0, 1)] + c[node_at(1, 0, 1)]) + (c[node_at(0, 1, 1)] + c[node_at(1, 1, 1)]);
    double esum = (ez0 + ez1) + ((C[8] + C[9]) + (C[10] + C[11]));
    coef = fma(-5.0, cz0 + cz1, esum);
  }
  const int emax = static_cast<int>(m >> 20);
  E = pow2d(min(3 * emax - 3107, 1000));
  return 0;
}

// Tensor position of the coefficient held by class slot `lane` (0-26).
__device__ __forceinline__ int tensor_pos(int lane) {
  if (lane < 8) return corner_t(lane);
  if (lane < 20) return edge_t(lane - 8);
  if (lane < 26) return face_t(lane - 20);
  return tix(1, 1, 1);
}

__device__ __forceinline__ void split5_row(const double* in, int stride_in, double* out,
                                           int stride_out) {
  double p0 = in[0], p1 = in[stride_in], p2 = in[2 * stride_in];
  double s = p0 + p1, t = p1 + p2;
  out[0] = p0;
  out[stride_out] = 0.5 * s;
  out[2 * stride_out] = 0.25 * (s + t);
  out[3 * stride_out] = 0.5 * t;
  out[4 * stride_out] = p2;
}

// Unscaled split of a row (hexval_internal.cuh): entry x carries 2^c(x).
__device__ __forceinline__ void split5u_row(const double* in, int stride_in, double* out,
                                            int stride_out) {
  const double p0 = in[0], p1 = in[stride_in], p2 = in[2 * stride_in];
  const double s = p0 + p1, t = p1 + p2;
  out[0] = p0;
  out[stride_out] = s;
  out[2 * stride_out] = s + t;
  out[3 * stride_out] = t;
  out[4 * stride_out] = p2;
}

// The three unscaled de Casteljau passes of a box whose 27 coefficients are
// in sm[0..27) (tensor order): its 125 split values into sm[147..272),
// indexed (i + 5 (j + 5 k)), value (i, j, k) carrying 2^split_exp3(i, j, k).
// All lanes.
__device__ __forceinline__ void split_box_warp(double* sm) {
  const int lane = threadIdx.x & 31;
  double* A = sm;        // [i + 3 j + 9 k]
  double* P1 = sm + 27;  // [i + 5 (j + 3 k)], i < 5
  double* P2 = sm + 72;  // [i + 5 (j + 5 k)], i, j < 5
  double* G = sm + 147;  // [i + 5 (j + 5 k)], i, j, k < 5
  __syncwarp();
  if (lane < 9) {  // along xi: row (j, k)
    int j = lane % 3, k = lane / 3;
    split5u_row(A + 3 * j + 9 * k, 1, P1 + 5 * (j + 3 * k), 1);
  }
  __syncwarp();
  if (lane < 15) {  // along eta: row (i, k)
    int i = lane % 5, k = lane / 5;
    split5u_row(P1 + i + 15 * k, 5, P2 + i + 25 * k, 5);
  }
  __syncwarp();
  if (lane < 25) {  // along zeta: row (i, j)
    int i = lane % 5, j = lane / 5;
    split5u_row(P2 + i + 5 * j, 25, G + i + 5 * j, 25);
  }
  __syncwarp();
}

// Classification of child `o` (lane o < 8) of a box split by split_box_warp
// against the bound key: the state bits it contributes and whether it must be queued (as
// refine_box in tail.cu).
__device__ __forceinline__ void classify_child_warp(const double* G, uint32_t key, bool last,
                                                    uint32_t& bits, bool& want) {
  const int lane = threadIdx.x & 31;
  bits = 0;
  want = false;
  if (lane >= 8) return;
  const int sx = 2 * (lane & 1), sy = 2 * ((lane >> 1) & 1), sz = 2 * (lane >> 2);
  bool nonpos = false, amb = false, notcert = false, amb2 = false;
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 3; ++i) {
        Sign3 q = sign_d_split(G[(sx + i) + 5 * ((sy + j) + 5 * (sz + k))],
                               key, split_exp3(sx + i, sy + j, sz + k));
        if ((i != 1) && (j != 1) && (k != 1)) {
          nonpos |= q.nonpos;
          amb |= !(q.nonpos | q.pos);
        } else {
          notcert |= q.nonpos;
          amb2 |= !(q.nonpos | q.pos);
        }
      }
  if (nonpos) bits = kStInvalid;
  else if (amb) bits = kStAmbig;
  else if (notcert) { if (last) bits = kStCap; else want = true; }
  else if (amb2) bits = kStAmbig;
}

// In-warp refinement (FP32-filtered form): a few elements a batch need
// subdivision after their FP64 redo; the warp that redid one refines it at
// once, breadth first in a workspace of its own, with the same arithmetic,
// bounds and order-free verdict as the refinement of tail.cu, instead of
// queueing it for the tail kernel.  Returns the flag byte, or -1 when the
// element must go to the tail's refinement after all (no workspace left, a
// level of more than kIwBoxes boxes, or a sign FP64 cannot settle).  `un` =
// this lane's unscaled root coefficient (class slot lane < 27).
static __device__ __noinline__ int refine_in_warp(const Batch& p, double un, double E0, double M0,
                                                  double* sm) {
  const Scratch& S = p.s;
  const int lane = threadIdx.x & 31;
  if (!S.iw || !split_range_ok(M0)) return -1;
  unsigned int slot = 0;
  if (lane == 0) slot = atomicAdd(&S.cnt->iw_count, 1u);
  slot = __shfl_sync(kFull, slot, 0);
  if (slot >= kIwSlots) return -1;
  double* W = S.iw + static_cast<uint64_t>(slot) * 2 * 27 * kIwBoxes;  // [buf][t][box]
  if (lane < 27) W[static_cast<uint64_t>(tensor_pos(lane)) * kIwBoxes] = un;
  __syncwarp();
  unsigned int nb = 1;
  int cur = 0;
  const double* G = sm + 147;
  for (int level = 0; level < p.max_depth; ++level) {
    const int child_level = level + 1;
    const bool last = child_level >= p.max_depth;
    const double E = fma(static_cast<double>(child_level) * 0x1p-49, M0, E0);
    const uint32_t key = dhi(E);
    uint32_t bits = 0;
    unsigned int nn = 0;
    const double* in = W + static_cast<uint64_t>(cur) * 27 * kIwBoxes;
    double* out = W + static_cast<uint64_t>(cur ^ 1) * 27 * kIwBoxes;
    for (unsigned int j = 0; j < nb && !(bits & kStInvalid); ++j) {
      if (lane < 27) sm[lane] = in[static_cast<uint64_t>(lane) * kIwBoxes + j];
      split_box_warp(sm);
      uint32_t cbits;
      bool want;
      classify_child_warp(G, key, last, cbits, want);
      bits |= __reduce_or_sync(kFull, cbits);
      const uint32_t queue = (bits & kStInvalid) ? 0u : (__ballot_sync(kFull, want) & 0xffu);
      for (uint32_t q = queue; q; q &= q - 1) {
        const int o = __ffs(q) - 1;
        if (nn < kIwBoxes) {
          const int sx = 2 * (o & 1), sy = 2 * ((o >> 1) & 1), sz = 2 * (o >> 2);
          if (lane < 27) {
            const int x = sx + lane % 3, y = sy + (lane / 3) % 3, z = sz + lane / 9;
            out[static_cast<uint64_t>(lane) * kIwBoxes + nn] =
                down2(G[x + 5 * (y + 5 * z)], split_exp3(x, y, z));
          }
        } else {
          bits |= kStOverflow;
        }
        ++nn;
      }
      __syncwarp();
    }
    // the verdict rules of finalize_slot, level by level
    if (bits & kStInvalid) return make_flag(kVInvalid, child_level, 0);
    if (bits & (kStAmbig | kStOverflow)) return -1;
    if (nn == 0) return (bits & kStCap) ? make_flag(kVUndecided, p.max_depth, 0)
                                        : make_flag(kVValid, child_level, 0);
    nb = nn;
    cur ^= 1;
  }
  return -1;  // not reached: the last level queues nothing
}

// Warp-cooperative fp64_element (element64.cuh): element e of the batch,
// all 32 lanes, `sm` = this warp's shared scratch.
static __device__ __noinline__ void fp64_element_warp(const Batch& p, uint32_t e, double* sm) {
  const Scratch& S = p.s;
  const int lane = threadIdx.x & 31;
  const int64_t g = p.base + e;
  double smp, coef, E;
  const int rc = warp_root64(p, g, sm, smp, coef, E);
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  if (rc) {
    if (lane == 0) {
      p.flags[g] = make_flag(rc == 1 ? kVUndecided : kVNonfinite, 0, 0);
      if (p.bmin) p.bmin[g] = qnan;
      if (p.bmax) p.bmax[g] = qnan;
      if (rc == 1) set_status(S.status, kSbIndex);
    }
    return;
  }
  // certified classification (element64.cuh: classify_root)
  const uint32_t k1 = dhi(E);
  // sample keys: corners k1, edge samples x4; coefficient keys: edges x2,
  // faces x4, centre x8
  uint32_t skey = lane < 8 ? k1 : k1 + (2u << 20);
  Sign3 qs = sign_d(smp, skey);
  bool s_nonpos = __any_sync(kFull, lane < 20 && qs.nonpos);
  bool s_amb = __any_sync(kFull, lane < 20 && !(qs.nonpos | qs.pos));
  uint32_t ckey = lane < 20 ? k1 + (1u << 20) : (lane < 26 ? k1 + (2u << 20) : k1 + (3u << 20));
  Sign3 qc = sign_d(coef, ckey);
  bool c_notcert = __any_sync(kFull, lane >= 8 && lane < 27 && qc.nonpos);
  bool c_amb = __any_sync(kFull, lane >= 8 && lane < 27 && !(qc.nonpos | qc.pos));
  int outcome = s_nonpos ? 0 : (s_amb ? 3 : (c_notcert ? 2 : (c_amb ? 3 : 1)));
  if (outcome == 2 && p.max_depth == 0) outcome = 6;
  // unscaled coefficient of this lane, min / max over the 27
  double un = lane < 8 ? coef : (lane < 20 ? coef * 0.5 : (lane < 26 ? coef * 0.25 : coef * 0.125));
  long long key = dkey(un);
  long long kmin = lane < 27 ? key : 0x7fffffffffffffffLL;
  long long kmax = lane < 27 ? key : (-0x7fffffffffffffffLL - 1);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(kFull, kmin, d));
    kmax = max(kmax, __shfl_xor_sync(kFull, kmax, d));
  }
  const double lo = dunkey(kmin), hi = dunkey(kmax);
  if (outcome == 2) {
    const int f = refine_in_warp(p, un, E, fmax(fabs(lo), fabs(hi)) + E, sm);
    if (f >= 0) {
      if (lane == 0) {
        atomicAdd(&S.cnt->iw_done, 1u);
        p.flags[g] = static_cast<uint8_t>(f);
        if (p.bmin) p.bmin[g] = lo;
        if (p.bmax) p.bmax[g] = hi;
      }
      return;
    }
  }
  if (outcome == 2) {
    // tensor position of this lane's coefficient
    int t = -1;
    if (lane < 8) t = corner_t(lane);
    else if (lane < 20) t = edge_t(lane - 8);
    else if (lane < 26) t = face_t(lane - 20);
    else if (lane == 26) t = tix(1, 1, 1);
    unsigned int slot = 0;
    if (lane == 0) slot = atomicAdd(&S.cnt->level_count[0], 1u);
    slot = __shfl_sync(kFull, slot, 0);
    if (slot < S.qcap) {
      if (t >= 0) S.qcoef[0][static_cast<uint64_t>(t) * S.qcap + slot] = un;
      if (lane == 0) {
        S.slot_elem[slot] = e;
        S.slot_state[slot] = 0u;
        S.slot_lev[slot] = 0u;
        S.slot_e0[slot] = E;
        S.slot_m0[slot] = fmax(fabs(lo), fabs(hi)) + E;
        S.qslot[0][slot] = slot;
        if (S.qpos[0]) S.qpos[0][slot] = 0ull;
      }
    } else {
      outcome = 3;  // queue full: exact tier
      if (lane == 0) set_status(S.status, kSbQueue);
    }
  }
  if (lane != 0) return;
  if (outcome == 3) {
    unsigned int x = atomicAdd(&S.cnt->exact_count, 1u);
    if (x < S.exact_cap) {
      S.exact_list[x] = e;
    } else {
      p.flags[g] = make_flag(kVUndecided, 0, 0);
      set_status(S.status, kSbQueue);
    }
  } else if (outcome != 2) {
    p.flags[g] = make_flag(outcome == 0 ? kVInvalid : (outcome == 1 ? kVValid : kVUndecided), 0, 0);
  }
  if (p.bmin) p.bmin[g] = lo;
  if (p.bmax) p.bmax[g] = hi;
}

// Warp-cooperative refine_box: box `idx` of level `level`, all 32 lanes.
static __device__ __noinline__ void refine_box_warp(const Batch& p, int level, unsigned int idx,
                                             double* sm) {
  const Scratch& S = p.s;
  const int lane = threadIdx.x & 31;
  const int in = level & 1, out = in ^ 1;
  const int child_level = level + 1;
  const bool last = child_level >= p.max_depth;
  const uint32_t sraw = ldcg(S.qslot[in] + idx);
  if (sraw & kDeadBox) return;  // certified by the exact check
  const uint32_t slot = sraw;
  if (ldcg(S.slot_state + slot) & (kStInvalid | kStAmbig | kStOverflow)) return;
  if (lane == 0) atomicAdd(&S.cnt->split64, 1u);
  const bool xok = S.xb_cap != 0 && S.qpos[in] != nullptr;
  const uint64_t ppos = xok ? ldcg(S.qpos[in] + idx) : 0ull;
  double* A = sm;          // [i + 3 j + 9 k]
  double* P1 = sm + 27;    // [i + 5 (j + 3 k)], i < 5
  double* P2 = sm + 72;    // [i + 5 (j + 5 k)], i, j < 5
  double* G = sm + 147;    // [i + 5 (j + 5 k)], i, j, k < 5
  if (lane < 27) A[lane] = ldcg(S.qcoef[in] + static_cast<uint64_t>(lane) * S.qcap + idx);
  const double m0 = ldcg(S.slot_m0 + slot);
  const double E = fma(static_cast<double>(child_level) * 0x1p-49, m0, ldcg(S.slot_e0 + slot));
  const uint32_t key = dhi(E);
  // unscaled split (hexval_internal.cuh): value (x, y, z) carries 2^split_exp3(x, y, z)
  __syncwarp();
  if (lane < 9) {  // along xi: row (j, k)
    int j = lane % 3, k = lane / 3;
    split5u_row(A + 3 * j + 9 * k, 1, P1 + 5 * (j + 3 * k), 1);
  }
  __syncwarp();
  if (lane < 15) {  // along eta: row (i, k)
    int i = lane % 5, k = lane / 5;
    split5u_row(P1 + i + 15 * k, 5, P2 + i + 25 * k, 5);
  }
  __syncwarp();
  if (lane < 25) {  // along zeta: row (i, j)
    int i = lane % 5, j = lane / 5;
    split5u_row(P2 + i + 5 * j, 25, G + i + 5 * j, 25);
  }
  __syncwarp();
  // lane o < 8 classifies child o
  uint32_t bits = split_range_ok(m0) ? 0u : kStAmbig;  // else the exact tier decides
  bool want = false, xwant = false;
  if (lane < 8 && !bits) {
    const int sx = 2 * (lane & 1), sy = 2 * ((lane >> 1) & 1), sz = 2 * (lane >> 2);
    bool nonpos = false, amb = false, notcert = false, amb2 = false;
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          Sign3 q = sign_d_split(G[(sx + i) + 5 * ((sy + j) + 5 * (sz + k))],
                                 key, split_exp3(sx + i, sy + j, sz + k));
          if ((i != 1) && (j != 1) && (k != 1)) {
            nonpos |= q.nonpos;
            amb |= !(q.nonpos | q.pos);
          } else {
            notcert |= q.nonpos;
            amb2 |= !(q.nonpos | q.pos);
          }
        }
    const bool unsure = !nonpos && (amb || (!notcert && amb2));
    if (nonpos) bits = kStInvalid;
    else if (unsure) {
      if (xok) { xwant = true; want = !last; }  // exact check (refine_box in tail.cu)
      else bits = kStAmbig;
    }
    else if (notcert) { if (last) bits = kStCap; else want = true; }
  }
  bits = __reduce_or_sync(kFull, bits);
  uint32_t queue = __ballot_sync(kFull, want) & 0xffu;
  uint32_t xq = __ballot_sync(kFull, xwant) & 0xffu;
  if (bits & kStInvalid) queue = xq = 0;
  unsigned int base = 0, xbase = 0;
  if (queue) {
    if (lane == 0) base = atomicAdd(&S.cnt->level_count[child_level], __popc(queue));
    base = __shfl_sync(kFull, base, 0);
  }
  if (xq) {
    if (lane == 0) xbase = atomicAdd(&S.cnt->xb_count, __popc(xq));
    xbase = __shfl_sync(kFull, xbase, 0);
  }
  unsigned int pos = base, xpos = xbase;
  for (uint32_t q = queue | xq; q; q &= q - 1) {
    const int o = __ffs(q) - 1;
    const uint64_t cpos = 2ull * ppos + (static_cast<uint64_t>(o & 1) |
                                         (static_cast<uint64_t>((o >> 1) & 1) << 16) |
                                         (static_cast<uint64_t>(o >> 2) << 32));
    uint32_t qi = kNoBox;
    if ((queue >> o) & 1u) {
      if (pos < S.qcap) {
        const int sx = 2 * (o & 1), sy = 2 * ((o >> 1) & 1), sz = 2 * (o >> 2);
        if (lane < 27) {
          const int x = sx + lane % 3, y = sy + (lane / 3) % 3, z = sz + lane / 9;
          S.qcoef[out][static_cast<uint64_t>(lane) * S.qcap + pos] =
              down2(G[x + 5 * (y + 5 * z)], split_exp3(x, y, z));
        }
        if (lane == 0) {
          S.qslot[out][pos] = slot;
          if (xok) S.qpos[out][pos] = cpos;
        }
        qi = pos;
      } else {
        bits |= kStOverflow;
      }
      ++pos;
    }
    if ((xq >> o) & 1u) {
      if (xpos < S.xb_cap) {
        if (lane == 0) {
          S.xb_slot[xpos] = slot;
          S.xb_qi[xpos] = qi;
          S.xb_pos[xpos] = cpos;
        }
      } else {
        bits |= kStAmbig;  // list full: the full exact tier decides the element
      }
      ++xpos;
    }
  }
  if (lane == 0) {
    if (bits) atomicOr(&S.slot_state[slot], bits);
    if (bits & (kStAmbig | kStOverflow)) atomicAdd(&S.cnt->amb_count, 1u);
    if (bits & kStOverflow) set_status(S.status, kSbQueue);
    S.slot_lev[slot] = static_cast<uint32_t>(child_level);
  }
  __syncwarp();
}

}  // namespace hexval
