// Refinement in FP32 (FP32-filtered form): the elements the FP32 pass found
// to need subdivision (all 20 samples certainly positive, a coefficient
// certainly non-positive) are refined breadth first with FP32 boxes, exactly
// as the FP64 refinement of tail.cu (Sec. 6: split at 1/2 along xi, eta,
// zeta by quadratic de Casteljau, computed unscaled as hexval_internal.cuh
// describes and then normalised, split_box32; a child with a corner
// certainly <= 0 makes the element INVALID at that level, a child with all
// 27 certainly > 0 is certified, any other child is queued, or the depth
// cap is reached).
// An element whose boxes meet a sign that the FP32 bound cannot settle, or
// a full queue, is listed in esc2 and redone from scratch in FP64.
//
// Error bound of every coefficient at depth d: E0 + d 2^-20 M0, with E0 the
// FP32 bound of the depth-0 coefficients and M0 >= |every coefficient| (the
// children are convex combinations; one level adds at most 6 roundings of
// size 2^-24 M0).
#pragma once

#include "element32.cuh"

namespace hexval {

// Unscaled split of a row (hexval_internal.cuh): entry x carries 2^c(x).
__device__ __forceinline__ void split5uf(float p0, float p1, float p2, float q[5]) {
  const float s = p0 + p1, t = p1 + p2;
  q[0] = p0;
  q[1] = s;
  q[2] = s + t;
  q[3] = t;
  q[4] = p2;
}

// The three unscaled de Casteljau passes of a box whose 27 coefficients are
// A (tensor order) into G, then every value multiplied by 2^-split_exp3: G
// holds the 125 values of the halving split (the multiplications are exact
// but for a result below the normal range, rounded or flushed by less than
// 2^-126, which the per-level slack covers inside split_range_ok's range).
__device__ __forceinline__ void split_box32(const float A[27], float G[5][5][5]) {
  float P1[5][3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float q[5];
      split5uf(A[tix(0, j, k)], A[tix(1, j, k)], A[tix(2, j, k)], q);
#pragma unroll
      for (int i = 0; i < 5; ++i) P1[i][j][k] = q[i];
    }
  float P2[5][5][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      float q[5];
      split5uf(P1[i][0][k], P1[i][1][k], P1[i][2][k], q);
#pragma unroll
      for (int j = 0; j < 5; ++j) P2[i][j][k] = q[j];
    }
#pragma unroll
  for (int j = 0; j < 5; ++j)
#pragma unroll
    for (int i = 0; i < 5; ++i) split5uf(P2[i][j][0], P2[i][j][1], P2[i][j][2], G[i][j]);
#pragma unroll
  for (int x = 0; x < 5; ++x)
#pragma unroll
    for (int y = 0; y < 5; ++y)
#pragma unroll
      for (int z = 0; z < 5; ++z) {
        const int m = split_exp3(x, y, z);
        if (m) G[x][y][z] *= 1.f / static_cast<float>(1 << m);
      }
}

// Classes of child (sx, sy, sz) of a box split by split_box32 against the
// bound E, from the minimum of its 8 corner coefficients and of its 19
// others: a corner certainly <= 0 (min < -E), a corner whose sign E cannot
// settle (else min <= E), another coefficient certainly <= 0, another
// unsettled -- the sign tests of Sec. 6's child decision, each class
// needing only the smallest value of its set (the last two matter only
// without the one before).
struct Child32 {
  bool nonpos, amb, notcert, amb2;
};
__device__ __forceinline__ Child32 classify_child32(const float G[5][5][5], int sx, int sy,
                                                    int sz, float E) {
  float c[8], o[19];
  int nc = 0, no = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float v = G[sx + i][sy + j][sz + k];
        if ((i != 1) && (j != 1) && (k != 1))
          c[nc++] = v;
        else
          o[no++] = v;
      }
  const float mc = min_of<8>(c), mo = min_of<19>(o);
  return {mc < -E, mc <= E, mo < -E, mo <= E};
}

// The first level of the FP32 refinement of one element, by one thread
// (level1_kernel, HEXVAL_OPT_LEVEL1): its root box (the 27 depth-0
// coefficients s in tensor order, as root32 stores them, M0 = max(|lo|,
// |hi|) + E0 as root32 forms it) is split exactly as refine_box32 splits a
// level-0 box, with the same bound E0 + 2^-20 M0 and the same
// classification of the 8 children.  Returns the flag byte when level 1
// decides the element -- a child corner certainly <= 0 (INVALID@1), all
// children certified (VALID@1), or uncertified children at a depth cap of 1
// (UNDECIDED) -- and -1 when it needs deeper levels or meets a sign FP32
// cannot settle; the element then goes on to the tail's FP32 refinement,
// which reaches the same verdict from the same root box.
__device__ __forceinline__ int refine1_fp32(const Scaled<float>& s, float E0, float lo, float hi,
                                            int max_depth) {
  float A[27];
  store_tensor(s, A);
  const float M0 = fmaxf(fabsf(lo), fabsf(hi)) + E0;
  if (!split_range_ok(M0)) return -1;  // the tail sends it to FP64
  const float E = fmaf(0x1p-20f, M0, E0);
  float G[5][5][5];
  split_box32(A, G);
  bool invalid = false, open = false, capped = false;
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const Child32 q = classify_child32(G, 2 * (o & 1), 2 * ((o >> 1) & 1), 2 * (o >> 2), E);
    const bool nonpos = q.nonpos, amb = q.amb, notcert = q.notcert, amb2 = q.amb2;
    if (nonpos) {
      invalid = true;
    } else if (amb) {
      open = true;  // the FP32 refinement would send the element to FP64
    } else if (notcert) {
      if (max_depth <= 1)
        capped = true;
      else
        open = true;  // a child to queue for level 2
    } else if (amb2) {
      open = true;
    }
  }
  if (invalid) return make_flag(kVInvalid, 1, 0);
  if (open) return -1;
  if (capped) return make_flag(kVUndecided, max_depth, 0);
  return make_flag(kVValid, 1, 0);
}

// The elements the FP32 refinement of the tail works on: the refinement list
// from entry r32_in_pass on, or, after the first-level kernel
// (HEXVAL_OPT_LEVEL1), the list r32b of those it left undecided.
__device__ __forceinline__ const uint32_t* refine_list(const Batch& p) {
  return p.level1 ? p.s.r32b : p.s.r32 + p.r32_in_pass;
}

// Root box of the i-th element of refine_list (slot i, box i of level 0):
// the FP32 coefficients recomputed exactly as the FP32 pass computed them,
// with their bound.  Slots beyond the queue capacity are marked for the FP64
// redo.
__device__ __forceinline__ void root32(const Batch& p, bool act, unsigned int i) {
  if (!act) return;
  const Scratch& S = p.s;
  const uint32_t e = ldcg(refine_list(p) + i);
  V3<float> Y[8];
  float X, E = 0.f, lo = 0.f, hi = 0.f;
  bool bad;
  Scaled<float> s;
  load_element32(p, p.base + e, Y, X, bad);  // in range: checked by the FP32 pass
  const bool ok = p.indexed ? fp32_root<true>(Y, X, bad, s, E) : fp32_root<false>(Y, X, bad, s, E);
  if (ok) fp32_classify(s, E, lo, hi);
  const bool fits = i < S.q32cap;
  if (fits) {
    float A[27];
    store_tensor(s, A);
#pragma unroll
    for (int t = 0; t < 27; ++t) S.q32coef[0][static_cast<uint64_t>(t) * S.q32cap + i] = A[t];
    S.q32slot[0][i] = i;
  }
  S.s32_elem[i] = e;
  // (ok is always true: the pass formed the same bound)
  S.s32_state[i] = !fits ? kStOverflow : (ok ? 0u : kStAmbig);
  S.s32_lev[i] = 0u;
  S.s32_e0[i] = E;
  S.s32_m0[i] = fmaxf(fabsf(lo), fabsf(hi)) + E;
}

// One FP32 box of level `level` (act = false: idle lane).  Called by all lanes.
__device__ __forceinline__ void refine_box32(const Batch& p, int level, bool act,
                                             unsigned int idx) {
  const Scratch& S = p.s;
  const int in = level & 1, out = in ^ 1;
  const int child_level = level + 1;
  const bool last = child_level >= p.max_depth;
  const uint32_t slot = act ? ldcg(S.q32slot[in] + idx) : 0u;
  if (act) act = !(ldcg(S.s32_state + slot) & (kStInvalid | kStAmbig | kStOverflow));
  {  // boxes split, one atomic per warp
    const unsigned int m = __ballot_sync(0xffffffffu, act);
    if (m && (threadIdx.x & 31u) == static_cast<unsigned int>(__ffs(m) - 1))
      atomicAdd(&S.cnt->split32, static_cast<unsigned int>(__popc(m)));
  }
  float G[5][5][5];  // the 125 values of the split (split_box32)
  float E = 0.f;
  uint32_t bits = 0;
  if (act) {
    const float* qc = S.q32coef[in];
    float A[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) A[t] = ldcg(qc + static_cast<uint64_t>(t) * S.q32cap + idx);
    const float m0 = ldcg(S.s32_m0 + slot);
    E = fmaf(static_cast<float>(child_level) * 0x1p-20f, m0, ldcg(S.s32_e0 + slot));
    if (!split_range_ok(m0)) bits = kStAmbig;  // redone in FP64
    split_box32(A, G);
  }
  uint32_t queue = 0;
  if (act && !bits) {
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const Child32 q = classify_child32(G, 2 * (o & 1), 2 * ((o >> 1) & 1), 2 * (o >> 2), E);
      const bool nonpos = q.nonpos, amb = q.amb, notcert = q.notcert, amb2 = q.amb2;
      if (nonpos) {
        bits |= kStInvalid;
      } else if (amb) {
        bits |= kStAmbig;
      } else if (notcert) {
        if (last)
          bits |= kStCap;
        else
          queue |= 1u << o;
      } else if (amb2) {
        bits |= kStAmbig;
      }
    }
    if (bits & kStInvalid) queue = 0;  // the element is decided on this level
  }
  // one atomic per warp for all the children the warp queues
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned int cnt = __popc(queue);
  unsigned int incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= static_cast<unsigned int>(d)) incl += v;
  }
  const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned int pos = 0;
  if (total) {
    if (lane == 31) pos = atomicAdd(&S.cnt->level32_count[child_level], total);
    pos = __shfl_sync(0xffffffffu, pos, 31) + incl - cnt;
  }
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    if ((queue >> o) & 1u) {
      if (pos < S.q32cap) {
        const int sx = 2 * (o & 1), sy = 2 * ((o >> 1) & 1), sz = 2 * (o >> 2);
        float* dst = S.q32coef[out];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
              dst[static_cast<uint64_t>(tix(i, j, k)) * S.q32cap + pos] = G[sx + i][sy + j][sz + k];
        S.q32slot[out][pos] = slot;
      } else {
        bits |= kStOverflow;
      }
      ++pos;
    }
  }
  if (act) {
    if (bits) atomicOr(&S.s32_state[slot], bits);
    S.s32_lev[slot] = static_cast<uint32_t>(child_level);
  }
}

// Verdict of FP32-refined element `s`, or its listing for the FP64 redo.
// Called by all lanes.
__device__ __forceinline__ void finalize32(const Batch& p, bool act, unsigned int s) {
  const Scratch& S = p.s;
  const uint32_t st = act ? ldcg(S.s32_state + s) : 0u;
  const uint32_t lev = act ? ldcg(S.s32_lev + s) : 0u;
  const uint32_t e = act ? ldcg(S.s32_elem + s) : 0u;
  const bool redo = act && !(st & kStInvalid) && (st & (kStAmbig | kStOverflow));
  const unsigned int pos = warp_append(&S.cnt->esc2_count, redo);
  if (!act) return;
  if (redo) {
    S.esc2[pos] = e;  // capacity = batch size
    return;
  }
  uint8_t flag;
  if (st & kStInvalid)
    flag = make_flag(kVInvalid, lev, 0);
  else if (st & kStCap)
    flag = make_flag(kVUndecided, p.max_depth, 0);
  else
    flag = make_flag(kVValid, lev, 0);
  p.flags[p.base + e] = flag;
}

}  // namespace hexval
