// Everything after the bulk pass, in one persistent cooperative launch:
//  phase R  (FP32 form) refinement in FP32 of the elements the FP32 pass
//           listed (refine32.cuh); elements whose signs FP32 cannot settle
//           are listed for the FP64 redo;
//  phase E  (FP32 form) the escalated elements the FP32 pass (or the
//           double-float or the partial FP64 redo) left, and those of
//           phase R, redone in FP64 (element64.cuh);
//  phase X0 elements whose root signs could not be certified: decided
//           exactly at depth 0, or refined from their FP64 root box;
//  levels   refinement of undecided elements (Sec. 6, recursive_subdivision),
//           breadth first, one level per grid-wide step, each followed by
//           phase XB, the exact check of the boxes an uncertain sign left
//           open (exact_warp.cuh);
//  phase F  verdicts of the refined elements;
//  phase X  the full exact tier (exact.cuh) for what is left (coordinates
//           outside the fast exact range, a full queue or list), only when
//           some element needs it.
// Grid-wide steps are separated by a bounded grid barrier (tail_barrier; a
// block whose wait runs out stops its work and only joins the final fold).
// Every count that decides a branch is read after a barrier (or was written
// by an earlier launch), so all blocks take the same branches; with nothing
// to do the kernel returns at its first instructions.  The last block to
// finish folds the batch counters into the statistics and resets them.
//
// Refinement.  Level d holds boxes of depth d whose corners are certainly
// positive and which are certainly not certified.  Each is split at 1/2
// along xi, eta and zeta (quadratic de Casteljau: a row (p0, p1, p2) becomes
// (p0, (p0+p1)/2, (p0+2p1+p2)/4, (p1+p2)/2, p2), computed unscaled with its
// power-of-two factors kept apart as hexval_internal.cuh describes; the left
// child keeps the first three, the right child the last three) and its 8
// children of depth d+1 are classified:
//   a corner coefficient certainly <= 0          -> element INVALID at d+1
//   all 27 certainly > 0                         -> child certified
//   corners certainly > 0, another certainly <=0 -> child queued for d+2
//                                                   (or the cap is hit)
//   a sign that the error bound cannot settle    -> exact check of the box
//                                                   after the level.
// INVALID found on a level wins over anything else found on that level, which
// gives the order-independent verdict (shallowest level with a non-positive
// corner) whatever the order in which boxes are processed.
//
// Error bound of every coefficient at depth d: E0 + d 2^-49 M0, E0 bounding
// the depth-0 coefficients and M0 >= |every coefficient| (children are convex
// combinations; one level adds at most 6 roundings of size u M0).
#include "element64.cuh"
#include "exact.cuh"
#include "exact_warp.cuh"
#include "refine32.cuh"
#include "warp_items.cuh"

namespace hexval {

namespace {

constexpr int kTailThreads = 128;

// Inlining of the per-item routines into the persistent kernel.
#ifndef HEXVAL_TAIL_INLINE
#define HEXVAL_TAIL_INLINE __forceinline__
#endif

// Unscaled split of a row (hexval_internal.cuh): entry x carries 2^c(x).
__device__ __forceinline__ void split5u(double p0, double p1, double p2, double q[5]) {
  const double s = p0 + p1, t = p1 + p2;
  q[0] = p0;
  q[1] = s;
  q[2] = s + t;
  q[3] = t;
  q[4] = p2;
}

// One box of level `level` (act = false: idle lane).  Called by all lanes.
__device__ HEXVAL_TAIL_INLINE void refine_box(const Batch& p, int level, bool act, unsigned int idx) {
  const Scratch& S = p.s;
  const int in = level & 1, out = in ^ 1;
  const int child_level = level + 1;
  const bool last = child_level >= p.max_depth;
  uint32_t slot = act ? ldcg(S.qslot[in] + idx) : 0u;
  if (slot & kDeadBox) act = false;  // certified by the exact check
  slot &= ~kDeadBox;
  if (act) act = !(ldcg(S.slot_state + slot) & (kStInvalid | kStAmbig | kStOverflow));
  {  // boxes split, one atomic per warp
    const unsigned int m = __ballot_sync(0xffffffffu, act);
    if (m && (threadIdx.x & 31u) == static_cast<unsigned int>(__ffs(m) - 1))
      atomicAdd(&S.cnt->split64, static_cast<unsigned int>(__popc(m)));
  }
  // exact check of uncertain children possible (box positions kept)
  const bool xok = S.xb_cap != 0 && S.qpos[in] != nullptr;
  const uint64_t ppos = (act && xok) ? ldcg(S.qpos[in] + idx) : 0ull;
  double G[5][5][5];  // unscaled: entry (x, y, z) carries 2^split_exp3(x, y, z)
  uint32_t key = 0;
  uint32_t bits = 0;  // element state bits found by this box
  if (act) {
    const double* qc = S.qcoef[in];
    double A[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) A[t] = ldcg(qc + static_cast<uint64_t>(t) * S.qcap + idx);
    const double m0 = ldcg(S.slot_m0 + slot);
    double E = fma(static_cast<double>(child_level) * 0x1p-49, m0, ldcg(S.slot_e0 + slot));
    key = dhi(E);
    if (!split_range_ok(m0)) bits = kStAmbig;  // the exact tier decides it
    double P1[5][3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double q[5];
        split5u(A[tix(0, j, k)], A[tix(1, j, k)], A[tix(2, j, k)], q);
#pragma unroll
        for (int i = 0; i < 5; ++i) P1[i][j][k] = q[i];
      }
    double P2[5][5][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        double q[5];
        split5u(P1[i][0][k], P1[i][1][k], P1[i][2][k], q);
#pragma unroll
        for (int j = 0; j < 5; ++j) P2[i][j][k] = q[j];
      }
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
      for (int i = 0; i < 5; ++i) split5u(P2[i][j][0], P2[i][j][1], P2[i][j][2], G[i][j]);
  }
  uint32_t queue = 0;  // children to queue
  uint32_t xq = 0;     // children whose class an uncertain sign decides: exact check
  if (act && !bits) {
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int sx = 2 * (o & 1), sy = 2 * ((o >> 1) & 1), sz = 2 * (o >> 2);
      bool nonpos = false, amb = false, notcert = false, amb2 = false;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            Sign3 q = sign_d_split(G[sx + i][sy + j][sz + k],
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
      if (nonpos) {
        bits |= kStInvalid;
      } else if (unsure) {
        if (xok) {  // queued as if not certified; the exact check may drop it
          xq |= 1u << o;
          if (!last) queue |= 1u << o;
        } else {
          bits |= kStAmbig;
        }
      } else if (notcert) {
        if (last)
          bits |= kStCap;
        else
          queue |= 1u << o;
      }
    }
    if (bits & kStInvalid) queue = xq = 0;  // the element is decided on this level
  }
  // one atomic per warp for all the children the warp queues
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned int cnt = __popc(queue);
  unsigned int incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    unsigned int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= static_cast<unsigned int>(d)) incl += v;
  }
  const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned int pos = 0;
  if (total) {
    if (lane == 31) pos = atomicAdd(&S.cnt->level_count[child_level], total);
    pos = __shfl_sync(0xffffffffu, pos, 31) + incl - cnt;
  }
  unsigned int xpos = 0;
  if (__any_sync(0xffffffffu, xq != 0u)) {  // rare
    const unsigned int xc = __popc(xq);
    unsigned int xincl = xc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      unsigned int v = __shfl_up_sync(0xffffffffu, xincl, d);
      if (lane >= static_cast<unsigned int>(d)) xincl += v;
    }
    const unsigned int xtotal = __shfl_sync(0xffffffffu, xincl, 31);
    if (lane == 31) xpos = atomicAdd(&S.cnt->xb_count, xtotal);
    xpos = __shfl_sync(0xffffffffu, xpos, 31) + xincl - xc;
  }
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const uint64_t cpos = 2ull * ppos + (static_cast<uint64_t>(o & 1) |
                                         (static_cast<uint64_t>((o >> 1) & 1) << 16) |
                                         (static_cast<uint64_t>(o >> 2) << 32));
    uint32_t qi = kNoBox;
    if ((queue >> o) & 1u) {
      if (pos < S.qcap) {
        const int sx = 2 * (o & 1), sy = 2 * ((o >> 1) & 1), sz = 2 * (o >> 2);
        double* dst = S.qcoef[out];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
              dst[static_cast<uint64_t>(tix(i, j, k)) * S.qcap + pos] =
                  down2(G[sx + i][sy + j][sz + k], split_exp3(sx + i, sy + j, sz + k));
        S.qslot[out][pos] = slot;
        if (xok) S.qpos[out][pos] = cpos;
        qi = pos;
      } else {
        bits |= kStOverflow;
      }
      ++pos;
    }
    if ((xq >> o) & 1u) {
      if (xpos < S.xb_cap) {
        S.xb_slot[xpos] = slot;
        S.xb_qi[xpos] = qi;
        S.xb_pos[xpos] = cpos;
      } else {
        bits |= kStAmbig;  // list full: the full exact tier decides the element
      }
      ++xpos;
    }
  }
  if (act) {
    if (bits) atomicOr(&S.slot_state[slot], bits);
    if (bits & (kStAmbig | kStOverflow)) atomicAdd(&S.cnt->amb_count, 1u);
    if (bits & kStOverflow) set_status(S.status, kSbQueue);
    S.slot_lev[slot] = static_cast<uint32_t>(child_level);
  }
}

// Verdict of refined element `s`; elements that need the exact tier are
// appended to its list.  Called by all lanes.
__device__ HEXVAL_TAIL_INLINE void finalize_slot(const Batch& p, bool act, unsigned int s) {
  const Scratch& S = p.s;
  uint32_t st = act ? ldcg(S.slot_state + s) : 0u;
  uint32_t lev = act ? ldcg(S.slot_lev + s) : 0u;
  uint32_t e = act ? ldcg(S.slot_elem + s) : 0u;
  bool to_exact = act && !(st & kStInvalid) && (st & (kStAmbig | kStOverflow));
  unsigned int pos = warp_append(&S.cnt->exact_count, to_exact);
  if (!act) return;
  uint8_t flag;
  const int xu = (st & kStXUsed) ? 1 : 0;  // a box sign settled exactly
  if (st & kStInvalid) {
    flag = make_flag(kVInvalid, lev, xu);
  } else if (to_exact) {
    if (pos < S.exact_cap) {
      S.exact_list[pos] = e;
      return;
    }
    set_status(S.status, kSbQueue);
    flag = make_flag(kVUndecided, p.max_depth, 0);
  } else if (st & kStCap) {
    flag = make_flag(kVUndecided, p.max_depth, xu);
  } else {
    flag = make_flag(kVValid, lev, xu);
  }
  p.flags[p.base + e] = flag;
}

// Exact check of entry i of the exact-check list (a child of depth `level`
// whose class an uncertain sign decides; exact_warp.cuh): a corner <= 0
// makes the element INVALID on this level; all 27 > 0 certify the box, whose
// queue entry is then marked dead; otherwise the box stays queued, or hits
// the cap on the last level.  Coordinates outside the fast exact range send
// the element to the full exact tier.  All 32 lanes call it.
__device__ __forceinline__ void exact_check_box(const Batch& p, int level, unsigned int i,
                                                double* sm) {
  const Scratch& S = p.s;
  const uint32_t slot = ldcg(S.xb_slot + i);
  if (ldcg(S.slot_state + slot) & (kStInvalid | kStAmbig | kStOverflow)) return;
  const uint32_t qi = ldcg(S.xb_qi + i);
  const int r = exact_tier::exact_box_warp(p, ldcg(S.slot_elem + slot), level,
                                           ldcg(S.xb_pos + i), reinterpret_cast<uint32_t*>(sm));
  if ((threadIdx.x & 31) == 0) {
    if (r < 0) {
      atomicOr(&S.slot_state[slot], kStAmbig);
      atomicAdd(&S.cnt->amb_count, 1u);
    } else {
      uint32_t bits = kStXUsed;
      if (r == 0) bits |= kStInvalid;
      if (r == 2 && qi == kNoBox) bits |= kStCap;
      atomicOr(&S.slot_state[slot], bits);
      if (r == 1 && qi != kNoBox) S.qslot[level & 1][qi] = slot | kDeadBox;
    }
  }
  __syncwarp();
}

// Element of exact-list entry i whose root an uncertain sign left open
// (listed by the depth-0 passes), before the refinement levels: decided
// exactly at depth 0 when it can be; when it needs subdivision (every sample
// > 0, a coefficient <= 0, both exactly) its FP64 root box enters level 0 of
// the refinement like any other, with the exact box check for later
// uncertain signs.  Entries handled here are replaced by kNoBox; the others
// (coordinates outside the fast exact range, a full queue) stay for the full
// tier.  All 32 lanes call it.
__device__ __forceinline__ void exact_root_entry(const Batch& p, unsigned int i, double* sm) {
  const Scratch& S = p.s;
  const int lane = threadIdx.x & 31;
  const uint32_t e = ldcg(S.exact_list + i);
  const int64_t g = p.base + e;
  const int f = exact_tier::exact_depth0_warp(p, e, reinterpret_cast<uint32_t*>(sm));
  if (f == -2) return;
  if (f >= 0 || p.max_depth == 0) {
    if (lane == 0) {
      p.flags[g] = f >= 0 ? static_cast<uint8_t>(f | 0x80) : make_flag(kVUndecided, 0, 1);
      S.exact_list[i] = kNoBox;
    }
    __syncwarp();
    return;
  }
  double smp, coef, E;
  if (warp_root64(p, g, sm, smp, coef, E)) return;
  const double un =
      lane < 8 ? coef : (lane < 20 ? coef * 0.5 : (lane < 26 ? coef * 0.25 : coef * 0.125));
  long long kmin = lane < 27 ? dkey(un) : 0x7fffffffffffffffLL;
  long long kmax = lane < 27 ? dkey(un) : (-0x7fffffffffffffffLL - 1);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(kFull, kmin, d));
    kmax = max(kmax, __shfl_xor_sync(kFull, kmax, d));
  }
  const double M0 = fmax(fabs(dunkey(kmin)), fabs(dunkey(kmax))) + E;
  unsigned int slot = 0;
  if (lane == 0) slot = atomicAdd(&S.cnt->level_count[0], 1u);
  slot = __shfl_sync(kFull, slot, 0);
  if (slot >= S.qcap) return;  // queue full: the full tier decides it
  int t = -1;
  if (lane < 8) t = corner_t(lane);
  else if (lane < 20) t = edge_t(lane - 8);
  else if (lane < 26) t = face_t(lane - 20);
  else if (lane == 26) t = tix(1, 1, 1);
  if (t >= 0) S.qcoef[0][static_cast<uint64_t>(t) * S.qcap + slot] = un;
  if (lane == 0) {
    S.slot_elem[slot] = e;
    S.slot_state[slot] = kStXUsed;
    S.slot_lev[slot] = 0u;
    S.slot_e0[slot] = E;
    S.slot_m0[slot] = M0;
    S.qslot[0][slot] = slot;
    S.qpos[0][slot] = 0ull;
    S.exact_list[i] = kNoBox;
  }
  __syncwarp();
}

// Work items of a grid-wide step are dealt to warps round robin over the
// blocks first, so that a short list is spread over all SMs (each warp takes
// 32 consecutive items; the trip count is uniform within a warp).
#define FOR_EACH_ITEM(n, i, act)                                                     \
  for (unsigned int w_ = blockIdx.x + gridDim.x * (threadIdx.x >> 5), i = 0, act = 0; \
       w_ * 32u < (n); w_ += gridDim.x * (blockDim.x >> 5))                           \
    if ((i = w_ * 32u + (threadIdx.x & 31u)), (act = i < (n)), true)

__device__ HEXVAL_TAIL_INLINE void fp64_item(const Batch& p, bool act, uint32_t e) {
  fp64_element(p, act, e);
}

// Steps with at most Batch::warp_items items per warp use the
// warp-cooperative routines (latency), larger ones one item per thread
// (throughput).

// Items dealt to warps one at a time, round robin over the blocks first.
#define FOR_EACH_WARP_ITEM(n, i)                                                    \
  for (unsigned int i = blockIdx.x + gridDim.x * (threadIdx.x >> 5); i < (n);      \
       i += gridDim.x * (blockDim.x >> 5))

// Grid-wide barrier of the tail kernel (a cooperative launch: all blocks
// co-resident) with a bounded wait: after `limit` polls of the arrival
// counter (each an L2 round trip) the block records kSbTimeout and the
// barrier returns false, after which the block does no further work of the
// batch and only takes part in the end-of-kernel counter fold, so that no
// block ever reads data another block may not have written.  Blocks waiting
// at a later barrier then give up the same way.
__device__ __forceinline__ bool tail_barrier(unsigned int* arrive, unsigned int& epoch,
                                             uint32_t* status, long long limit) {
  __shared__ int timed_out;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(arrive, 1u);
    const unsigned int target = epoch * gridDim.x;
    long long spins = 0;
    int to = 0;
    while (ld_acquire(arrive) < target) {
      if (++spins > limit) {
        atomicOr(status, kSbTimeout);
        to = 1;
        break;
      }
    }
    timed_out = to;
    __threadfence();
  }
  __syncthreads();
  return timed_out == 0;
}

// Folds the batch counters into the statistics and resets them: all threads
// of one block, once every block of the batch's last kernel is done with the
// counters.  Warp 0 reads them (the per-level counts one per lane), then the
// block zeroes them together.
__device__ __forceinline__ void fold_stats_and_reset(const Batch& p, unsigned int nx,
                                                     unsigned int n_redo) {
  const Scratch& S = p.s;
  Counters* C = S.cnt;
  Stats* st = S.stats;
  const unsigned int t = threadIdx.x;
  if (t < 32) {
    unsigned long long c = 0, c32 = 0;
    if (t >= 1 && t <= kMaxDepth + 1) {
      c = ldcg(&C->level_count[t]);
      c32 = ldcg(&C->level32_count[t]);
    }
    unsigned long long mx = c > c32 ? c : c32;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, d);
      mx = o > mx ? o : mx;
    }
    if (t == 0) {
      const unsigned int nr = ldcg(&C->r32_count);
      const unsigned int nr_here = nr < p.r32_in_pass ? nr : p.r32_in_pass;
      atomicAdd(&st->elements, static_cast<unsigned long long>(p.n));
      atomicAdd(&st->escalated_fp64, static_cast<unsigned long long>(ldcg(&C->esc_count)) +
                                         ldcg(&C->esc2_count) + nr_here);
      const unsigned int n1 = ldcg(&C->l1_count);
      atomicAdd(&st->refined, static_cast<unsigned long long>(ldcg(&C->level_count[0])) +
                                  (nr - nr_here) + ldcg(&C->iw_done));
      // boxes actually split (root boxes included; a box whose element was
      // settled on an earlier level is skipped and not counted), and the
      // root boxes the first-level kernel split
      const unsigned long long s32 = static_cast<unsigned long long>(ldcg(&C->split32)) + n1;
      atomicAdd(&st->boxes, static_cast<unsigned long long>(ldcg(&C->split64)) + s32);
      atomicAdd(&st->boxes_fp32, s32);
      atomicAdd(&st->exact, static_cast<unsigned long long>(nx));
      atomicAdd(&st->escalated_df, static_cast<unsigned long long>(ldcg(&C->df_count)));
      atomicMax(&st->max_level_boxes, mx);
      atomicAdd(&st->redone_tail, static_cast<unsigned long long>(n_redo));
      atomicAdd(&st->partial_fp64, static_cast<unsigned long long>(ldcg(&C->part_count)));
    }
  }
  __syncthreads();  // every read above is done before the reset
  unsigned int* w = reinterpret_cast<unsigned int*>(C);
  for (unsigned int k = t; k < sizeof(Counters) / sizeof(unsigned int); k += blockDim.x) w[k] = 0u;
  __threadfence();
}

__global__ void __launch_bounds__(kTailThreads, 1) tail_kernel(Batch p, int from_list,
                                                             long long spin_limit) {
  pdl_wait();
  const Scratch& S = p.s;
  Counters* C = S.cnt;
  // escalation list entries [esc_in_pass, n_list) are left for this kernel,
  // or, after the double-float or the partial FP64 redo, the esc3 list it
  // leaves
  const unsigned int n_list = from_list ? ldcg(&C->esc_count) : 0u;
  const unsigned int n_esc = !from_list ? 0u
                             : p.dfredo || p.partial64
                                 ? ldcg(&C->esc3_count)
                                 : (n_list > p.esc_in_pass ? n_list - p.esc_in_pass : 0u);
  // refinement list entries [r32_in_pass, n_rl) are left for this kernel,
  // or, after the first-level kernel, the r32b list it leaves
  const unsigned int n_rl = from_list ? ldcg(&C->r32_count) : 0u;
  const unsigned int n_r = !from_list ? 0u
                           : p.level1 ? ldcg(&C->r32b_count)
                                      : (n_rl > p.r32_in_pass ? n_rl - p.r32_in_pass : 0u);
  if (n_esc == 0 && n_r == 0 && ldcg(&C->level_count[0]) == 0 && ldcg(&C->exact_count) == 0) {
    // nothing left: every block reads only counters that are, or become,
    // zero here, so block 0 may end the batch at once
    if (blockIdx.x == 0) fold_stats_and_reset(p, 0u, 0u);
    return;
  }
  __shared__ double wsm[kTailThreads / 32][kWarpScratch];
  static_assert(exact_tier::kFastWords <= 2 * kWarpScratch, "warp scratch too small");
  static_assert(27 * exact_tier::kBoxWords <= 2 * kWarpScratch, "warp scratch too small");
  double* mysm = wsm[threadIdx.x >> 5];
  const unsigned int warp_items = p.warp_items * gridDim.x * (blockDim.x >> 5);
  unsigned int epoch = 0;
  unsigned int n_esc2 = 0;
  unsigned int n_redo = 0;  // elements of phase E
  // false once a grid barrier timed out: the block then skips to the end
  bool go = true;
  auto sync = [&]() {
    go = go && tail_barrier(&C->arrive, epoch, S.status, spin_limit);
    return go;
  };
  if (n_r) {  // phase R: refinement in FP32 of the elements listed by the FP32 pass
    FOR_EACH_ITEM(n_r, i, act) root32(p, act, i);
    sync();
    for (int level = 0; go && level < p.max_depth; ++level) {
      const unsigned int n = min(level == 0 ? n_r : ldcg(&C->level32_count[level]),
                                 static_cast<unsigned int>(S.q32cap));
      if (n == 0) break;
      FOR_EACH_ITEM(n, i, act) refine_box32(p, level, act, i);
      sync();
    }
    if (go) {
      FOR_EACH_ITEM(n_r, i, act) finalize32(p, act, i);
      sync();
    }
    if (go) n_esc2 = ldcg(&C->esc2_count);
  }
  if (go && n_esc + n_esc2) {  // phase E: list entries, then the FP32 refinement's
    const uint32_t* esc = p.dfredo || p.partial64 ? S.esc3 : S.esc + p.esc_in_pass;
    const unsigned int n_e = n_esc + n_esc2;
    n_redo = n_e;
    if (n_e <= warp_items) {
      FOR_EACH_WARP_ITEM(n_e, i)
        fp64_element_warp(p, i < n_esc ? ldcg(esc + i) : ldcg(S.esc2 + (i - n_esc)), mysm);
    } else {
      FOR_EACH_ITEM(n_e, i, act)
        fp64_item(p, act, act ? (i < n_esc ? ldcg(esc + i) : ldcg(S.esc2 + (i - n_esc))) : 0u);
    }
    sync();
  }
  // phase X0: elements listed for the exact tier by the depth-0 passes
  const unsigned int nx0 = min(ldcg(&C->exact_count), static_cast<unsigned int>(S.exact_cap));
  if (go && nx0 && S.xb_cap && S.qpos[0]) {
    FOR_EACH_WARP_ITEM(nx0, i) exact_root_entry(p, i, mysm);
    sync();
  }
  const unsigned int n0 =
      go ? min(ldcg(&C->level_count[0]), static_cast<unsigned int>(S.qcap)) : 0u;
  unsigned int xb_done = 0;  // exact-check entries settled so far
  for (int level = 0; go && n0 && level < p.max_depth; ++level) {
    const unsigned int n = min(ldcg(&C->level_count[level]),
                               static_cast<unsigned int>(S.qcap));
    if (n == 0) break;
    if (n <= warp_items) {
      FOR_EACH_WARP_ITEM(n, i) refine_box_warp(p, level, i, mysm);
    } else {
      FOR_EACH_ITEM(n, i, act) refine_box(p, level, act, i);
    }
    if (!sync()) break;
    // exact check of the children of this level that an uncertain sign left open
    const unsigned int nxb = min(ldcg(&C->xb_count), static_cast<unsigned int>(S.xb_cap));
    if (nxb > xb_done) {
      FOR_EACH_WARP_ITEM(nxb - xb_done, i) exact_check_box(p, level + 1, xb_done + i, mysm);
      xb_done = nxb;
      sync();
    }
  }
  // Elements for the exact tier: those already listed, and those whose boxes
  // met an uncertain sign or a full queue (listed by phase F below).
  const bool exact = go && (ldcg(&C->exact_count) != 0u || ldcg(&C->amb_count) != 0u);
  if (go && n0) {  // phase F
    FOR_EACH_ITEM(n0, i, act) finalize_slot(p, act, i);
    if (exact) sync();
  }
  unsigned int nx = 0;
  if (go && exact) {
    // phase X: the first kWorkers warps, one element at a time each; depth-0
    // decisions by the whole warp, anything deeper by lane 0 (full tier)
    nx = min(ldcg(&C->exact_count), static_cast<unsigned int>(S.exact_cap));
    const unsigned int nwarps = gridDim.x * (blockDim.x >> 5);
    uint32_t* esm = reinterpret_cast<uint32_t*>(mysm);
    for (unsigned int w = blockIdx.x + gridDim.x * (threadIdx.x >> 5); w < exact_tier::kWorkers;
         w += nwarps)
      for (unsigned int i = w; i < nx; i += exact_tier::kWorkers) {
        const uint32_t e = ldcg(S.exact_list + i);
        if (e == kNoBox) continue;  // settled in phase X0
        const int flag = exact_tier::exact_depth0_warp(p, e, esm);
        if ((threadIdx.x & 31u) == 0u) {
          if (flag >= 0)
            p.flags[p.base + e] = static_cast<uint8_t>(flag | 0x80);
          else
            exact_tier::exact_element(p, e, w);
        }
        __syncwarp();
      }
  }
  // the last block ends the batch
  __shared__ int last_block;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last_block = atomicAdd(&C->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last_block) {
    __threadfence();
    fold_stats_and_reset(p, nx, n_redo);
  }
}

int tail_blocks() {
  static int blocks = 0;
  if (!blocks) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tail_kernel, kTailThreads, 0);
    blocks = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }
  return blocks;
}

}  // namespace

uint64_t exact_work_words() {
  return static_cast<uint64_t>(exact_tier::kInts) * exact_tier::kLimbsMax * exact_tier::kWorkers;
}

// Cooperative (all blocks resident: the grid barrier) and, where the CUDA driver
// accepts it, programmatic (it may become resident while the bulk pass
// finishes; tail_kernel starts with pdl_wait).  spin_limit = polls of the
// grid barrier before it gives up (kSpinLimit by default).
cudaError_t launch_tail(const Batch& p, bool from_list, long long spin_limit, cudaStream_t st) {
  Batch arg = p;
  int fl = from_list ? 1 : 0;
  long long lim = spin_limit > 0 ? spin_limit : kSpinLimit;
  static int pdl_ok = 1;
  if (pdl_ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tail_blocks());
    cfg.blockDim = dim3(kTailThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    if (cudaLaunchKernelEx(&cfg, tail_kernel, arg, fl, lim) == cudaSuccess) return cudaSuccess;
    cudaGetLastError();
    pdl_ok = 0;  // not accepted: plain cooperative launches from now on
  }
  void* args[] = {&arg, &fl, &lim};
  return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(tail_kernel), dim3(tail_blocks()),
                                     dim3(kTailThreads), args, 0, st);
}

cudaError_t launch_tail(const Batch& p, bool from_list, cudaStream_t st) {
  return launch_tail(p, from_list, kSpinLimit, st);
}

}  // namespace hexval
