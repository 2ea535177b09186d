// Refinement of undecided elements (Sec. 6, recursive_subdivision), breadth
// first, one level per launch.
//
// Level d holds the boxes of depth d whose corners are certainly positive and
// which are certainly not certified.  refine_kernel pops each box, splits its
// 27 coefficients at 1/2 along xi, eta and zeta (quadratic de Casteljau: a
// row (p0, p1, p2) becomes (p0, (p0+p1)/2, (p0+2p1+p2)/4, (p1+p2)/2, p2), the
// left child keeps the first three, the right child the last three) and
// classifies the 8 children of depth d+1:
//   a corner coefficient certainly <= 0          -> element INVALID at d+1
//   all 27 certainly > 0                         -> child certified
//   corners certainly > 0, another certainly <=0 -> child queued for d+2
//                                                   (or the cap is hit)
//   a sign that the error bound cannot settle    -> element goes exact.
// Per element, INVALID found on a level wins over anything else found on the
// same level, which gives the order-independent verdict (shallowest level
// with a non-positive corner) whatever the order the boxes are processed in.
//
// Error bound of every coefficient at depth d: E0 + d * 2^-49 * M0 where E0
// bounds the depth-0 coefficients and M0 >= |every coefficient| (children are
// convex combinations; one level adds at most 6 roundings of size u M0).
#include "hexval_internal.cuh"

namespace hexval {

namespace {

constexpr int kRefineThreads = 128;
constexpr int kFinalizeThreads = 256;

__device__ __forceinline__ void split5(double p0, double p1, double p2, double q[5]) {
  double s = p0 + p1, t = p1 + p2;
  q[0] = p0;
  q[1] = 0.5 * s;
  q[2] = 0.25 * (s + t);
  q[3] = 0.5 * t;
  q[4] = p2;
}

__global__ void __launch_bounds__(kRefineThreads) refine_kernel(Batch p, int level) {
  const Scratch& S = p.s;
  const unsigned int n_in = min(S.cnt->level_count[level], static_cast<unsigned int>(S.qcap));
  const int in = level & 1, out = in ^ 1;
  const int child_level = level + 1;
  const bool last = child_level >= p.max_depth;
  const double* qc = S.qcoef[in];
  const uint32_t* qs = S.qslot[in];
  const unsigned int stride = gridDim.x * blockDim.x;
  for (unsigned int base = blockIdx.x * blockDim.x; base < n_in; base += stride) {
    unsigned int idx = base + threadIdx.x;
    bool act = idx < n_in;
    uint32_t slot = act ? qs[idx] : 0u;
    if (act) act = !(S.slot_state[slot] & (kStInvalid | kStAmbig | kStOverflow));
    double G[5][5][5];
    uint32_t key = 0;
    if (act) {
      double A[27];
#pragma unroll
      for (int t = 0; t < 27; ++t) A[t] = qc[static_cast<uint64_t>(t) * S.qcap + idx];
      double E = fma(static_cast<double>(child_level) * 0x1p-49, S.slot_m0[slot], S.slot_e0[slot]);
      key = dhi(E);
      double P1[5][3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          double q[5];
          split5(A[tix(0, j, k)], A[tix(1, j, k)], A[tix(2, j, k)], q);
#pragma unroll
          for (int i = 0; i < 5; ++i) P1[i][j][k] = q[i];
        }
      double P2[5][5][3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          double q[5];
          split5(P1[i][0][k], P1[i][1][k], P1[i][2][k], q);
#pragma unroll
          for (int j = 0; j < 5; ++j) P2[i][j][k] = q[j];
        }
#pragma unroll
      for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int i = 0; i < 5; ++i) split5(P2[i][j][0], P2[i][j][1], P2[i][j][2], G[i][j]);
    }
    // classify the 8 children
    uint32_t bits = 0;   // element state bits found by this box
    uint32_t queue = 0;  // children to queue
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
            Sign3 q = sign_d(G[sx + i][sy + j][sz + k], key);
            bool c = (i != 1) && (j != 1) && (k != 1);
            if (c) {
              nonpos |= q.nonpos;
              amb |= !(q.nonpos | q.pos);
            } else {
              notcert |= q.nonpos;
              amb2 |= !(q.nonpos | q.pos);
            }
          }
      if (!act) continue;
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
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      bool want = (queue >> o) & 1u;
      unsigned int pos = warp_append(&S.cnt->level_count[child_level], want);
      if (want) {
        if (pos < S.qcap) {
          const int sx = 2 * (o & 1), sy = 2 * ((o >> 1) & 1), sz = 2 * (o >> 2);
          double* dst = S.qcoef[out];
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
              for (int i = 0; i < 3; ++i)
                dst[static_cast<uint64_t>(tix(i, j, k)) * S.qcap + pos] = G[sx + i][sy + j][sz + k];
          S.qslot[out][pos] = slot;
        } else {
          bits |= kStOverflow;
        }
      }
    }
    if (act) {
      if (bits) atomicOr(&S.slot_state[slot], bits);
      if (bits & kStOverflow) set_status(S.status, kSbQueue);
      S.slot_lev[slot] = static_cast<uint32_t>(child_level);
    }
  }
}

// Verdicts of the refined elements; elements that need the exact tier are
// appended to its list.
__global__ void __launch_bounds__(kFinalizeThreads) finalize_kernel(Batch p) {
  const Scratch& S = p.s;
  const unsigned int n = min(S.cnt->level_count[0], static_cast<unsigned int>(S.qcap));
  unsigned int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x * blockDim.x >= n) return;
  bool act = s < n;
  uint32_t st = act ? S.slot_state[s] : 0u;
  uint32_t lev = act ? S.slot_lev[s] : 0u;
  uint32_t e = act ? S.slot_elem[s] : 0u;
  bool to_exact = act && !(st & kStInvalid) && (st & (kStAmbig | kStOverflow));
  unsigned int pos = warp_append(&S.cnt->exact_count, to_exact);
  if (!act) return;
  uint8_t flag;
  if (st & kStInvalid) {
    flag = make_flag(kVInvalid, lev, 0);
  } else if (to_exact) {
    if (pos < S.exact_cap) {
      S.exact_list[pos] = e;
      return;
    }
    set_status(S.status, kSbQueue);
    flag = make_flag(kVUndecided, p.max_depth, 0);
  } else if (st & kStCap) {
    flag = make_flag(kVUndecided, p.max_depth, 0);
  } else {
    flag = make_flag(kVValid, lev, 0);
  }
  p.flags[p.base + e] = flag;
}

}  // namespace

int refine_blocks() {
  static int blocks = 0;
  if (!blocks) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, refine_kernel, kRefineThreads, 0);
    blocks = (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
  }
  return blocks;
}

cudaError_t launch_refine(const Batch& p, int level, cudaStream_t st) {
  refine_kernel<<<refine_blocks(), kRefineThreads, 0, st>>>(p, level);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Batch& p, cudaStream_t st) {
  // the number of refined elements is only known on the device: launch for
  // the queue capacity bound of this batch and let idle blocks exit
  int64_t bound = p.n < static_cast<int64_t>(p.s.qcap) ? p.n : static_cast<int64_t>(p.s.qcap);
  if (bound <= 0) return cudaSuccess;
  unsigned int blocks = static_cast<unsigned int>((bound + kFinalizeThreads - 1) / kFinalizeThreads);
  finalize_kernel<<<blocks, kFinalizeThreads, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace hexval
