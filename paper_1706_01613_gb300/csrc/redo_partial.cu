// Partial FP64 redo of the FP32 form's escalations (HEXVAL_OPT_PARTIAL64):
// the escalation list entries the FP32 pass leaves (beyond the first
// esc_in_pass, which it redoes in FP64 itself) are taken one per thread.  The
// element's nodes are read once, in FP64; its FP32 classification is
// recomputed from them as the pass computed it (the same rounding to FP32,
// the same bound E: outcome 3), and only the signs it leaves unsettled are
// evaluated in FP64 (fp32_unsettled, fp64_partial).  What this decides at
// depth 0 is final, with the FP32 extremes as bmin / bmax; the rest is listed
// in esc3 for the tail kernel's full FP64 redo.  A kernel of its own so that
// the scattered element reads run at full occupancy: the cooperative tail
// kernel holds 8 warps per SM.
#include "element32.cuh"
#include "element64.cuh"

namespace hexval {
namespace {

constexpr int kPartialThreads = 128;

// Element e of the batch: all lanes call it (warp_append).
__device__ __forceinline__ void partial_item(const Batch& p, bool act, uint32_t e) {
  const Scratch& S = p.s;
  const int64_t g = p.base + e;
  int r = -1;
  float lo = 0.f, hi = 0.f;
  if (act) {
    V3<double> Xd[8];
    if (load_element(p, g, Xd)) {  // in range: checked by the FP32 pass
      V3<float> Y[8];
      bool bad = false;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        Y[k] = {d2f_int(Xd[k].x, bad), d2f_int(Xd[k].y, bad), d2f_int(Xd[k].z, bad)};
      Scaled<float> s;
      float E = 0.f;
      // |coordinate| bound as the pass forms it: all 8 nodes (SoA), node 1
      // completed with 3 L by fp32_root (indexed)
      const bool ok = p.indexed ? fp32_root<true>(Y, fabsmax3(Y[0]), bad, s, E)
                                : fp32_root<false>(Y, node_magnitude(Y), bad, s, E);
      if (ok && fp32_classify(s, E, lo, hi) == 3) r = fp64_partial(Xd, fp32_unsettled(s, E));
    }
  }
  const bool rest = act && r < 0;
  const unsigned int pos = warp_append(&S.cnt->esc3_count, rest);
  const unsigned int decided = __popc(__ballot_sync(0xffffffffu, act && !rest));
  if ((threadIdx.x & 31) == 0 && decided) atomicAdd(&S.cnt->part_count, decided);
  if (!act) return;
  if (rest) {
    S.esc3[pos] = e;  // at most one entry per element of the batch
    return;
  }
  p.flags[g] = make_flag(r == 0 ? kVInvalid : kVValid, 0, 0);
  if (p.bmin) p.bmin[g] = f2d_int(lo);
  if (p.bmax) p.bmax[g] = f2d_int(hi);
}

__global__ void __launch_bounds__(kPartialThreads) redo_partial_kernel(Batch p) {
  pdl_wait();
  pdl_trigger();
  const Scratch& S = p.s;
  const unsigned int n_list = ldcg(&S.cnt->esc_count);
  const unsigned int n = n_list > p.esc_in_pass ? n_list - p.esc_in_pass : 0u;
  const uint32_t* esc = S.esc + p.esc_in_pass;
  const unsigned int stride = gridDim.x * blockDim.x;
  // uniform trip count per warp: blockDim.x is a multiple of 32
  for (unsigned int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
    const unsigned int i = i0 + (threadIdx.x & 31u);
    const bool act = i < n;
    partial_item(p, act, act ? ldcg(esc + i) : 0u);
  }
}

int partial_blocks() {
  static int blocks = 0;
  if (!blocks) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, redo_partial_kernel, kPartialThreads, 0);
    blocks = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }
  return blocks;
}

}  // namespace

cudaError_t launch_redo_partial(const Batch& p, cudaStream_t st) {
  return launch_pdl(redo_partial_kernel, static_cast<unsigned int>(partial_blocks()),
                    kPartialThreads, 0, st, p);
}

}  // namespace hexval
