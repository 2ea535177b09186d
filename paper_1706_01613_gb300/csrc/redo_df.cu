// Double-float redo of the FP32 form's escalations (HEXVAL_OPT_DFREDO): the
// escalation list entries the FP32 pass leaves (beyond the first esc_in_pass,
// which it redoes in FP64 itself) are recomputed one per thread in
// double-float (element_df.cuh), about 44 bits at FP32 throughput; what the
// redo decides at depth 0 (valid or invalid) is final, and the rest (a sign
// still uncertain, a subdivision, an element outside the double-float range)
// is listed in esc3 for the tail kernel's FP64 redo.  A kernel of its own so
// that it runs at full occupancy: the cooperative tail kernel holds two
// blocks per SM.
#include "element_df.cuh"

namespace hexval {

namespace {

constexpr int kRedoThreads = 128;

// Element e of the batch: all lanes call it (warp_append).
__device__ __forceinline__ void df_item(const Batch& p, bool act, uint32_t e) {
  const Scratch& S = p.s;
  int outcome = 3;
  double lo = 0.0, hi = 0.0;
  const int64_t g = p.base + e;
  if (act) {
    Scaled<DF> s;
    float E;
    if (df_root(p, g, s, E)) outcome = df_classify(s, E, lo, hi);
  }
  const bool redo = act && outcome >= 2;
  const unsigned int pos = warp_append(&S.cnt->esc3_count, redo);
  const unsigned int decided = __popc(__ballot_sync(0xffffffffu, act && !redo));
  if ((threadIdx.x & 31) == 0 && decided) atomicAdd(&S.cnt->df_count, decided);
  if (!act) return;
  if (redo) {
    S.esc3[pos] = e;  // at most one entry per element of the batch
    return;
  }
  p.flags[g] = make_flag(outcome == 0 ? kVInvalid : kVValid, 0, 0);
  if (p.bmin) p.bmin[g] = lo;
  if (p.bmax) p.bmax[g] = hi;
}

__global__ void __launch_bounds__(kRedoThreads, 4) redo_df_kernel(Batch p) {
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
    df_item(p, act, act ? ldcg(esc + i) : 0u);
  }
}

int redo_blocks() {
  static int blocks = 0;
  if (!blocks) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, redo_df_kernel, kRedoThreads, 0);
    blocks = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }
  return blocks;
}

}  // namespace

cudaError_t launch_redo_df(const Batch& p, cudaStream_t st) {
  return launch_pdl(redo_df_kernel, static_cast<unsigned int>(redo_blocks()), kRedoThreads, 0, st, p);
}

}  // namespace hexval
