// First refinement level of the FP32-filtered form in a kernel of its own
// (HEXVAL_OPT_LEVEL1), between the FP32 pass and the tail.
//
// The elements the FP32 pass lists for the FP32 refinement (all 20 samples
// certainly positive, a coefficient certainly non-positive: Sec. 6, Step 4)
// are many on some inputs (about a quarter of boundary-layer elements) and
// most of them are decided on level 1.  The tail kernel, a cooperative
// launch with a few fat blocks, runs such a throughput step at low
// occupancy; here one thread per listed element, at full occupancy,
// recomputes the element's FP32 root box exactly as the tail would
// (load_element32, fp32_root, fp32_classify, refine32.cuh) and splits it once
// (refine1_fp32).  A verdict on level 1 is final; the elements that need
// deeper levels, or meet a sign FP32 cannot settle, are listed in r32b,
// which the tail's FP32 refinement takes instead of the refinement list, so
// they reach the same verdicts as without this kernel.
#include "refine32.cuh"

namespace hexval {

namespace {

constexpr int kLevel1Threads = 128;

// At most 128 registers (some of the 125 split values spill to L1): twice
// the resident warps of an uncapped build, measured faster on boundary
// layers (2^22 elements, 1.07 M listed: 191 -> 164 us).
__global__ void __launch_bounds__(kLevel1Threads, 4) level1_kernel(Batch p) {
  pdl_wait();
  pdl_trigger();
  const Scratch& S = p.s;
  const unsigned int n_rl = ldcg(&S.cnt->r32_count);
  const unsigned int n = n_rl > p.r32_in_pass ? n_rl - p.r32_in_pass : 0u;
  const uint32_t* list = S.r32 + p.r32_in_pass;
  const unsigned int stride = gridDim.x * blockDim.x;
  const unsigned int lane = threadIdx.x & 31u;
  // uniform trip count per warp: blockDim.x is a multiple of 32
  for (unsigned int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
    const unsigned int i = i0 + lane;
    const bool act = i < n;
    uint32_t e = 0;
    int flag = -1;
    if (act) {
      e = ldcg(list + i);
      V3<float> Y[8];
      float X, E = 0.f, lo = 0.f, hi = 0.f;
      bool bad;
      Scaled<float> s;
      load_element32(p, p.base + e, Y, X, bad);  // in range: checked by the FP32 pass
      const bool ok =
          p.indexed ? fp32_root<true>(Y, X, bad, s, E) : fp32_root<false>(Y, X, bad, s, E);
      if (ok) {
        fp32_classify(s, E, lo, hi);
        flag = refine1_fp32(s, E, lo, hi, p.max_depth);
      }
    }
    const bool left = act && flag < 0;
    const unsigned int pos = warp_append(&S.cnt->r32b_count, left);
    if (left) S.r32b[pos] = e;  // capacity = batch size
    if (act && flag >= 0) p.flags[p.base + e] = static_cast<uint8_t>(flag);
    const unsigned int m = __ballot_sync(0xffffffffu, act);
    if (lane == 0 && m) atomicAdd(&S.cnt->l1_count, static_cast<unsigned int>(__popc(m)));
  }
}

int level1_blocks() {
  static int blocks = 0;
  if (!blocks) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, level1_kernel, kLevel1Threads, 0);
    blocks = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }
  return blocks;
}

}  // namespace

// A full-occupancy grid that loops over the list (its length is known only
// on the device).
cudaError_t launch_level1(const Batch& p, cudaStream_t st) {
  if (p.n <= 0) return cudaSuccess;
  const int64_t need = (p.n + kLevel1Threads - 1) / kLevel1Threads;
  const int64_t blocks = level1_blocks();
  return launch_pdl(level1_kernel, static_cast<unsigned int>(need < blocks ? need : blocks),
                    kLevel1Threads, 0, st, p);
}

}  // namespace hexval
