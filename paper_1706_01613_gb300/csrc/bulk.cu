// Bulk pass: Steps 1-4 of the algorithm of Sec. 6 for every element, one
// element per thread.
//
//  bulk64_kernel   FP64: 20 samples (Sec. 5) -> 27 coefficients (Table
//                  t:Tsmall, Sec. 4) -> verdict at depth 0 with certified
//                  signs (element64.cuh).  Undecided elements enter level 0 of
//                  the refinement queue; uncertifiable ones the exact list.
//  bulk32_kernel   the same in FP32 with a certified FP32 error bound; only
//                  clear-cut elements are decided, the rest are escalated to
//                  FP64: the first esc_in_pass of a batch right here, by the
//                  whole warp (warp_items.cuh), the others by the tail kernel.
//  nodes32_kernel  FP64 nodes -> FP32 on the integer pipe, for the indexed
//                  FP32 pass (one conversion per node instead of per corner).
//
// FP32 error bound, u = 2^-24 (element32.cuh): with eps the per-component
// error of the computed edge vectors (input rounding included) and L the
// largest |component| among them, every sample and coefficient is within
// 200 eps L^2 + 740 u L^3 of its exact value; the kernel uses
// 256 eps L^2 + 1024 u L^3 with eps = 2^-23 X + 2^-24 L, X >= |coordinates|.
#include "element32.cuh"
#include "warp_items.cuh"

namespace hexval {

namespace {

constexpr int kBulkThreads = 256;    // largest block of the bulk kernels
constexpr int kBulk32Default = 128;  // default block of the FP32 kernels (measured best
                                     // with 64 on the 128^3 mesh, within noise of 128)

// Escalation of a warp's uncertain elements (all 32 lanes call it; `want`
// marks this lane's element e).  They are appended to the escalation list;
// those that land in its first esc_in_pass positions are redone in FP64 here,
// one at a time by the whole warp, on `sm` (kElemScratch doubles of shared
// memory per warp); the others are written to the list for the tail kernel.
__device__ __forceinline__ void escalate(const Batch& p, bool want, unsigned int e, double* sm) {
  if (!__any_sync(kFull, want)) return;
  const unsigned int pos = warp_append(&p.s.cnt->esc_count, want);
  if (want && pos >= p.esc_in_pass) p.s.esc[pos] = e;  // capacity = batch size
  unsigned int mine = __ballot_sync(kFull, want && pos < p.esc_in_pass);
  while (mine) {
    const int src = __ffs(mine) - 1;
    mine &= mine - 1;
    fp64_element_warp(p, __shfl_sync(kFull, e, src), sm);
  }
}

// Outputs of one element of the FP32 pass (all 32 lanes call it; outcomes of
// fp32_classify, or 5 for a connectivity entry out of range): escalations go
// to FP64 (escalate); of the elements to refine, the first r32_in_pass of the
// batch are redone in FP64 here by the whole warp and the others are listed
// for the FP32 refinement (their flag comes later); the rest get their
// verdict here.
__device__ __forceinline__ void finish32(const Batch& p, bool act, int outcome, unsigned int e,
                                         float lo, float hi, double* sm) {
  const Scratch& S = p.s;
  const bool want_e = act && outcome == 3;
  escalate(p, want_e, e, sm);
  const bool want_r = act && outcome == 2 && p.max_depth > 0;
  unsigned int rpos = 0;
  bool r_here = false;
  if (__any_sync(kFull, want_r)) {  // rare: skip the list work otherwise
    rpos = warp_append(&S.cnt->r32_count, want_r);
    r_here = want_r && rpos < p.r32_in_pass;  // FP64 redo right here
    unsigned int mine = __ballot_sync(kFull, r_here);
    while (mine) {
      const int src = __ffs(mine) - 1;
      mine &= mine - 1;
      fp64_element_warp(p, __shfl_sync(kFull, e, src), sm);
    }
  }
  if (!act || want_e || r_here) return;
  const int64_t g = p.base + e;
  if (outcome == 5) {
    p.flags[g] = make_flag(kVUndecided, 0, 0);
    set_status(S.status, kSbIndex);
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (p.bmin) p.bmin[g] = nan;
    if (p.bmax) p.bmax[g] = nan;
    return;
  }
  if (want_r)
    S.r32[rpos] = e;  // capacity = batch size
  else  // outcome 2 with a depth cap of 0: undecided at the root
    p.flags[g] = make_flag(outcome == 0 ? kVInvalid : (outcome == 1 ? kVValid : kVUndecided), 0, 0);
  if (p.bmin) p.bmin[g] = f2d_int(lo);
  if (p.bmax) p.bmax[g] = f2d_int(hi);
}

// This warp's part of the dynamic shared memory of a bulk FP32 kernel.
__device__ __forceinline__ double* warp_scratch() {
  extern __shared__ double bulk_sm[];
  return bulk_sm + (threadIdx.x >> 5) * kElemScratch;
}

inline size_t scratch_bytes(int threads) {
  return static_cast<size_t>(threads / 32) * kElemScratch * sizeof(double);
}

__global__ void __launch_bounds__(kBulkThreads) bulk64_kernel(Batch p) {
  pdl_wait();
  pdl_trigger();
  unsigned int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool act = i < static_cast<unsigned int>(p.n);
  fp64_element(p, act, act ? i : 0u);
}

// Decides what FP32 can decide; everything else is escalated to FP64.
// At most 64 registers: this kernel relies on many resident warps to cover
// its gather latency (measured faster than an 80-register build without
// spills, at two-thirds of the warps).
template <bool INDEXED>
__global__ void __launch_bounds__(kBulkThreads, 4) bulk32_kernel(Batch p) {
  pdl_wait();
  pdl_trigger();
  const Scratch& S = p.s;
  unsigned int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool act = i < static_cast<unsigned int>(p.n);
  int64_t g = p.base + i;
  int outcome = -1;  // 0 inv, 1 valid, 3 escalate, 5 bad index
  float lo = 0.f, hi = 0.f;
  if (act) {
    bool bad = false;
    V3<float> Y[8];
    float X;  // bound on |coordinate| of the element
    if (!INDEXED) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        Y[k].x = d2f_int(__ldg(p.soa + (3 * k + 0) * p.stride + g), bad);
        Y[k].y = d2f_int(__ldg(p.soa + (3 * k + 1) * p.stride + g), bad);
        Y[k].z = d2f_int(__ldg(p.soa + (3 * k + 2) * p.stride + g), bad);
      }
      X = node_magnitude(Y);
    } else {
      const int4* c4 = reinterpret_cast<const int4*>(p.conn + 8 * g);
      const int4 c0 = __ldg(c4), c1 = __ldg(c4 + 1);
      if (!ids_in_range(c0, c1, p.n_nodes)) {
        outcome = 5;
      } else {
        const int id[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
        const float4* N = reinterpret_cast<const float4*>(S.node32);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float4 h = __ldg(N + id[k]);
          Y[k] = {h.x, h.y, h.z};
        }
        X = fabsmax3(Y[0]);  // completed with 3 L; out-of-range nodes: +inf records
      }
    }
    if (outcome < 0) outcome = fp32_decide<INDEXED>(Y, X, bad, lo, hi);
  }
  finish32(p, act, outcome, i, lo, hi, warp_scratch());
}

// Indexed FP32 pass on a persistent grid with its inputs staged through
// shared memory by asynchronous copies.  Block b works on tiles b, b + G,
// b + 2G, ... (G blocks, one element per thread and tile).  At the start of
// tile j a thread takes the node records of its element of tile j and the
// connectivity row of its element of tile j+1 out of shared memory into
// registers, then starts the copies of the connectivity of tile j+2 and of
// the node records of tile j+1 into the same places, and works on tile j
// while they are in flight: neither the HBM latency of the connectivity nor
// the L2 latency of the gathered node records is exposed.  Each thread
// stages only its own element's data, so no block barrier is needed.
// Shared memory per block of T threads (W warps):
//   node records  float4 [W][8 nodes][32 lanes]      128 T bytes
//   connectivity  int4   [2 halves][T]                 32 T bytes
//   FP64 scratch  double [W][kElemScratch]            (escalations)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned int s = static_cast<unsigned int>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

inline size_t staged_bytes(int threads) {
  return static_cast<size_t>(threads) * 160 + scratch_bytes(threads);
}

// Up to 85 registers (no spills): the staging hides the gather latency, so
// this kernel needs fewer resident warps than bulk32_kernel.
__global__ void __launch_bounds__(kBulkThreads, 3) bulk32s_kernel(Batch p) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ float4 stage[];
  const Scratch& S = p.s;
  const unsigned int T = blockDim.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  float4* const my_nodes = stage + w * 256u + lane;                            // record k: [32 k]
  int4* const my_conn = reinterpret_cast<int4*>(stage + 8u * T) + threadIdx.x;  // half h: [h T]
  double* const wsc = reinterpret_cast<double*>(stage + 10u * T) + w * kElemScratch;
  const float4* const N = reinterpret_cast<const float4*>(S.node32);
  const unsigned int n = static_cast<unsigned int>(p.n);  // a batch holds < 2^31 elements
  const unsigned int tiles = (n + T - 1) / T;
  if (blockIdx.x >= tiles) return;
  const unsigned int my_tiles = (tiles - 1 - blockIdx.x) / gridDim.x + 1;
  const unsigned int step = gridDim.x * T;
  auto issue_conn = [&](unsigned int e) {
    if (e < n) {
      const int* src = p.conn + 8 * (p.base + static_cast<int64_t>(e));
      cp_async16(my_conn, src);
      cp_async16(my_conn + T, src + 4);
    }
  };
  // node records of element e from its connectivity (in registers); false
  // if an entry is out of range (nothing is copied then)
  auto issue_nodes = [&](unsigned int e, const int4& c0, const int4& c1) {
    const int id[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    const bool ok = ids_in_range(c0, c1, p.n_nodes);
    if (ok && e < n) {
#pragma unroll
      for (int k = 0; k < 8; ++k) cp_async16(my_nodes + 32 * k, N + id[k]);
    }
    return ok;
  };
  unsigned int e = blockIdx.x * T + threadIdx.x;  // this thread's element of tile j
  issue_conn(e);
  cp_commit();
  cp_wait_all();
  int4 c0 = my_conn[0], c1 = my_conn[T];
  __syncwarp();
  issue_conn(e + step);
  bool ok_next = issue_nodes(e, c0, c1);
  cp_commit();
  for (unsigned int j = 0; j < my_tiles; ++j, e += step) {
    cp_wait_all();  // node records of tile j, connectivity of tile j+1
    const bool act = e < n, ok = ok_next;
    V3<float> Y[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float4 h = my_nodes[32 * k];
      Y[k] = {h.x, h.y, h.z};
    }
    c0 = my_conn[0];
    c1 = my_conn[T];
    __syncwarp();  // reads done before the copies below overwrite
    issue_conn(e + 2 * step);
    ok_next = issue_nodes(e + step, c0, c1);
    cp_commit();
    int outcome = -1;
    float lo = 0.f, hi = 0.f;
    if (act) {
      outcome = ok ? fp32_decide<true>(Y, fabsmax3(Y[0]), false, lo, hi) : 5;
    }
    finish32(p, act, outcome, e, lo, hi, wsc);
  }
  cp_wait_all();
}

int bulk32s_blocks(int threads) {
  static int cached_threads = -1, blocks = 0;
  if (threads != cached_threads) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(bulk32s_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(staged_bytes(kBulkThreads)));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, bulk32s_kernel, threads,
                                                  staged_bytes(threads));
    blocks = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
    cached_threads = threads;
  }
  return blocks;
}

template <int LANE>
__device__ __forceinline__ float lane(const F2& a) {
  return LANE == 0 ? a.v.x : a.v.y;
}

template <int LANE>
__device__ __forceinline__ void lane_of(const Scaled<F2>& s, Scaled<float>& q) {
#pragma unroll
  for (int k = 0; k < 8; ++k) q.corner[k] = lane<LANE>(s.corner[k]);
#pragma unroll
  for (int e = 0; e < 12; ++e) {
    q.edgeC[e] = lane<LANE>(s.edgeC[e]);
    q.edge[e] = lane<LANE>(s.edge[e]);
  }
#pragma unroll
  for (int f = 0; f < 6; ++f) q.face[f] = lane<LANE>(s.face[f]);
  q.centre = lane<LANE>(s.centre);
}

template <int LANE>
__device__ __forceinline__ V3<float> lane_v(const V3<F2>& v) {
  return {lane<LANE>(v.x), lane<LANE>(v.y), lane<LANE>(v.z)};
}

template <int LANE>
__device__ __forceinline__ float edge_magnitude_lane(const V3<F2> a[4], const V3<F2> b[4],
                                                     const V3<F2> g[4]) {
  V3<float> x[4], y[4], z[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    x[q] = lane_v<LANE>(a[q]);
    y[q] = lane_v<LANE>(b[q]);
    z[q] = lane_v<LANE>(g[q]);
  }
  return edge_magnitude(x, y, z);
}

// The FP32 decision of two elements with packed f32x2 arithmetic (lane 0 and
// lane 1 of every F2 value): per element the same operations, roundings,
// bound and outcome as fp32_decide.  X0 / X1 as for fp32_root.
template <bool INDEXED>
__device__ __forceinline__ void fp32_decide2(const V3<F2> Y[8], float X0, float X1, bool bad0,
                                             bool bad1, int& r0, int& r1, float& lo0, float& hi0,
                                             float& lo1, float& hi1) {
  V3<F2> a[4], b[4], gg[4];
  edges_from_nodes(Y, a, b, gg);
  const float L0 = edge_magnitude_lane<0>(a, b, gg), L1 = edge_magnitude_lane<1>(a, b, gg);
  if (INDEXED) {
    X0 = fmaf(3.f, L0, X0);
    X1 = fmaf(3.f, L1, X1);
  }
  const float eps0 = fmaf(0x1p-24f, L0, 0x1p-23f * X0), eps1 = fmaf(0x1p-24f, L1, 0x1p-23f * X1);
  const float L20 = L0 * L0, L21 = L1 * L1;
  const float E0 = fmaf(256.f * eps0, L20, 1024.f * 0x1p-24f * (L20 * L0)) * 1.0001f;
  const float E1 = fmaf(256.f * eps1, L21, 1024.f * 0x1p-24f * (L21 * L1)) * 1.0001f;
  bad0 |= !(L0 >= 0x1p-30f) || !(E0 < 0x1p100f);
  bad1 |= !(L1 >= 0x1p-30f) || !(E1 < 0x1p100f);
  Scaled<F2> s;
  coefficients_from_edges(a, b, gg, s);
  Scaled<float> q;
  lane_of<0>(s, q);
  r0 = fp32_classify(q, E0, lo0, hi0);
  lane_of<1>(s, q);
  r1 = fp32_classify(q, E1, lo1, hi1);
  if (bad0) r0 = 3;
  if (bad1) r1 = 3;
}

// The FP32 pass on two elements per thread (2t and 2t+1) with packed f32x2
// arithmetic; decisions and bounds per element exactly as bulk32_kernel.
constexpr int kPairThreads = 128;

template <bool INDEXED>
__global__ void __launch_bounds__(kPairThreads, 4) bulk32x2_kernel(Batch p) {
  pdl_wait();
  pdl_trigger();
  const Scratch& S = p.s;
  const unsigned int t = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned int i0 = 2 * t, i1 = 2 * t + 1;
  const unsigned int n = static_cast<unsigned int>(p.n);
  const bool act0 = i0 < n, act1 = i1 < n;
  const unsigned int j1 = act1 ? i1 : i0;  // an idle second lane repeats the first
  int out0 = -1, out1 = -1;                // 0 inv, 1 valid, 3 escalate, 5 bad index
  float lo0 = 0.f, hi0 = 0.f, lo1 = 0.f, hi1 = 0.f;
  if (act0) {
    bool bad0 = false, bad1 = false;
    V3<F2> Y[8];
    float X0 = 0.f, X1 = 0.f;
    if (!INDEXED) {
      const int64_t g0 = p.base + i0, g1 = p.base + j1;
      V3<float> Y0[8], Y1[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const double* q = p.soa + (3 * k) * p.stride;
        Y0[k].x = d2f_int(__ldg(q + g0), bad0);
        Y1[k].x = d2f_int(__ldg(q + g1), bad1);
        Y0[k].y = d2f_int(__ldg(q + p.stride + g0), bad0);
        Y1[k].y = d2f_int(__ldg(q + p.stride + g1), bad1);
        Y0[k].z = d2f_int(__ldg(q + 2 * p.stride + g0), bad0);
        Y1[k].z = d2f_int(__ldg(q + 2 * p.stride + g1), bad1);
        Y[k].x = F2(Y0[k].x, Y1[k].x);
        Y[k].y = F2(Y0[k].y, Y1[k].y);
        Y[k].z = F2(Y0[k].z, Y1[k].z);
      }
      X0 = node_magnitude(Y0);
      X1 = node_magnitude(Y1);
    } else {
      const int4* c4 = reinterpret_cast<const int4*>(p.conn + 8 * (p.base + i0));
      int4 c0 = __ldg(c4), c1 = __ldg(c4 + 1);
      int4 c2 = act1 ? __ldg(c4 + 2) : c0, c3 = act1 ? __ldg(c4 + 3) : c1;
      if (!ids_in_range(c0, c1, p.n_nodes)) {
        out0 = 5;
        c0 = c1 = make_int4(0, 0, 0, 0);  // node 0 exists (n_nodes >= 1)
      }
      if (!ids_in_range(c2, c3, p.n_nodes)) {
        out1 = 5;
        c2 = c3 = make_int4(0, 0, 0, 0);
      }
      const int id0[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
      const int id1[8] = {c2.x, c2.y, c2.z, c2.w, c3.x, c3.y, c3.z, c3.w};
      const float4* N = reinterpret_cast<const float4*>(S.node32);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 h0 = __ldg(N + id0[k]), h1 = __ldg(N + id1[k]);
        Y[k].x = F2(h0.x, h1.x);
        Y[k].y = F2(h0.y, h1.y);
        Y[k].z = F2(h0.z, h1.z);
      }
      // completed with 3 L; out-of-range nodes: +inf records
      X0 = max3f(fabsf(Y[0].x.v.x), fabsf(Y[0].y.v.x), fabsf(Y[0].z.v.x));
      X1 = max3f(fabsf(Y[0].x.v.y), fabsf(Y[0].y.v.y), fabsf(Y[0].z.v.y));
    }
    int r0, r1;
    fp32_decide2<INDEXED>(Y, X0, X1, bad0, bad1, r0, r1, lo0, hi0, lo1, hi1);
    if (out0 < 0) out0 = r0;
    if (out1 < 0) out1 = r1;
  }
  finish32(p, act0, out0, i0, lo0, hi0, warp_scratch());
  finish32(p, act1, out1, i1, lo1, hi1, warp_scratch());
}

// FP64 node -> FP32 record {x, y, z, w} (16 bytes, one vector load in the
// bulk pass).  A node with a coordinate outside the FP32 range gets
// x = y = z = +inf and w = 1, which sends every element touching it to FP64
// (element32.cuh).
__device__ __forceinline__ float4 node_record(float x, float y, float z, bool bad) {
  const float inf = __int_as_float(0x7f800000);
  return bad ? make_float4(inf, inf, inf, 1.f) : make_float4(x, y, z, 0.f);
}

__global__ void __launch_bounds__(256) nodes32_kernel(const double* nodes, int64_t n_nodes,
                                                      float4* out) {
  pdl_trigger();
  int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  bool bad = false;
  float x = d2f_int(__ldg(nodes + 3 * i), bad);
  float y = d2f_int(__ldg(nodes + 3 * i + 1), bad);
  float z = d2f_int(__ldg(nodes + 3 * i + 2), bad);
  out[i] = node_record(x, y, z, bad);
}

// Two nodes per thread with 16-byte loads (nodes 16-byte aligned).
__global__ void __launch_bounds__(256) nodes32x2_kernel(const double2* nodes, int64_t n_nodes,
                                                        float4* out) {
  pdl_trigger();
  int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t i = 2 * t;
  if (i >= n_nodes) return;
  if (i + 1 < n_nodes) {
    double2 a = __ldg(nodes + 3 * t), b = __ldg(nodes + 3 * t + 1), c = __ldg(nodes + 3 * t + 2);
    bool bad0 = false, bad1 = false;
    float x0 = d2f_int(a.x, bad0), y0 = d2f_int(a.y, bad0), z0 = d2f_int(b.x, bad0);
    float x1 = d2f_int(b.y, bad1), y1 = d2f_int(c.x, bad1), z1 = d2f_int(c.y, bad1);
    out[i] = node_record(x0, y0, z0, bad0);
    out[i + 1] = node_record(x1, y1, z1, bad1);
  } else {
    const double* q = reinterpret_cast<const double*>(nodes) + 3 * i;
    bool bad = false;
    float x = d2f_int(__ldg(q), bad), y = d2f_int(__ldg(q + 1), bad), z = d2f_int(__ldg(q + 2), bad);
    out[i] = node_record(x, y, z, bad);
  }
}

}  // namespace

cudaError_t launch_bulk64(const Batch& p, cudaStream_t st) {
  if (p.n <= 0) return cudaSuccess;
  const int bt = p.bulk_threads ? p.bulk_threads : kBulkThreads;
  unsigned int blocks = static_cast<unsigned int>((p.n + bt - 1) / bt);
  return launch_pdl(bulk64_kernel, blocks, bt, 0, st, p);
}

cudaError_t launch_bulk32(const Batch& p, cudaStream_t st) {
  if (p.n <= 0) return cudaSuccess;
  if (p.pair32) {
    const int bt = p.bulk_threads ? min(p.bulk_threads, kPairThreads) : kPairThreads;
    int64_t threads = (p.n + 1) / 2;
    unsigned int blocks = static_cast<unsigned int>((threads + bt - 1) / bt);
    if (p.indexed)
      return launch_pdl(bulk32x2_kernel<true>, blocks, bt, scratch_bytes(bt), st, p);
    return launch_pdl(bulk32x2_kernel<false>, blocks, bt, scratch_bytes(bt), st, p);
  }
  const int bt = p.bulk_threads ? p.bulk_threads : kBulk32Default;
  if (p.indexed && p.prefetch32) {
    int64_t need = (p.n + bt - 1) / bt;
    int64_t blocks = bulk32s_blocks(bt);
    return launch_pdl(bulk32s_kernel, static_cast<unsigned int>(need < blocks ? need : blocks), bt,
                      staged_bytes(bt), st, p);
  }
  unsigned int blocks = static_cast<unsigned int>((p.n + bt - 1) / bt);
  if (p.indexed) return launch_pdl(bulk32_kernel<true>, blocks, bt, scratch_bytes(bt), st, p);
  return launch_pdl(bulk32_kernel<false>, blocks, bt, scratch_bytes(bt), st, p);
}

cudaError_t launch_nodes32(const Batch& p, cudaStream_t st) {
  if (p.n_nodes <= 0) return cudaSuccess;
  if (reinterpret_cast<uintptr_t>(p.nodes) % 16 == 0) {
    int64_t threads = (p.n_nodes + 1) / 2;
    unsigned int blocks = static_cast<unsigned int>((threads + 255) / 256);
    nodes32x2_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const double2*>(p.nodes),
                                             p.n_nodes, reinterpret_cast<float4*>(p.s.node32));
    return cudaGetLastError();
  }
  unsigned int blocks = static_cast<unsigned int>((p.n_nodes + 255) / 256);
  nodes32_kernel<<<blocks, 256, 0, st>>>(p.nodes, p.n_nodes,
                                         reinterpret_cast<float4*>(p.s.node32));
  return cudaGetLastError();
}

}  // namespace hexval
