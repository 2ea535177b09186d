// Bulk pass: Steps 1-4 of the algorithm of Sec. 6 for every element, one
// element per thread.
//
//  bulk64_kernel   FP64: 20 samples (Sec. 5) -> 27 coefficients (Table
//                  t:Tsmall, Sec. 4) -> verdict at depth 0, with certified
//                  signs.  Undecided elements enter level 0 of the refinement
//                  queue; uncertifiable ones go to the exact tier.
//  bulk32_kernel   the same in FP32 with a certified FP32 error bound; only
//                  clear-cut elements are decided, the rest are appended to
//                  the escalation list and redone by bulk64_kernel.
//  nodes32_kernel  FP64 nodes -> (hi, lo) FP32 pairs for the indexed FP32
//                  pass, on the integer pipe.
//
// Error bounds (derivations in the design notes):
//  FP64: with L the largest |component| of the 12 computed edge vectors and
//        u = 2^-53, every sample and coefficient is within 930 u L^3 of its
//        exact value; the kernel uses E = 2^(3 e_L - 3107) >= 2^-42 L^3 with
//        e_L the biased exponent of L.
//  FP32: with u = 2^-24, eps the per-component error of the edge vectors
//        (input rounding included): |error| <= 200 eps L^2 + 740 u L^3; the
//        kernel uses 256 eps L^2 + 1024 u L^3.
#include "hexval_internal.cuh"

namespace hexval {

namespace {

constexpr int kBulkThreads = 256;

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

__device__ __forceinline__ void minmax_f(const Scaled<float>& s, float& lo, float& hi) {
  float mn0 = s.corner[0], mx0 = s.corner[0];
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    mn0 = fminf(mn0, s.corner[k]);
    mx0 = fmaxf(mx0, s.corner[k]);
  }
  float mn1 = s.edge[0], mx1 = s.edge[0];
#pragma unroll
  for (int e = 1; e < 12; ++e) {
    mn1 = fminf(mn1, s.edge[e]);
    mx1 = fmaxf(mx1, s.edge[e]);
  }
  float mn2 = s.face[0], mx2 = s.face[0];
#pragma unroll
  for (int f = 1; f < 6; ++f) {
    mn2 = fminf(mn2, s.face[f]);
    mx2 = fmaxf(mx2, s.face[f]);
  }
  lo = fminf(fminf(mn0, mn1 * 0.5f), fminf(mn2 * 0.25f, s.centre * 0.125f));
  hi = fmaxf(fmaxf(mx0, mx1 * 0.5f), fmaxf(mx2 * 0.25f, s.centre * 0.125f));
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
  double t[27];
  store_tensor(s, t);
#pragma unroll
  for (int q = 0; q < 27; ++q) S.qcoef[0][q * S.qcap + slot] = t[q];
}

// One element in FP64.  `e` is the element's index within the batch.
template <bool FROM_LIST>
__global__ void __launch_bounds__(kBulkThreads) bulk64_kernel(Batch p) {
  const Scratch& S = p.s;
  unsigned int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned int n = FROM_LIST ? S.cnt->esc_count : static_cast<unsigned int>(p.n);
  if (FROM_LIST && blockIdx.x * blockDim.x >= n) return;  // whole block idle
  bool act = i < n;
  uint32_t e = act ? (FROM_LIST ? S.esc[i] : i) : 0u;
  int64_t g = p.base + e;

  V3<double> X[8];
  int outcome = -1;  // 0 inv, 1 valid, 2 refine, 3 exact, 4 nonfinite, 5 bad index
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
  // refinement queue (level 0) and exact list, warp-aggregated
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
  switch (outcome) {
    case 0: flag = make_flag(kVInvalid, 0, 0); break;
    case 1: flag = make_flag(kVValid, 0, 0); break;
    case 4: flag = make_flag(kVNonfinite, 0, 0); lo = hi = __longlong_as_double(0x7ff8000000000000LL); break;
    case 5: flag = make_flag(kVUndecided, 0, 0); lo = hi = __longlong_as_double(0x7ff8000000000000LL);
            set_status(S.status, kSbIndex); break;
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

// ---------------------------------------------------------------- FP32 ----
// FP64 -> FP32 on the integer pipe, rounding the magnitude to nearest (ties
// up): |result - x| <= 2^-24 |x|.  Sets `bad` when x is outside the exponent
// range [2^-126, 2^125) (zero is fine).
__device__ __forceinline__ float d2f_int(double x, bool& bad) {
  long long bits = __double_as_longlong(x);
  uint32_t hi = static_cast<uint32_t>(bits >> 32), lo = static_cast<uint32_t>(bits);
  uint32_t e = (hi >> 20) & 0x7ffu;
  bool zero = ((hi << 1) | lo) == 0u;
  uint32_t f = __funnelshift_l(lo, hi, 3);
  f = (f & 0x7fffffffu) ^ 0x40000000u;  // exponent field e - 896 for e in [897, 1149]
  f += (lo >> 28) & 1u;                 // rounding (a carry moves into the exponent)
  f |= hi & 0x80000000u;
  bad |= !zero && (e - 897u > 252u);
  return zero ? __uint_as_float(hi & 0x80000000u) : __uint_as_float(f);
}

__device__ __forceinline__ float fabsmax3(float m, const V3<float>& v) {
  return fmaxf(m, fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.z))));
}

// Decides what FP32 can decide; everything else is escalated to FP64.
// INDEXED: nodes come from the (hi, lo) FP32 copy made by nodes32_kernel and
// are translated to node 1 before the edge vectors are formed.
template <bool INDEXED>
__global__ void __launch_bounds__(kBulkThreads) bulk32_kernel(Batch p) {
  const Scratch& S = p.s;
  unsigned int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool act = i < static_cast<unsigned int>(p.n);
  int64_t g = p.base + i;
  int outcome = -1;  // 0 inv, 1 valid, 3 escalate, 5 bad index
  float lo = 0.f, hi = 0.f;
  if (act) {
    bool bad = false;
    V3<float> a[4], b[4], gg[4];
    float X;  // bound on |coordinate| of the element
    float epsK;  // per-component error of the edge vectors, as eps = epsK-term + u L
    if (!INDEXED) {
      V3<float> Y[8];
      X = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        Y[k].x = d2f_int(__ldg(p.soa + (3 * k + 0) * p.stride + g), bad);
        Y[k].y = d2f_int(__ldg(p.soa + (3 * k + 1) * p.stride + g), bad);
        Y[k].z = d2f_int(__ldg(p.soa + (3 * k + 2) * p.stride + g), bad);
        X = fabsmax3(X, Y[k]);
      }
      edges_from_nodes(Y, a, b, gg);
      epsK = 0x1p-23f * X;  // two inputs rounded at 2^-24 |x| each
    } else {
      const int4* c4 = reinterpret_cast<const int4*>(p.conn + 8 * g);
      int4 c0 = __ldg(c4), c1 = __ldg(c4 + 1);
      int id[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
      bool ok = true;
#pragma unroll
      for (int k = 0; k < 8; ++k) ok &= (id[k] >= 0) & (static_cast<int64_t>(id[k]) < p.n_nodes);
      if (!ok) {
        outcome = 5;
      } else {
        const float4* N = reinterpret_cast<const float4*>(S.node32);
        float4 h0 = __ldg(N + 2 * static_cast<int64_t>(id[0]));
        float4 l0 = __ldg(N + 2 * static_cast<int64_t>(id[0]) + 1);
        V3<float> D[8];
        D[0] = {0.f, 0.f, 0.f};
        bad |= h0.w != 0.f;
#pragma unroll
        for (int k = 1; k < 8; ++k) {
          float4 h = __ldg(N + 2 * static_cast<int64_t>(id[k]));
          float4 l = __ldg(N + 2 * static_cast<int64_t>(id[k]) + 1);
          bad |= h.w != 0.f;
          D[k].x = (h.x - h0.x) + (l.x - l0.x);
          D[k].y = (h.y - h0.y) + (l.y - l0.y);
          D[k].z = (h.z - h0.z) + (l.z - l0.z);
        }
        edges_from_nodes(D, a, b, gg);
        X = fmaxf(fabsf(h0.x), fmaxf(fabsf(h0.y), fabsf(h0.z)));
        epsK = 0x1p-43f * X;  // the lo parts are exact to 2^-46 |x|
      }
    }
    if (outcome < 0) {
      float L = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        L = fabsmax3(L, a[q]);
        L = fabsmax3(L, b[q]);
        L = fabsmax3(L, gg[q]);
      }
      // eps: SoA 2^-23 X + 2^-24 L;  indexed 13 * 2^-24 L + 2^-43 X
      float eps = INDEXED ? fmaf(13.f * 0x1p-24f, L, epsK) : fmaf(0x1p-24f, L, epsK);
      float L2 = L * L;
      float E = fmaf(256.f * eps, L2, 1024.f * 0x1p-24f * (L2 * L)) * 1.0001f;
      // too small (underflow) or too large (overflow) for the FP32 bound
      bad |= !(L >= 0x1p-30f) || !(E < 0x1p100f);
      if (bad) {
        outcome = 3;
      } else {
        Scaled<float> s;
        coefficients_from_edges(a, b, gg, s);
        int r = classify_root(s, keys_f(E));
        outcome = (r == 0 || r == 1) ? r : 3;
        minmax_f(s, lo, hi);
      }
    }
  }
  bool want_e = act && outcome == 3;
  unsigned int pos = warp_append(&S.cnt->esc_count, want_e);
  if (!act) return;
  if (want_e) {
    S.esc[pos] = i;  // capacity = batch size: cannot overflow
    return;
  }
  if (outcome == 5) {
    p.flags[g] = make_flag(kVUndecided, 0, 0);
    set_status(S.status, kSbIndex);
    double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (p.bmin) p.bmin[g] = nan;
    if (p.bmax) p.bmax[g] = nan;
    return;
  }
  p.flags[g] = make_flag(outcome == 0 ? kVInvalid : kVValid, 0, 0);
  if (p.bmin) p.bmin[g] = static_cast<double>(lo);
  if (p.bmax) p.bmax[g] = static_cast<double>(hi);
}

// FP64 node -> (hi, lo) FP32 pair on the integer pipe: hi = x truncated to 24
// significant bits (exact), lo = the next 23 bits of x - hi (so |hi + lo - x|
// <= 2^-46 |x|).  Record layout: float4 {hi.x, hi.y, hi.z, bad}, float4
// {lo.x, lo.y, lo.z, 0}; bad = 1 if a coordinate is outside [2^-103, 2^125)
// (zero allowed) or not finite.
__device__ __forceinline__ void split_int(double x, float& hi_f, float& lo_f, bool& bad) {
  long long bits = __double_as_longlong(x);
  uint32_t hi = static_cast<uint32_t>(bits >> 32), lo = static_cast<uint32_t>(bits);
  uint32_t e = (hi >> 20) & 0x7ffu;
  uint32_t sgn = hi & 0x80000000u;
  bool zero = ((hi << 1) | lo) == 0u;
  uint32_t f = __funnelshift_l(lo, hi, 3);
  f = ((f & 0x7fffffffu) ^ 0x40000000u) | sgn;
  // lo part: mantissa bits 28..6 of the low word, weight 2^(e-1069)
  uint32_t m = (lo >> 6) & 0x7fffffu;
  uint32_t ex = (e - 919u) << 23;
  float la = __uint_as_float(ex | m | sgn);
  float lb = __uint_as_float(ex | sgn);
  bad |= !zero && (e - 920u > 229u);  // e in [920, 1149]
  hi_f = zero ? 0.f : __uint_as_float(f);
  lo_f = zero ? 0.f : (la - lb);
}

__global__ void __launch_bounds__(256) nodes32_kernel(const double* nodes, int64_t n_nodes,
                                                      float4* out) {
  int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  bool bad = false;
  float hx, hy, hz, lx, ly, lz;
  split_int(__ldg(nodes + 3 * i), hx, lx, bad);
  split_int(__ldg(nodes + 3 * i + 1), hy, ly, bad);
  split_int(__ldg(nodes + 3 * i + 2), hz, lz, bad);
  out[2 * i] = make_float4(hx, hy, hz, bad ? 1.f : 0.f);
  out[2 * i + 1] = make_float4(lx, ly, lz, 0.f);
}

}  // namespace

cudaError_t launch_bulk64(const Batch& p, bool from_list, cudaStream_t st) {
  if (p.n <= 0) return cudaSuccess;
  unsigned int blocks = static_cast<unsigned int>((p.n + kBulkThreads - 1) / kBulkThreads);
  if (from_list)
    bulk64_kernel<true><<<blocks, kBulkThreads, 0, st>>>(p);
  else
    bulk64_kernel<false><<<blocks, kBulkThreads, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_bulk32(const Batch& p, cudaStream_t st) {
  if (p.n <= 0) return cudaSuccess;
  unsigned int blocks = static_cast<unsigned int>((p.n + kBulkThreads - 1) / kBulkThreads);
  if (p.indexed)
    bulk32_kernel<true><<<blocks, kBulkThreads, 0, st>>>(p);
  else
    bulk32_kernel<false><<<blocks, kBulkThreads, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_nodes32(const Batch& p, cudaStream_t st) {
  if (p.n_nodes <= 0) return cudaSuccess;
  unsigned int blocks = static_cast<unsigned int>((p.n_nodes + 255) / 256);
  nodes32_kernel<<<blocks, 256, 0, st>>>(p.nodes, p.n_nodes,
                                         reinterpret_cast<float4*>(p.s.node32));
  return cudaGetLastError();
}

}  // namespace hexval
