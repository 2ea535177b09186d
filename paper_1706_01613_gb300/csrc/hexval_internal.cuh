// Internal definitions shared by the CUDA translation units of libhexval.
//
// Method: Johnen, Weill & Remacle, "Robust and efficient validation of the
// linear hexahedral element" (IMR 2017).  Notation follows the paper: the
// element map x(xi) of Appendix A, J = det(x_xi, x_eta, x_zeta) (Eq. e:det3d),
// the 27 Bezier coefficients b of J (Sec. 3), the 20 sampled values that
// determine them (Sec. 4-5) and the decision algorithm of Sec. 6.
//
// Layout of the 27 coefficients on the device: tensor order t = i + 3j + 9k
// with (i, j, k) in {0,1,2}^3 the Bernstein indices along (xi, eta, zeta).
// Corners have i, j, k in {0, 2}.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hexval.h"

namespace hexval {

// ---------------------------------------------------------------- codes ----
constexpr int kVValid = HEXVAL_VALID;
constexpr int kVInvalid = HEXVAL_INVALID;
constexpr int kVUndecided = HEXVAL_UNDECIDED;
constexpr int kVNonfinite = HEXVAL_NONFINITE;

__host__ __device__ __forceinline__ uint8_t make_flag(int verdict, int depth, int exact) {
  return static_cast<uint8_t>(verdict | (depth << 3) | (exact << 7));
}

// per-refined-element state bits (slot_state)
constexpr uint32_t kStInvalid = 1u;   // a certified non-positive corner on the last level
constexpr uint32_t kStAmbig = 2u;     // an uncertifiable sign: exact tier needed
constexpr uint32_t kStCap = 4u;       // uncertified box at the depth cap
constexpr uint32_t kStOverflow = 8u;  // a child did not fit in the queue: exact tier
constexpr uint32_t kStXUsed = 16u;    // a box sign was settled exactly (flag bit 7)

// A refinement-queue entry whose slot id carries this bit is skipped (a box
// the exact check certified after it was queued).
constexpr uint32_t kDeadBox = 0x80000000u;
// Exact-check list entry without a queued box (child on the last level).
constexpr uint32_t kNoBox = 0xffffffffu;
// Entries of the exact-check list of a batch (boxes whose signs FP64 cannot
// settle, checked exactly one by one).
constexpr uint64_t kXbCap = 1u << 16;

// sticky device status bits
constexpr uint32_t kSbIndex = 1u;
constexpr uint32_t kSbQueue = 2u;
constexpr uint32_t kSbTimeout = 4u;
constexpr uint32_t kSbRange = 8u;

constexpr int kMaxDepth = 15;

// Per-batch counters.  They are zero when a batch starts: the tail kernel,
// which ends every batch, resets them once every block is done with them
// (and the handle creation zeroes them once).
struct Counters {
  unsigned int level_count[kMaxDepth + 2];  // boxes queued per level; [0] = refined elements
  unsigned int esc_count;                   // FP32 -> FP64 escalations (list + in-pass)
  unsigned int exact_count;                 // exact-tier list
  unsigned int arrive;                      // grid barrier of the tail kernel
  unsigned int done;                        // blocks of the tail kernel that finished
  unsigned int amb_count;                   // boxes that sent their element to the exact tier
  unsigned int r32_count;                   // FP32 form: elements refined in FP32 (list r32)
  unsigned int esc2_count;                  // FP32 refinement -> FP64 escalations (list esc2)
  unsigned int level32_count[kMaxDepth + 2];  // FP32 boxes queued per level
  unsigned int minj_next;                   // element counter of the minimum-of-J kernel
  unsigned int iw_count;                    // in-warp refinement workspaces taken
  unsigned int iw_done;                     // elements decided by the in-warp refinement
  unsigned int esc3_count;                  // double-float or partial FP64 redo -> tail (esc3)
  unsigned int df_count;                    // decided by the double-float redo
  unsigned int xb_count;                    // exact-check list (boxes)
  unsigned int l1_count;                    // elements the first-level kernel split
  unsigned int r32b_count;                  // of those, left undecided (list r32b)
  unsigned int split64;                     // FP64 boxes split by the refinement
  unsigned int split32;                     // FP32 boxes split by the refinement
  unsigned int part_count;                  // escalations the partial FP64 redo decided
};

// Escalations of the FP32 pass: the first Batch::esc_in_pass elements
// appended to the escalation list of a batch are redone in FP64 by the FP32
// pass itself (one element at a time by a whole warp, on the FP64 unit that
// the FP32 pass leaves idle); their list entries stay unwritten.  Entries
// from esc_in_pass on are written and redone by the tail kernel.  Of the
// elements the FP32 pass finds to need subdivision, the first
// Batch::r32_in_pass are redone in FP64 by the pass itself (and refined in
// FP64: for a handful of elements that is cheaper than the FP32 refinement's
// own steps), the others are refined in FP32 by the tail kernel (phase R).
// Defaults of the configuration:
constexpr unsigned int kEscInPassDefault = 4096;
constexpr unsigned int kR32InPassDefault = 512;
constexpr unsigned int kWarpItemsDefault = 8;

// In-warp FP64 refinement (warp_items.cuh): workspaces per batch and boxes
// per level of one workspace.
constexpr unsigned int kIwSlots = 64;
constexpr unsigned int kIwBoxes = 64;

// Counters accumulated across calls (hexval_get_stats).
struct Stats {
  unsigned long long elements, escalated_fp64, refined, boxes, exact, max_level_boxes,
      escalated_df, boxes_fp32, redone_tail, partial_fp64;
};

// Device scratch owned by a handle.
struct Scratch {
  // refinement queue: two level buffers, SoA [27][cap] coefficients + slot ids
  // + box positions (x | y << 16 | z << 32 on the dyadic grid of the level;
  // optional: without them every uncertain sign goes to the full exact tier)
  double* qcoef[2];
  uint32_t* qslot[2];
  uint64_t* qpos[2];
  uint64_t qcap;
  // exact-check list: slot, queue position of the box in the next level (or
  // kNoBox), box position; capacity xb_cap (0: no exact check)
  uint32_t* xb_slot;
  uint32_t* xb_qi;
  uint64_t* xb_pos;
  uint64_t xb_cap;
  // per refined element ("slot"), indexed by its position in level 0
  uint32_t* slot_elem;
  uint32_t* slot_state;
  uint32_t* slot_lev;
  double* slot_e0;  // error bound of the depth-0 coefficients
  double* slot_m0;  // bound on |coefficient| of every box of the element
  // FP32 -> FP64 escalation list (element ids of the batch)
  uint32_t* esc;
  // exact tier
  uint32_t* exact_list;
  uint64_t exact_cap;
  uint32_t* exact_work;  // per-worker stacks (exact.cuh)
  uint64_t exact_work_words;
  // FP32 copies of the nodes for the indexed path: hi, lo (x, y, z each)
  float* node32;
  uint64_t max_nodes;
  Counters* cnt;
  Stats* stats;
  uint32_t* status;
  // prefix sums of the compaction tiles (compact.cu)
  uint64_t* tiles;
  uint64_t tiles_cap;
  // FP32 form: refinement in FP32 (tail.cu, phase R) of the elements listed
  // in r32, with its own box queue and per-element state; elements it cannot
  // settle are listed in esc2 for the FP64 redo
  uint32_t* r32;
  uint32_t* esc2;
  float* q32coef[2];
  uint32_t* q32slot[2];
  uint64_t q32cap;
  uint32_t* s32_elem;
  uint32_t* s32_state;
  uint32_t* s32_lev;
  float* s32_e0;
  float* s32_m0;
  // FP32 form: workspaces of the in-warp FP64 refinement (warp_items.cuh)
  double* iw;
  // FP32 form: elements the double-float redo (redo_df.cu) or the partial
  // FP64 redo (redo_partial.cu) leaves to the full FP64 redo
  uint32_t* esc3;
  // FP32 form: elements the first-level kernel leaves to the tail (level1.cu)
  uint32_t* r32b;
};

// One batch of elements, as seen by every kernel.
struct Batch {
  int64_t n;       // elements in the batch
  int64_t base;    // index of its first element in the caller's arrays
  // SoA input (24 planes with stride `stride`) or indexed input
  const double* soa;
  int64_t stride;
  const double* nodes;
  int64_t n_nodes;
  const int32_t* conn;
  int indexed;
  int pair32;        // FP32 pass: two elements per thread with packed f32x2 math
  int bulk_threads;  // block size of the bulk kernels (0: default)
  int prefetch32;    // indexed FP32 pass on a persistent grid with prefetch
  int dfredo;        // FP32 form: escalations redone in double-float first
  int level1;        // FP32 form: first refinement level in a kernel of its own
  int partial64;     // FP32 form: escalations first redone only in their unsettled signs
  unsigned int esc_in_pass;  // FP32 escalations of a batch redone in FP64 by the FP32 pass
  unsigned int r32_in_pass;  // elements to refine redone in FP64 by the FP32 pass
  unsigned int warp_items;   // tail: warp-per-item steps up to this many items per warp
  // outputs (indexed by base + e)
  uint8_t* flags;
  double* bmin;
  double* bmax;
  int max_depth;
  Scratch s;
};

// ------------------------------------------------------ small utilities ----
template <typename T>
struct V3 {
  T x, y, z;
};

template <typename T>
__device__ __forceinline__ V3<T> vsub(const V3<T>& a, const V3<T>& b) {
  return {a.x - b.x, a.y - b.y, a.z - b.z};
}
template <typename T>
__device__ __forceinline__ V3<T> vadd(const V3<T>& a, const V3<T>& b) {
  return {a.x + b.x, a.y + b.y, a.z + b.z};
}

// det(A, B, C) = A . (B x C); every product term passes through at most 5
// roundings (2 in the cross product, 3 in the dot product).
__device__ __forceinline__ double det3(const V3<double>& A, const V3<double>& B,
                                       const V3<double>& C) {
  double cx = fma(B.y, C.z, -(B.z * C.y));
  double cy = fma(B.z, C.x, -(B.x * C.z));
  double cz = fma(B.x, C.y, -(B.y * C.x));
  return fma(A.z, cz, fma(A.y, cy, A.x * cx));
}
__device__ __forceinline__ float det3(const V3<float>& A, const V3<float>& B,
                                      const V3<float>& C) {
  float cx = fmaf(B.y, C.z, -(B.z * C.y));
  float cy = fmaf(B.z, C.x, -(B.x * C.z));
  float cz = fmaf(B.x, C.y, -(B.y * C.x));
  return fmaf(A.z, cz, fmaf(A.y, cy, A.x * cx));
}

// A pair of FP32 values, one per element of a pair processed by one thread,
// computed with the packed f32x2 instructions of sm_100+ (one instruction for
// both lanes: half the issue slots of scalar FP32 at the same FLOP rate).
// Every operation rounds each lane exactly as its scalar counterpart.
struct F2 {
  float2 v;
  __device__ __forceinline__ F2() {}
  __device__ __forceinline__ explicit F2(float c) : v(make_float2(c, c)) {}
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
  F2 r;
  r.v = __fadd2_rn(a.v, b.v);
  return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
  F2 r;
  r.v = __fmul2_rn(a.v, b.v);
  return r;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  unsigned long long x = *reinterpret_cast<unsigned long long*>(&a.v);
  unsigned long long y = *reinterpret_cast<unsigned long long*>(&b.v), z;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
  F2 r;
  r.v = *reinterpret_cast<float2*>(&z);
  return r;
}
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) {
  F2 r;
  r.v = __ffma2_rn(a.v, b.v, c.v);
  return r;
}
using ::fma;  // keep the FP64 / FP32 overloads visible next to the F2 one
// det(A, B, C) for two elements: cross product with separate products and a
// subtraction (2 roundings per term, as the scalar FMA form), then the dot
// product (3 roundings).
__device__ __forceinline__ F2 det3(const V3<F2>& A, const V3<F2>& B, const V3<F2>& C) {
  F2 cx = B.y * C.z - B.z * C.y;
  F2 cy = B.z * C.x - B.x * C.z;
  F2 cz = B.x * C.y - B.y * C.x;
  return fma(A.z, cz, fma(A.y, cy, A.x * cx));
}

// Node k (Appendix A order) at the reference corner (xi, eta, zeta) in {0,1}^3.
__host__ __device__ constexpr int node_at(int xi, int eta, int zeta) {
  return (eta ? (xi ? 2 : 3) : (xi ? 1 : 0)) + 4 * zeta;
}

// Tensor index of Bernstein indices (i, j, k).
__host__ __device__ constexpr int tix(int i, int j, int k) { return i + 3 * j + 9 * k; }

// ------------------------------------------- the 27 coefficients of J ------
// Edge vectors of the trilinear map (Sec. 5):
//   a[eta + 2 zeta]  = x(1,eta,zeta) - x(0,eta,zeta)   (edges along xi)
//   b[xi + 2 zeta]   = x(xi,1,zeta) - x(xi,0,zeta)     (edges along eta)
//   g[xi + 2 eta]    = x(xi,eta,1) - x(xi,eta,0)       (edges along zeta)
// so x_xi(xi,eta,zeta) is the bilinear blend of the a's over (eta, zeta), etc.
// At a corner J = det(a, b, g) of the three edges meeting there (the corner
// tetrahedra of Sec. 5); at an edge midpoint two columns are averages of two
// parallel edges: J = det(a, (b0+b1)/2, (g0+g1)/2) for the xi-edge at
// eta = zeta = 0, the value the paper writes as the volume of the tetrahedron
// (n1, n2, m34, m56).  The kernels evaluate C = 4 J there with the sums.
//
// With the 20 samples the coefficients follow Table t:Tsmall; scaled to
// avoid multiplications (the scale of each class is exact):
//   corner:  b          = c
//   edge:    2 b_e      = C_e - c_a - c_b            (a, b: end corners)
//   face:    4 b_f      = sum_4 C_e - 3 sum_4 c       (its edges / corners)
//   centre:  8 b_c      = sum_12 C_e - 5 sum_8 c
template <typename T>
struct Scaled {
  T corner[8];  // index = node id (Appendix A order)
  T edge[12];   // 2 b: xi-edges (eta,zeta)=(0,0),(1,0),(0,1),(1,1); eta-edges
                // (xi,zeta) same order; zeta-edges (xi,eta) same order
  T face[6];    // 4 b: zeta=0, zeta=1, eta=0, eta=1, xi=0, xi=1
  T centre;     // 8 b
  T edgeC[12];  // the 12 samples C = 4 J at the edge midpoints
};

// Tensor index of each scaled entry (used when the coefficients are stored).
__host__ __device__ constexpr int corner_t(int k) {
  // node k -> (xi, eta, zeta)
  return tix((k == 1 || k == 2 || k == 5 || k == 6) ? 2 : 0,
             (k == 2 || k == 3 || k == 6 || k == 7) ? 2 : 0, k >= 4 ? 2 : 0);
}
__host__ __device__ constexpr int edge_t(int e) {
  return e < 4 ? tix(1, 2 * (e & 1), 2 * (e >> 1))
               : (e < 8 ? tix(2 * (e & 1), 1, 2 * ((e - 4) >> 1))
                        : tix(2 * (e & 1), 2 * ((e - 8) >> 1), 1));
}
__host__ __device__ constexpr int face_t(int f) {
  return f == 0 ? tix(1, 1, 0)
                : f == 1 ? tix(1, 1, 2)
                         : f == 2 ? tix(1, 0, 1)
                                  : f == 3 ? tix(1, 2, 1) : f == 4 ? tix(0, 1, 1) : tix(2, 1, 1);
}

// Computes the scaled coefficients from the 12 edge vectors.
template <typename T>
__device__ __forceinline__ void coefficients_from_edges(const V3<T> a[4], const V3<T> b[4],
                                                        const V3<T> g[4], Scaled<T>& s) {
  // corners
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y)
#pragma unroll
      for (int x = 0; x < 2; ++x)
        s.corner[node_at(x, y, z)] = det3(a[y + 2 * z], b[x + 2 * z], g[x + 2 * y]);
  // sums of parallel edges (x2 the averaged columns)
  V3<T> sb[2], sg[2], sa[2], sg2[2], sa2[2], sb2[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    sb[u] = vadd(b[0 + 2 * u], b[1 + 2 * u]);   // xi-edges at zeta = u: x_eta
    sg[u] = vadd(g[0 + 2 * u], g[1 + 2 * u]);   // xi-edges at eta = u:  x_zeta
    sa[u] = vadd(a[0 + 2 * u], a[1 + 2 * u]);   // eta-edges at zeta = u: x_xi
    sg2[u] = vadd(g[u], g[u + 2]);              // eta-edges at xi = u:   x_zeta
    sa2[u] = vadd(a[u], a[u + 2]);              // zeta-edges at eta = u: x_xi
    sb2[u] = vadd(b[u], b[u + 2]);              // zeta-edges at xi = u:  x_eta
  }
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y) s.edgeC[y + 2 * z] = det3(a[y + 2 * z], sb[z], sg[y]);
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) s.edgeC[4 + x + 2 * z] = det3(sa[z], b[x + 2 * z], sg2[x]);
#pragma unroll
  for (int y = 0; y < 2; ++y)
#pragma unroll
    for (int x = 0; x < 2; ++x) s.edgeC[8 + x + 2 * y] = det3(sa2[y], sb2[x], g[x + 2 * y]);
  // Table t:Tsmall, scaled
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y)
      s.edge[y + 2 * z] =
          s.edgeC[y + 2 * z] - s.corner[node_at(0, y, z)] - s.corner[node_at(1, y, z)];
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x)
      s.edge[4 + x + 2 * z] =
          s.edgeC[4 + x + 2 * z] - s.corner[node_at(x, 0, z)] - s.corner[node_at(x, 1, z)];
#pragma unroll
  for (int y = 0; y < 2; ++y)
#pragma unroll
    for (int x = 0; x < 2; ++x)
      s.edge[8 + x + 2 * y] =
          s.edgeC[8 + x + 2 * y] - s.corner[node_at(x, y, 0)] - s.corner[node_at(x, y, 1)];
  // faces: zeta = u (xi-edges at zeta=u, eta-edges at zeta=u)
  T cz[2], cy[2], cx[2];  // corner sums per face
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    cz[u] = (s.corner[node_at(0, 0, u)] + s.corner[node_at(1, 0, u)]) +
            (s.corner[node_at(0, 1, u)] + s.corner[node_at(1, 1, u)]);
    cy[u] = (s.corner[node_at(0, u, 0)] + s.corner[node_at(1, u, 0)]) +
            (s.corner[node_at(0, u, 1)] + s.corner[node_at(1, u, 1)]);
    cx[u] = (s.corner[node_at(u, 0, 0)] + s.corner[node_at(u, 1, 0)]) +
            (s.corner[node_at(u, 0, 1)] + s.corner[node_at(u, 1, 1)]);
  }
  T ez[2], ey[2], ex[2];  // edge-sample sums per face
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    ez[u] = (s.edgeC[0 + 2 * u] + s.edgeC[1 + 2 * u]) + (s.edgeC[4 + 2 * u] + s.edgeC[5 + 2 * u]);
    ey[u] = (s.edgeC[u] + s.edgeC[u + 2]) + (s.edgeC[8 + 2 * u] + s.edgeC[9 + 2 * u]);
    ex[u] = (s.edgeC[4 + u] + s.edgeC[6 + u]) + (s.edgeC[8 + u] + s.edgeC[10 + u]);
  }
  const T m3 = T(-3), m5 = T(-5);
  s.face[0] = fma(m3, cz[0], ez[0]);
  s.face[1] = fma(m3, cz[1], ez[1]);
  s.face[2] = fma(m3, cy[0], ey[0]);
  s.face[3] = fma(m3, cy[1], ey[1]);
  s.face[4] = fma(m3, cx[0], ex[0]);
  s.face[5] = fma(m3, cx[1], ex[1]);
  // centre: all 12 samples and all 8 corners
  T esum = (ez[0] + ez[1]) + ((s.edgeC[8] + s.edgeC[9]) + (s.edgeC[10] + s.edgeC[11]));
  T csum = cz[0] + cz[1];
  s.centre = fma(m5, csum, esum);
}

// Unscaled coefficient in tensor order from the scaled classes.
template <typename T>
__device__ __forceinline__ void store_tensor(const Scaled<T>& s, T out[27]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) out[corner_t(k)] = s.corner[k];
#pragma unroll
  for (int e = 0; e < 12; ++e) out[edge_t(e)] = s.edge[e] * T(0.5);
#pragma unroll
  for (int f = 0; f < 6; ++f) out[face_t(f)] = s.face[f] * T(0.25);
  out[tix(1, 1, 1)] = s.centre * T(0.125);
}

// ------------------------------------------- integer-pipe classification ----
// Magnitude / sign tests on the bit patterns keep comparisons off the FP64
// pipe.  For an IEEE double v: hi = top 32 bits.  |v| > E certainly holds if
// (hi & 0x7fffffff) > hi(E) with E a power of two (its low word is zero):
// the test is conservative by at most one part in 2^20.
__device__ __forceinline__ uint32_t dhi(double v) {
  return static_cast<uint32_t>(__double_as_longlong(v) >> 32);
}
__device__ __forceinline__ uint32_t fbits(float v) { return __float_as_uint(v); }

// Certified classes of a value with error bound E (E passed as its magnitude
// key): 0 certainly <= 0, 1 certainly > 0, 2 ambiguous.
struct Sign3 {
  bool nonpos;  // certainly <= 0
  bool pos;     // certainly > 0
};
__device__ __forceinline__ Sign3 sign_d(double v, uint32_t ekey) {
  uint32_t h = dhi(v);
  bool big = (h & 0x7fffffffu) > ekey;
  return {big && (h >> 31), big && !(h >> 31)};
}
__device__ __forceinline__ Sign3 sign_f(float v, uint32_t ekey) {
  uint32_t h = fbits(v);
  bool big = (h & 0x7fffffffu) > ekey;
  return {big && (h >> 31), big && !(h >> 31)};
}

// Order-preserving integer key of a double (for exact min / max on the
// integer pipe).
__device__ __forceinline__ long long dkey(double v) {
  long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dunkey(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

// Power of two 2^p as a double built from its exponent (clamped to the
// normal range).
__device__ __forceinline__ double pow2d(int p) {
  int e = p + 1023;
  e = e < 1 ? 1 : (e > 2046 ? 2046 : e);
  return __longlong_as_double(static_cast<long long>(e) << 52);
}
__device__ __forceinline__ float pow2f(int p) {
  int e = p + 127;
  e = e < 1 ? 1 : (e > 254 ? 254 : e);
  return __uint_as_float(static_cast<uint32_t>(e) << 23);
}

// ------------------------------------------------ unscaled box splitting ----
// The quadratic de Casteljau split of a row (p0, p1, p2) at 1/2 is
// (p0, s/2, (s+t)/4, t/2, p2) with s = p0 + p1, t = p1 + p2 (Sec. 6).  The
// refinement computes it unscaled, (p0, s, s+t, t, p2): entry x carries the
// factor 2^c(x), c = (0, 1, 2, 1, 0), and costs 3 additions per row instead
// of 6 operations.  The scalings being exact, every unscaled entry is exactly
// 2^c times the halved one (no overflow: |p| <= M keeps every entry of a
// box's three passes within 64 M).  After the three passes entry
// (x, y, z) of the 5x5x5 grid carries 2^(c(x)+c(y)+c(z)).  The FP64
// refinement takes the factor into its sign tests (sign_d_split) and removes
// it from the children it stores by exponent arithmetic (down2): no FP64
// instruction for either.  The FP32 refinement multiplies the 125 values by
// 2^-m (split_box32, refine32.cuh): FP32 multiplies are cheap, and the
// child classification then needs only two minima per child.
__host__ __device__ constexpr int split_exp(int x) { return x < 2 ? x : 4 - x; }
__host__ __device__ constexpr int split_exp3(int x, int y, int z) {
  return split_exp(x) + split_exp(y) + split_exp(z);
}

// sign_d of the value 2^-m v against the key of E, v carrying the factor
// 2^m: the magnitude's exponent field less m, compared as a signed integer
// (a magnitude below 2^m is never certain).  The same test as
// sign_d(2^-m v, key) for a normal 2^-m v; for a subnormal one it is as
// conservative (its magnitude is below every normal E).  Needs key + (m <<
// 20) < 2^31, which the range of M0 the split runs in (split_range_ok,
// E <= M0) guarantees.
__device__ __forceinline__ Sign3 sign_d_split(double v, uint32_t ekey, int m) {
  const uint32_t h = dhi(v);
  const bool big = static_cast<int>((h & 0x7fffffffu) - (static_cast<uint32_t>(m) << 20)) >
                   static_cast<int>(ekey);
  return {big && (h >> 31), big && !(h >> 31)};
}

// 2^-m u for 0 <= m <= 6 by exponent arithmetic on the integer pipe: exact
// when the result is normal; a result below the normal range becomes a zero
// of u's sign (absolute error < 2^-1022).
__device__ __forceinline__ double down2(double u, int m) {
  const long long b = __double_as_longlong(u);
  const uint32_t e = (static_cast<uint32_t>(b >> 32) >> 20) & 0x7ffu;
  return __longlong_as_double(e > static_cast<uint32_t>(m) ? b - (static_cast<long long>(m) << 52)
                                                           : b & (1LL << 63));
}

// Range of the root magnitude bound M0 in which the unscaled split runs; a
// box of an element outside it is left to the next tier.  Above: 64 M0 stays
// finite.  Below: the per-level bound d 2^-49 M0 (FP32: d 2^-20 M0) allows
// 16 roundings of u M0 per level where a split makes at most 6, and the
// other 10 u M0 cover the flush of down2 (2^-1022 <= 2^-62 M0 for M0 >=
// 2^-960; 2^-126 <= 2^-26 M0 for M0 >= 2^-100).
constexpr double kSplitMaxM0 = 0x1p1000;
constexpr double kSplitMinM0 = 0x1p-960;
constexpr float kSplitMaxM0f = 0x1p120f;
constexpr float kSplitMinM0f = 0x1p-100f;

// M0 within that range (integer compares of the bit patterns, M0 >= 0)
__device__ __forceinline__ bool split_range_ok(double m0) {
  const uint32_t h = static_cast<uint32_t>(__double_as_longlong(m0) >> 32);
  return h >= static_cast<uint32_t>(__double_as_longlong(kSplitMinM0) >> 32) &&
         h < static_cast<uint32_t>(__double_as_longlong(kSplitMaxM0) >> 32);
}
__device__ __forceinline__ bool split_range_ok(float m0) {
  const uint32_t b = __float_as_uint(m0);
  return b >= __float_as_uint(kSplitMinM0f) && b < __float_as_uint(kSplitMaxM0f);
}

// Biased exponent of the largest |component| among the 12 edge vectors
// (integer max over the high words).
__device__ __forceinline__ int max_exponent_d(const V3<double> a[4], const V3<double> b[4],
                                              const V3<double> g[4]) {
  uint32_t m = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    m = max(m, dhi(a[q].x) & 0x7fffffffu);
    m = max(m, dhi(a[q].y) & 0x7fffffffu);
    m = max(m, dhi(a[q].z) & 0x7fffffffu);
    m = max(m, dhi(b[q].x) & 0x7fffffffu);
    m = max(m, dhi(b[q].y) & 0x7fffffffu);
    m = max(m, dhi(b[q].z) & 0x7fffffffu);
    m = max(m, dhi(g[q].x) & 0x7fffffffu);
    m = max(m, dhi(g[q].y) & 0x7fffffffu);
    m = max(m, dhi(g[q].z) & 0x7fffffffu);
  }
  return static_cast<int>(m >> 20);
}

// ------------------------------------------------------- warp helpers ------
// Warp-aggregated append: every lane calls it (pred may be false); returns
// the lane's position in the list (valid when pred is true).
__device__ __forceinline__ unsigned int warp_append(unsigned int* counter, bool pred) {
  unsigned int mask = __ballot_sync(0xffffffffu, pred);
  unsigned int lane = threadIdx.x & 31u;
  unsigned int base = 0;
  if (mask) {
    int leader = __ffs(mask) - 1;
    if (static_cast<int>(lane) == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
  }
  return base + __popc(mask & ((1u << lane) - 1u));
}

__device__ __forceinline__ void set_status(uint32_t* status, uint32_t bit) {
  atomicOr(status, bit);
}

// Loads that bypass the (non-coherent) L1: data written by other blocks of
// the same launch.
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

// Default budget (polls of the arrival counter, each an L2 round trip: well
// over a second in all) of the tail kernel's bounded grid barrier (tail.cu).
constexpr long long kSpinLimit = 1ll << 24;

// ---------------------------------------------------- element loading ------
// Loads the 8 nodes (24 coordinates) of element g of the batch.  Returns
// false (and sets the status) when a connectivity entry is out of range.
__device__ __forceinline__ bool load_element(const Batch& p, int64_t g, V3<double> X[8]) {
  if (!p.indexed) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      X[k].x = __ldg(p.soa + (3 * k + 0) * p.stride + g);
      X[k].y = __ldg(p.soa + (3 * k + 1) * p.stride + g);
      X[k].z = __ldg(p.soa + (3 * k + 2) * p.stride + g);
    }
    return true;
  }
  const int4* c4 = reinterpret_cast<const int4*>(p.conn + 8 * g);
  int4 c0 = __ldg(c4), c1 = __ldg(c4 + 1);
  int id[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 8; ++k) ok &= (id[k] >= 0) & (static_cast<int64_t>(id[k]) < p.n_nodes);
  if (!ok) return false;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double* q = p.nodes + 3 * static_cast<int64_t>(id[k]);
    X[k].x = __ldg(q);
    X[k].y = __ldg(q + 1);
    X[k].z = __ldg(q + 2);
  }
  return true;
}

// Edge vectors from the nodes (see coefficients_from_edges).
template <typename T>
__device__ __forceinline__ void edges_from_nodes(const V3<T> X[8], V3<T> a[4], V3<T> b[4],
                                                 V3<T> g[4]) {
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y) a[y + 2 * z] = vsub(X[node_at(1, y, z)], X[node_at(0, y, z)]);
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) b[x + 2 * z] = vsub(X[node_at(x, 1, z)], X[node_at(x, 0, z)]);
#pragma unroll
  for (int y = 0; y < 2; ++y)
#pragma unroll
    for (int x = 0; x < 2; ++x) g[x + 2 * y] = vsub(X[node_at(x, y, 1)], X[node_at(x, y, 0)]);
}

// A batch of linear quadrangles (Sec. 2.1).
struct QuadBatch {
  int64_t n;
  const double* soa;  // [4][2][stride] planes, or
  int64_t stride;
  const double* nodes;  // [n_nodes][2] (16-byte aligned) with
  int64_t n_nodes;
  const int32_t* conn;  // [n][4] (16-byte aligned)
  int indexed;
  uint8_t* flags;
  double* jmin;
  double* jmax;
  uint32_t* status;
};

// ------------------------------------------------------------- launches ----
// Host-side launchers (defined in the .cu files).
cudaError_t launch_bulk64(const Batch& p, cudaStream_t st);
cudaError_t launch_bulk32(const Batch& p, cudaStream_t st);
cudaError_t launch_nodes32(const Batch& p, cudaStream_t st);
cudaError_t launch_tail(const Batch& p, bool from_list, cudaStream_t st);

// Programmatic dependent launch: a kernel launched with launch_pdl may begin
// (its blocks become resident) while the kernel before it in the stream
// finishes; it calls pdl_wait before touching anything, which returns once
// that kernel has completed and its writes are visible.  pdl_trigger lets
// the next kernel begin launching.  Both are no-ops in a normal launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned int grid, unsigned int block,
                              size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
// FP32 form with HEXVAL_OPT_DFREDO: double-float redo of the escalations
// the FP32 pass leaves (between the bulk and tail kernels).
cudaError_t launch_redo_df(const Batch& p, cudaStream_t st);
// FP32 form with HEXVAL_OPT_PARTIAL64: FP64 redo of the unsettled signs of
// the escalations the FP32 pass leaves (between the bulk and tail kernels).
cudaError_t launch_redo_partial(const Batch& p, cudaStream_t st);
// FP32 form with HEXVAL_OPT_LEVEL1: the first refinement level of the
// elements the FP32 pass lists for the FP32 refinement (before the tail).
cudaError_t launch_level1(const Batch& p, cudaStream_t st);
cudaError_t launch_quads(const QuadBatch& p, bool fp32, cudaStream_t st);
cudaError_t launch_quality(const Batch& p, float* sj, cudaStream_t st);
cudaError_t launch_minj(const Batch& p, double rel_tol, int max_depth, double* lo, double* hi,
                        uint8_t* depth, unsigned int* counter, cudaStream_t st);
int64_t compact_tiles(int64_t n);
cudaError_t launch_compact(const uint8_t* flags, int64_t n, uint32_t mask, uint64_t* tiles,
                           int32_t* ids, int32_t* count, cudaStream_t st);
uint64_t exact_work_words();

}  // namespace hexval
