// Validity of linear quadrangles (Sec. 2.1): the Jacobian determinant of the
// bilinear map is bilinear, J = sum_k L_k J_k with J_k its value at corner k,
// so the element is valid iff all four corner values are positive.  With
// nodes 1..4 at (0,0), (1,0), (1,1), (0,1) and x_ij = x_j - x_i:
//   J(0,0) = x12 y14 - y12 x14        J(1,0) = x12 y23 - y12 x23
//   J(1,1) = x43 y23 - y43 x23        J(0,1) = x43 y14 - y43 x14
// (the corner of each value follows from the Jacobian matrix of Sec. 2.1;
// the two last products are printed against the opposite shape functions).
//
// One quadrangle per thread.  FP64 form: 8 differences and 4 products with
// a certified bound |J - J_exact| <= 2^-49 L^2 (L = the largest |edge
// component|, each product passes through <= 4 roundings of size 2^-53 L^2,
// and the bound is taken at the next power of two of L).  FP32 form:
// coordinates rounded to FP32 on the integer pipe, the same formulas with
// the bound of the rounded inputs; elements it cannot settle are redone in
// FP64 by the same thread.  A sign that FP64 cannot settle is computed
// exactly: the 8 coordinates are scaled to integers (as in the hexahedron's
// exact tier) and each J_k is a 256-bit integer (coordinate spans of at most
// 120 bits; wider spans give UNDECIDED and the range status).
#include "exact_warp.cuh"

namespace hexval {

namespace {

constexpr int kQuadThreads = 256;

struct Quad64 {
  double x[4], y[4];
};

// corner values in node order from the 8 differences
__device__ __forceinline__ void quad_corners(const double x[4], const double y[4], double J[4],
                                             double& L) {
  const double x12 = x[1] - x[0], y12 = y[1] - y[0], x43 = x[2] - x[3], y43 = y[2] - y[3];
  const double x14 = x[3] - x[0], y14 = y[3] - y[0], x23 = x[2] - x[1], y23 = y[2] - y[1];
  J[0] = fma(x12, y14, -(y12 * x14));
  J[1] = fma(x12, y23, -(y12 * x23));
  J[2] = fma(x43, y23, -(y43 * x23));
  J[3] = fma(x43, y14, -(y43 * x14));
  L = fmax(fmax(fmax(fabs(x12), fabs(y12)), fmax(fabs(x43), fabs(y43))),
           fmax(fmax(fabs(x14), fabs(y14)), fmax(fabs(x23), fabs(y23))));
}

__device__ __forceinline__ void quad_corners(const float x[4], const float y[4], float J[4],
                                             float& L) {
  const float x12 = x[1] - x[0], y12 = y[1] - y[0], x43 = x[2] - x[3], y43 = y[2] - y[3];
  const float x14 = x[3] - x[0], y14 = y[3] - y[0], x23 = x[2] - x[1], y23 = y[2] - y[1];
  J[0] = fmaf(x12, y14, -(y12 * x14));
  J[1] = fmaf(x12, y23, -(y12 * x23));
  J[2] = fmaf(x43, y23, -(y43 * x23));
  J[3] = fmaf(x43, y14, -(y43 * x14));
  L = fmaxf(fmaxf(fmaxf(fabsf(x12), fabsf(y12)), fmaxf(fabsf(x43), fabsf(y43))),
            fmaxf(fmaxf(fabsf(x14), fabsf(y14)), fmaxf(fabsf(x23), fabsf(y23))));
}

// Exact signs of the four corner values: bit k set if J_k > 0; -1 if the
// coordinate span exceeds 120 bits.
__device__ __noinline__ int quad_exact_positive(const Quad64& q) {
  unsigned long long M[8];
  int Q[8];
  bool neg[8];
  int qmin = 1 << 20, top = -(1 << 20);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const double v = c < 4 ? q.x[c] : q.y[c - 4];
    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
    const int ex = static_cast<int>((bits >> 52) & 0x7ff);
    unsigned long long m = bits & 0xfffffffffffffull;
    if (ex) m |= 1ull << 52;
    int qq = (ex ? ex : 1) - 1075;
    neg[c] = bits >> 63;
    if (m) {
      const int tz = __ffsll(static_cast<long long>(m)) - 1;
      m >>= tz;
      qq += tz;
      qmin = min(qmin, qq);
      top = max(top, qq + 63 - __clzll(static_cast<long long>(m)));
    }
    M[c] = m;
    Q[c] = qq;
  }
  const int B = top >= qmin ? top - qmin + 1 : 0;
  if (B > exact_tier::kFastBits) return -1;
  exact_tier::Wide<4> X[4], Y[4];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    exact_tier::Wide<4> w;
    const int sh = M[c] ? Q[c] - qmin : 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int lo = 32 * i - sh;
      unsigned long long t = 0;
      if (lo >= 0) t = lo < 64 ? (M[c] >> lo) : 0ull;
      else if (lo > -64) t = M[c] << (-lo);
      w.v[i] = static_cast<uint32_t>(t);
    }
    if (neg[c]) w = exact_tier::wneg(w);
    if (c < 4) X[c] = w; else Y[c - 4] = w;
  }
  using exact_tier::wmul;
  using exact_tier::wsub;
  const auto x12 = wsub(X[1], X[0]), y12 = wsub(Y[1], Y[0]), x43 = wsub(X[2], X[3]),
             y43 = wsub(Y[2], Y[3]), x14 = wsub(X[3], X[0]), y14 = wsub(Y[3], Y[0]),
             x23 = wsub(X[2], X[1]), y23 = wsub(Y[2], Y[1]);
  int pos = 0;
  pos |= exact_tier::wpositive(wsub(wmul(x12, y14), wmul(y12, x14))) ? 1 : 0;
  pos |= exact_tier::wpositive(wsub(wmul(x12, y23), wmul(y12, x23))) ? 2 : 0;
  pos |= exact_tier::wpositive(wsub(wmul(x43, y23), wmul(y43, x23))) ? 4 : 0;
  pos |= exact_tier::wpositive(wsub(wmul(x43, y14), wmul(y43, x14))) ? 8 : 0;
  return pos;
}

// FP64 decision of one quadrangle: writes flag, jmin, jmax.
__device__ __noinline__ void quad_fp64(const Quad64& q, const QuadBatch& p, int64_t g) {
  double J[4], L;
  quad_corners(q.x, q.y, J, L);
  bool finite = true;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    finite &= ((dhi(q.x[k]) & 0x7ff00000u) != 0x7ff00000u) &
              ((dhi(q.y[k]) & 0x7ff00000u) != 0x7ff00000u);
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  if (!finite) {
    p.flags[g] = make_flag(kVNonfinite, 0, 0);
    if (p.jmin) p.jmin[g] = qnan;
    if (p.jmax) p.jmax[g] = qnan;
    return;
  }
  // E = 2^(2 eL - 2093) >= 2^-49 L^2 with L < 2^(eL - 1022), and at least
  // 2^-1022 (covers the absolute error of underflowing products); with
  // L >= 2^500 a product may overflow: exact test
  const int eL = static_cast<int>(dhi(L) >> 20);
  const double E = pow2d(2 * eL - 2093);
  bool nonpos = false, unsure = eL >= 1023 + 500;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    nonpos |= J[k] <= -E;
    unsure |= !(J[k] > E) && !(J[k] <= -E);
  }
  uint8_t flag;
  if (nonpos) {
    flag = make_flag(kVInvalid, 0, 0);
  } else if (!unsure) {
    flag = make_flag(kVValid, 0, 0);
  } else {
    const int pos = quad_exact_positive(q);
    if (pos < 0) {
      set_status(p.status, kSbRange);
      flag = make_flag(kVUndecided, 0, 0);
    } else {
      flag = make_flag(pos == 15 ? kVValid : kVInvalid, 0, 1);
    }
  }
  p.flags[g] = flag;
  if (p.jmin) p.jmin[g] = fmin(fmin(J[0], J[1]), fmin(J[2], J[3]));
  if (p.jmax) p.jmax[g] = fmax(fmax(J[0], J[1]), fmax(J[2], J[3]));
}

__device__ __forceinline__ bool quad_load(const QuadBatch& p, int64_t g, Quad64& q) {
  if (!p.indexed) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      q.x[k] = __ldg(p.soa + (2 * k) * p.stride + g);
      q.y[k] = __ldg(p.soa + (2 * k + 1) * p.stride + g);
    }
    return true;
  }
  const int4 c = __ldg(reinterpret_cast<const int4*>(p.conn) + g);
  const int id[4] = {c.x, c.y, c.z, c.w};
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 4; ++k) ok &= static_cast<uint32_t>(id[k]) < static_cast<uint64_t>(p.n_nodes);
  if (!ok) return false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p.nodes) + id[k]);
    q.x[k] = v.x;
    q.y[k] = v.y;
  }
  return true;
}

__device__ __forceinline__ void quad_bad_index(const QuadBatch& p, int64_t g) {
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  p.flags[g] = make_flag(kVUndecided, 0, 0);
  if (p.jmin) p.jmin[g] = qnan;
  if (p.jmax) p.jmax[g] = qnan;
  set_status(p.status, kSbIndex);
}

__global__ void __launch_bounds__(kQuadThreads, 4) quad64_kernel(QuadBatch p) {
  const int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= p.n) return;
  Quad64 q;
  if (!quad_load(p, g, q)) {
    quad_bad_index(p, g);
    return;
  }
  quad_fp64(q, p, g);
}

// FP64 -> FP32 on the integer pipe as in the hexahedron's FP32 pass
// (|result - x| <= 2^-24 |x|; `bad` outside [2^-126, 2^125) or non-finite).
__device__ __forceinline__ float quad_d2f(double x, bool& bad) {
  long long bits = __double_as_longlong(x);
  uint32_t hi = static_cast<uint32_t>(bits >> 32), lo = static_cast<uint32_t>(bits);
  uint32_t e = (hi >> 20) & 0x7ffu;
  bool zero = ((hi << 1) | lo) == 0u;
  uint32_t f = __funnelshift_l(lo, hi, 3);
  f = (f & 0x7fffffffu) ^ 0x40000000u;
  f += (lo >> 28) & 1u;
  f |= hi & 0x80000000u;
  bad |= !zero && (e - 897u > 252u);
  return zero ? __uint_as_float(hi & 0x80000000u) : __uint_as_float(f);
}

__device__ __forceinline__ double quad_f2d(float v) {
  uint32_t b = __float_as_uint(v);
  uint32_t sgn = b & 0x80000000u;
  bool tiny = (b & 0x7f800000u) == 0u;
  uint32_t hi = tiny ? sgn : (sgn | (((b & 0x7fffffffu) >> 3) + (896u << 20)));
  uint32_t lo = tiny ? 0u : (b << 29);
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

// FP32 form.  Inputs within 2^-24 X of the FP64 values (X >= |coordinate|),
// so each computed difference is within eps = 2^-23 X + 2^-24 L of the
// exact one (L >= |computed difference|); a corner value is then within
// 4 eps (L + eps) + 2 eps^2 of its exact value from the inputs and within
// 4 u (L + eps)^2 (u = 2^-24) from its own roundings.
__device__ __forceinline__ void quad32_decide(const Quad64& q, const QuadBatch& p, int64_t g) {
  bool bad = false;
  float x[4], y[4], X = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    x[k] = quad_d2f(q.x[k], bad);
    y[k] = quad_d2f(q.y[k], bad);
    X = fmaxf(X, fmaxf(fabsf(x[k]), fabsf(y[k])));
  }
  float J[4], L;
  quad_corners(x, y, J, L);
  const float eps = fmaf(0x1p-24f, L, 0x1p-23f * X);
  const float Le = L + eps;
  const float E = fmaf(4.f * eps, Le, fmaf(2.f * eps, eps, 4.f * 0x1p-24f * Le * Le)) * 1.001f;
  bad |= !(L >= 0x1p-30f) || !(E < 0x1p100f);
  bool nonpos = false, unsure = bad;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    nonpos |= J[k] <= -E;
    unsure |= !(J[k] > E) && !(J[k] <= -E);
  }
  if (!bad && (nonpos || !unsure)) {
    p.flags[g] = make_flag(nonpos ? kVInvalid : kVValid, 0, 0);
    if (p.jmin) p.jmin[g] = quad_f2d(fminf(fminf(J[0], J[1]), fminf(J[2], J[3])));
    if (p.jmax) p.jmax[g] = quad_f2d(fmaxf(fmaxf(J[0], J[1]), fmaxf(J[2], J[3])));
    return;
  }
  quad_fp64(q, p, g);  // escalation
}

// Two quadrangles per thread, i and i + ceil(n/2), loaded before either is
// computed: twice the loads in flight per thread (the gather of the node
// coordinates is latency-bound).
__global__ void __launch_bounds__(kQuadThreads, 4) quad32_kernel(QuadBatch p) {
  const int64_t half = (p.n + 1) / 2;
  const int64_t g0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g0 >= half) return;
  const int64_t g1 = g0 + half;
  const bool two = g1 < p.n;
  Quad64 q0, q1;
  const bool ok0 = quad_load(p, g0, q0);
  const bool ok1 = two && quad_load(p, g1, q1);
  if (ok0) quad32_decide(q0, p, g0); else quad_bad_index(p, g0);
  if (two) {
    if (ok1) quad32_decide(q1, p, g1); else quad_bad_index(p, g1);
  }
}

}  // namespace

cudaError_t launch_quads(const QuadBatch& p, bool fp32, cudaStream_t st) {
  if (p.n <= 0) return cudaSuccess;
  if (fp32) {
    const int64_t half = (p.n + 1) / 2;
    quad32_kernel<<<static_cast<unsigned int>((half + kQuadThreads - 1) / kQuadThreads),
                    kQuadThreads, 0, st>>>(p);
  } else {
    quad64_kernel<<<static_cast<unsigned int>((p.n + kQuadThreads - 1) / kQuadThreads),
                    kQuadThreads, 0, st>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace hexval
