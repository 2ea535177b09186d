// Corner scaled Jacobian of linear hexahedra: the quality measure quoted in
// Sec. 7 (Fig. f:invalidHighCornerQual) -- at each corner, the determinant of
// the three edge vectors leaving it (the columns of the Jacobian matrix
// there, Eq. e:det3d), each divided by its length; the element value is the
// minimum over the 8 corners (0 at a corner with a zero-length edge).
//
// One element per thread, with no FP64 arithmetic (the FP64 unit of this
// GPU is slow enough that 21 FP64 subtractions per element would bound the
// kernel): each of the element's 24 coordinates becomes the 64-bit integer
// x 2^(1084 - E), E the largest biased exponent among them (magnitudes below
// 2^62; exact for coordinates within 2^9 of the largest in magnitude, short
// of it by less than 2^-61 of the largest otherwise); the differences to
// node 1 are then exact integers.  They are normalised together by one
// shift (the largest gets its top bit at bit 62), and the top 32 bits of
// each are rounded to FP32 and scaled by 2^-30 (|result| <= 2; the measure
// is scale invariant): a relative error of 2^-24 of the value and 2^-30 of
// the largest, independently of where the element sits.  Edge vectors,
// corner determinants and norms are FP32.
#include "hexval_internal.cuh"

namespace hexval {

namespace {

constexpr int kQualityThreads = 256;

// x 2^(1084 - E) as an integer (E >= the biased exponent of x): the 53-bit
// significand shifted left by 9 and right by E - e, with the sign of x.
// Zeros give 0; FP64 subnormals keep their significand without its scale
// (values far below every normal coordinate); bits below 2^(E - 1084) are
// dropped.
__device__ __forceinline__ long long fixed_of(double x, uint32_t E) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const uint32_t e = static_cast<uint32_t>(b >> 52) & 0x7ffu;
  unsigned long long m = (b & 0x000fffffffffffffull) | (e ? (1ull << 52) : 0ull);
  m = (m << 9) >> min(E - e, 63u);
  const long long s = static_cast<long long>(b) >> 63;  // 0 or -1
  return (static_cast<long long>(m) ^ s) - s;
}

// Node `id` of a 16-byte aligned node array: one 16-byte and one 8-byte load
// (an even node starts on a 16-byte boundary, an odd one 8 bytes past it).
__device__ __forceinline__ V3<double> load_node_aligned(const double* nodes, int64_t id) {
  const double* q = nodes + 3 * id;
  const int odd = static_cast<int>(id & 1);
  const double2 v = __ldg(reinterpret_cast<const double2*>(q + odd));
  const double w = __ldg(q + (odd ? 0 : 2));
  return odd ? V3<double>{w, v.x, v.y} : V3<double>{v.x, v.y, w};
}

// 1 / |v|; squared norms that would underflow are formed after scaling by 2^60
__device__ __forceinline__ float inv_norm(const V3<float>& v) {
  const float n2 = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z));
  if (n2 >= 0x1p-100f) return rsqrtf(n2);
  const V3<float> w{v.x * 0x1p60f, v.y * 0x1p60f, v.z * 0x1p60f};
  return rsqrtf(fmaf(w.x, w.x, fmaf(w.y, w.y, w.z * w.z))) * 0x1p60f;
}

template <bool ALIGNED>
__global__ void __launch_bounds__(kQualityThreads) quality_kernel(Batch p, float* sj) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  const int64_t g = p.base + i;
  V3<double> X[8];
  bool ok = true;
  if (ALIGNED) {  // indexed, nodes 16-byte aligned
    const int4* c4 = reinterpret_cast<const int4*>(p.conn + 8 * g);
    const int4 c0 = __ldg(c4), c1 = __ldg(c4 + 1);
    const int id[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
    for (int k = 0; k < 8; ++k) ok &= (id[k] >= 0) & (static_cast<int64_t>(id[k]) < p.n_nodes);
    if (ok) {
#pragma unroll
      for (int k = 0; k < 8; ++k) X[k] = load_node_aligned(p.nodes, id[k]);
    }
  } else {
    ok = load_element(p, g, X);
  }
  if (!ok) {
    sj[g] = __int_as_float(0x7fc00000);
    set_status(p.s.status, kSbIndex);
    return;
  }
  // the largest biased exponent; NaN / infinite coordinates give NaN
  uint32_t E = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    E = max(E, max(dhi(X[k].x) & 0x7ff00000u,
                   max(dhi(X[k].y) & 0x7ff00000u, dhi(X[k].z) & 0x7ff00000u)));
  E >>= 20;
  if (E == 0x7ffu) {
    sj[g] = __int_as_float(0x7fc00000);
    return;
  }
  // exact differences to node 1, and the bits any of them reaches
  long long D[7][3];
  unsigned long long reach = 0;
  {
    const long long f0x = fixed_of(X[0].x, E), f0y = fixed_of(X[0].y, E),
                    f0z = fixed_of(X[0].z, E);
#pragma unroll
    for (int k = 1; k < 8; ++k) {
      D[k - 1][0] = fixed_of(X[k].x, E) - f0x;
      D[k - 1][1] = fixed_of(X[k].y, E) - f0y;
      D[k - 1][2] = fixed_of(X[k].z, E) - f0z;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        reach |= static_cast<unsigned long long>(D[k - 1][c] ^ (D[k - 1][c] >> 63));
    }
  }
  // one left shift for all (|D| < 2^63 after it: the one's complement
  // magnitudes are below 2^(63 - L), so |D| <= 2^(63 - L)), top 32 bits to
  // FP32
  const int L = __clzll(static_cast<long long>(reach)) - 1;
  V3<float> Y[8];
  Y[0] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    float y[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      y[c] = __int2float_rn(static_cast<int>(
                 static_cast<unsigned long long>(D[k - 1][c]) << L >> 32)) * 0x1p-30f;
    Y[k] = {y[0], y[1], y[2]};
  }
  V3<float> a[4], b[4], c[4];
  edges_from_nodes(Y, a, b, c);
  float ra[4], rb[4], rc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    ra[q] = inv_norm(a[q]);
    rb[q] = inv_norm(b[q]);
    rc[q] = inv_norm(c[q]);
  }
  float q = 1.f;
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y)
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        const float j = det3(a[y + 2 * z], b[x + 2 * z], c[x + 2 * y]);
        // a zero-length edge makes j exactly 0 (and its inverse norm infinite);
        // |j| <= |a| |b| |c| keeps every partial product below 12
        const float s = j == 0.f ? 0.f : ((j * ra[y + 2 * z]) * rb[x + 2 * z]) * rc[x + 2 * y];
        q = fminf(q, s);
      }
  sj[g] = q;
}

}  // namespace

cudaError_t launch_quality(const Batch& p, float* sj, cudaStream_t st) {
  if (p.n <= 0) return cudaSuccess;
  const unsigned int blocks =
      static_cast<unsigned int>((p.n + kQualityThreads - 1) / kQualityThreads);
  if (p.indexed && reinterpret_cast<uintptr_t>(p.nodes) % 16 == 0)
    quality_kernel<true><<<blocks, kQualityThreads, 0, st>>>(p, sj);
  else
    quality_kernel<false><<<blocks, kQualityThreads, 0, st>>>(p, sj);
  return cudaGetLastError();
}

}  // namespace hexval
