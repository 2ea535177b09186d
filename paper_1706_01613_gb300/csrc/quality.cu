// Corner scaled Jacobian of linear hexahedra: the quality measure quoted in
// Sec. 7 (Fig. f:invalidHighCornerQual) -- at each corner, the determinant of
// the three edge vectors leaving it (the columns of the Jacobian matrix
// there, Eq. e:det3d), each divided by its length; the element value is the
// minimum over the 8 corners (0 at a corner with a zero-length edge).
//
// One element per thread.  The node coordinates relative to node 1 are
// formed in FP64 (21 subtractions), scaled by a power of two so that the
// largest is in [1, 2) (the measure is scale invariant) and rounded to FP32
// on the integer pipe; edge vectors, corner determinants and norms are FP32.
// The relative coordinates carry a rounding error of 2^-24 of the largest,
// so the result is accurate to about 1e-6 for elements of moderate aspect
// ratio, independently of where the element sits.
#include "hexval_internal.cuh"

namespace hexval {

namespace {

constexpr int kQualityThreads = 256;

// x 2^(1023 - emax) rounded to FP32 on the integer pipe (|result| < 2 when
// emax is the largest biased exponent among the values); magnitudes below
// 2^-126 after scaling (and FP64 subnormals) become zero.
__device__ __forceinline__ float d2f_rel(double x, uint32_t emax) {
  const long long bits = __double_as_longlong(x);
  uint32_t hi = static_cast<uint32_t>(bits >> 32);
  const uint32_t lo = static_cast<uint32_t>(bits);
  const uint32_t e = (hi >> 20) & 0x7ffu;
  const int e2 = static_cast<int>(e) - static_cast<int>(emax) + 1023;
  if (e == 0u || e2 < 897) return __uint_as_float(hi & 0x80000000u);
  hi = (hi & 0x800fffffu) | (static_cast<uint32_t>(e2) << 20);
  uint32_t f = __funnelshift_l(lo, hi, 3);
  f = (f & 0x7fffffffu) ^ 0x40000000u;  // exponent field e2 - 896
  f += (lo >> 28) & 1u;                 // rounding to nearest (ties up)
  f |= hi & 0x80000000u;
  return __uint_as_float(f);
}

// 1 / |v|; squared norms that would underflow are formed after scaling by 2^60
__device__ __forceinline__ float inv_norm(const V3<float>& v) {
  const float n2 = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z));
  if (n2 >= 0x1p-100f) return rsqrtf(n2);
  const V3<float> w{v.x * 0x1p60f, v.y * 0x1p60f, v.z * 0x1p60f};
  return rsqrtf(fmaf(w.x, w.x, fmaf(w.y, w.y, w.z * w.z))) * 0x1p60f;
}

__global__ void __launch_bounds__(kQualityThreads) quality_kernel(Batch p, float* sj) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  const int64_t g = p.base + i;
  V3<double> X[8];
  if (!load_element(p, g, X)) {
    sj[g] = __int_as_float(0x7fc00000);
    set_status(p.s.status, kSbIndex);
    return;
  }
  // coordinates relative to node 1 and the largest exponent among them
  V3<double> R[8];
  uint32_t emax = 0, nonfinite = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    nonfinite |= ((dhi(X[k].x) & 0x7ff00000u) == 0x7ff00000u) |
                 ((dhi(X[k].y) & 0x7ff00000u) == 0x7ff00000u) |
                 ((dhi(X[k].z) & 0x7ff00000u) == 0x7ff00000u);
    R[k] = {X[k].x - X[0].x, X[k].y - X[0].y, X[k].z - X[0].z};
    emax = max(emax, max(dhi(R[k].x) & 0x7ff00000u,
                         max(dhi(R[k].y) & 0x7ff00000u, dhi(R[k].z) & 0x7ff00000u)));
  }
  emax >>= 20;
  if (nonfinite || emax == 0x7ffu) {
    sj[g] = __int_as_float(0x7fc00000);
    return;
  }
  V3<float> Y[8];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    Y[k] = {d2f_rel(R[k].x, emax), d2f_rel(R[k].y, emax), d2f_rel(R[k].z, emax)};
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
  quality_kernel<<<blocks, kQualityThreads, 0, st>>>(p, sj);
  return cudaGetLastError();
}

}  // namespace hexval
