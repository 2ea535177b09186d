// Minimum of the Jacobian determinant to a tolerance (Sec. 1 and Sec. 3,
// after [johnen2013]): by the convex hull property the smallest Bezier
// coefficient of a box bounds J from below on it, and the smallest corner
// coefficient (a value of J) bounds its minimum from above; subdividing
// sharpens both, quadratically in the box size.
//
// Per element, with tol = rel_tol * max |b| (b the depth-0 coefficients),
// breadth first: every box whose lower bound is below U - tol is split in 8
// (the others cannot lower the answer by more than tol and stay as they are),
// U takes the smallest corner coefficient of the children, children whose
// lower bound is at least U are dropped, L is the smallest lower bound left
// (at most U); until U - L <= tol or the depth cap.  The boxes are classified
// against the U of the start of their level, so the result does not depend
// on the order in which they are processed.  Every coefficient carries the
// certified FP64 bound E0 + d 2^-49 M0 (as the refinement of tail.cu), so
// the true minimum lies in [L, U].
//
// One element per warp (elements dealt by an atomic counter), FP64: the
// warp computes the root coefficients together (warp_items.cuh) and expands
// each box together (the three de Casteljau passes over 9, 15 and 25 rows
// on its lanes), as an FP64 warp-instruction costs the same whatever its
// active lanes.  Each warp owns a slice of the handle's box queue (two level
// buffers); a level that outgrows it keeps the extra children's lower bounds
// in L and reports the element as not converged.
#include "warp_items.cuh"

namespace hexval {

namespace {

constexpr int kMinjThreads = 128;

struct MinjArgs {
  double rel_tol;
  int max_depth;
  double* lo;
  double* hi;
  uint8_t* depth;
  unsigned int* next;  // element counter (zeroed before the launch)
};

// Order-preserving keys for warp minima on the integer pipe.
__device__ __forceinline__ double warp_min_d(double v) {
  long long k = dkey(v);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const long long o = __shfl_xor_sync(kFull, k, d);
    k = o < k ? o : k;
  }
  return dunkey(k);
}

__device__ __forceinline__ double warp_max_abs(double v) {
  unsigned long long k = static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7fffffffffffffffull;
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(kFull, k, d);
    k = o > k ? o : k;
  }
  return __longlong_as_double(static_cast<long long>(k));
}

__global__ void __launch_bounds__(kMinjThreads) minj_kernel(Batch p, MinjArgs a) {
  __shared__ double wsm[kMinjThreads / 32][kWarpScratch];
  double* sm = wsm[threadIdx.x >> 5];
  const Scratch& S = p.s;
  const int lane = threadIdx.x & 31;
  const unsigned int nwarps = gridDim.x * (blockDim.x >> 5);
  const unsigned int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint64_t cap = S.qcap / nwarps;  // boxes per level buffer of this warp
  const uint64_t base = w * cap;
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  for (;;) {
    unsigned int e = 0;
    if (lane == 0) e = atomicAdd(a.next, 1u);
    e = __shfl_sync(kFull, e, 0);
    if (e >= static_cast<unsigned int>(p.n)) return;
    const int64_t g = p.base + e;
    double smp, coef, E0;
    const int rc = warp_root64(p, g, sm, smp, coef, E0);
    if (rc) {
      if (lane == 0) {
        a.lo[g] = qnan;
        a.hi[g] = qnan;
        a.depth[g] = 0;
        if (rc == 1) set_status(S.status, kSbIndex);
      }
      continue;
    }
    const double un =
        lane < 8 ? coef : (lane < 20 ? coef * 0.5 : (lane < 26 ? coef * 0.25 : coef * 0.125));
    const double big = __longlong_as_double(0x7fefffffffffffffLL);
    const double M = warp_max_abs(lane < 27 ? un : 0.0);
    const double M0 = M + E0, tol = a.rel_tol * M;
    double U = warp_min_d(lane < 8 ? un : big) + E0;
    double L = fmin(U, warp_min_d(lane < 27 ? un : big) - E0);
    double settled = big;
    uint64_t nb = 1;  // boxes of the current level
    int cur = 0, d = 0;
    bool capped = false;
    if (cap == 0) {
      capped = true;
      nb = 0;
    } else if (lane < 27) {
      S.qcoef[0][static_cast<uint64_t>(tensor_pos(lane)) * S.qcap + base] = un;
    }
    __syncwarp();
    while (U - L > tol && d < a.max_depth && nb > 0) {
      const double u0 = U;
      const double Ed = fma(static_cast<double>(d) * 0x1p-49, M0, E0);
      const double Ec = fma(static_cast<double>(d + 1) * 0x1p-49, M0, E0);
      double lowmin = big;  // smallest lower bound among the children kept
      uint64_t nn = 0;
      for (uint64_t j = 0; j < nb; ++j) {
        double* A = sm;
        double* P1 = sm + 27;
        double* P2 = sm + 72;
        double* G = sm + 147;
        const double v = lane < 27 ? ldcg(S.qcoef[cur] + static_cast<uint64_t>(lane) * S.qcap + base + j) : big;
        if (lane < 27) A[lane] = v;
        const double lob = warp_min_d(v) - Ed;
        if (lob >= u0) continue;  // cannot hold a value below U
        if (lob >= u0 - tol) {    // within the tolerance: kept as it is
          settled = fmin(settled, lob);
          continue;
        }
        __syncwarp();
        if (lane < 9) {
          const int jj = lane % 3, k = lane / 3;
          split5_row(A + 3 * jj + 9 * k, 1, P1 + 5 * (jj + 3 * k), 1);
        }
        __syncwarp();
        if (lane < 15) {
          const int i = lane % 5, k = lane / 5;
          split5_row(P1 + i + 15 * k, 5, P2 + i + 25 * k, 5);
        }
        __syncwarp();
        if (lane < 25) {
          const int i = lane % 5, jj = lane / 5;
          split5_row(P2 + i + 5 * jj, 25, G + i + 5 * jj, 25);
        }
        __syncwarp();
        // lane o < 8: child o's smallest coefficient and smallest corner
        double cmin = big, ccor = big;
        if (lane < 8) {
          const int sx = 2 * (lane & 1), sy = 2 * ((lane >> 1) & 1), sz = 2 * (lane >> 2);
          long long km = dkey(big), kc = dkey(big);
          for (int k = 0; k < 3; ++k)
            for (int jj = 0; jj < 3; ++jj)
              for (int i = 0; i < 3; ++i) {
                const long long q = dkey(G[(sx + i) + 5 * ((sy + jj) + 5 * (sz + k))]);
                km = q < km ? q : km;
                if (i != 1 && jj != 1 && k != 1) kc = q < kc ? q : kc;
              }
          cmin = dunkey(km);
          ccor = dunkey(kc);
        }
        U = fmin(U, warp_min_d(ccor) + Ec);
        // children that may still hold a value below U go to the next level
        const double clo = cmin - Ec;
        const unsigned int keep = __ballot_sync(kFull, lane < 8 && clo < U) & 0xffu;
        lowmin = fmin(lowmin, warp_min_d((keep >> lane) & 1u ? clo : big));
        for (unsigned int q = keep; q; q &= q - 1) {
          const int o = __ffs(q) - 1;
          if (nn < cap) {
            const int sx = 2 * (o & 1), sy = 2 * ((o >> 1) & 1), sz = 2 * (o >> 2);
            if (lane < 27) {
              const int i = lane % 3, jj = (lane / 3) % 3, k = lane / 9;
              S.qcoef[cur ^ 1][static_cast<uint64_t>(lane) * S.qcap + base + nn] =
                  G[(sx + i) + 5 * ((sy + jj) + 5 * (sz + k))];
            }
            ++nn;
          } else {
            capped = true;  // no room: its lower bound stays in L
            settled = fmin(settled, shfl_d(clo, o));
          }
        }
        __syncwarp();
      }
      ++d;
      cur ^= 1;
      nb = nn;
      L = fmin(fmin(U, settled), lowmin);
    }
    if (lane == 0) {
      a.lo[g] = L;
      a.hi[g] = U;
      const bool conv = U - L <= tol;
      a.depth[g] = static_cast<uint8_t>(d | ((conv && !capped) ? 0 : 0x80));
    }
    __syncwarp();
  }
}

int minj_blocks() {
  static int blocks = 0;
  if (!blocks) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, minj_kernel, kMinjThreads, 0);
    blocks = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }
  return blocks;
}

}  // namespace

cudaError_t launch_minj(const Batch& p, double rel_tol, int max_depth, double* lo, double* hi,
                        uint8_t* depth, unsigned int* counter, cudaStream_t st) {
  if (p.n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  MinjArgs a{rel_tol, max_depth, lo, hi, depth, counter};
  const int64_t want = (p.n + (kMinjThreads / 32) - 1) / (kMinjThreads / 32);
  const int blocks = static_cast<int>(want < minj_blocks() ? want : minj_blocks());
  minj_kernel<<<blocks, kMinjThreads, 0, st>>>(p, a);
  return cudaGetLastError();
}

}  // namespace hexval
