// Stream compaction of element ids by verdict: the last step of candidate
// filtering (many candidate hexahedra over one node array, of which the valid
// ones are kept), and a general "ids whose verdict is in a set" primitive.
//
// Three launches over tiles of 8192 flags (256 threads x 32 flags):
//   count    per tile, the number of selected flags
//   scan     one block: exclusive prefix sums of the tile counts, and the total
//   scatter  per tile, each thread's selected ids at tile offset + the
//            exclusive prefix of the counts of the threads before it, staged
//            in shared memory and written out coalesced
// The ids come out in ascending order (a stable compaction), identical to a
// sequential scan.
#include "hexval_internal.cuh"

namespace hexval {

namespace {

constexpr int kCompactThreads = 256;
constexpr int kPerThread = 32;
constexpr int kTile = kCompactThreads * kPerThread;
constexpr int kScanThreads = 1024;

// Selection bits of this thread's 32 flags (bit j: flag base + j).
__device__ __forceinline__ uint32_t select_bits(const uint8_t* flags, int64_t n, int64_t base,
                                                uint32_t mask) {
  uint32_t bits = 0;
  if (base + kPerThread <= n && (reinterpret_cast<uintptr_t>(flags + base) & 15u) == 0u) {
    const uint4* v = reinterpret_cast<const uint4*>(flags + base);
    const uint4 a = __ldg(v), b = __ldg(v + 1);
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t f = (w[q] >> (8 * k)) & 7u;
        bits |= ((mask >> f) & 1u) << (4 * q + k);
      }
  } else {
    for (int j = 0; j < kPerThread; ++j)
      if (base + j < n) bits |= ((mask >> (flags[base + j] & 7u)) & 1u) << j;
  }
  return bits;
}

// Exclusive prefix of v over the block (256 threads) and the block total.
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t& total) {
  __shared__ uint32_t warp_sum[kCompactThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) warp_sum[w] = incl;
  __syncthreads();
  uint32_t before = 0;
  total = 0;
#pragma unroll
  for (int k = 0; k < kCompactThreads / 32; ++k) {
    const uint32_t s = warp_sum[k];
    before += k < w ? s : 0u;
    total += s;
  }
  __syncthreads();  // warp_sum is reused by the next call
  return before + incl - v;
}

__global__ void __launch_bounds__(kCompactThreads) count_kernel(const uint8_t* flags, int64_t n,
                                                                uint32_t mask, uint64_t* tiles) {
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile + threadIdx.x * kPerThread;
  uint32_t total;
  block_exclusive(__popc(select_bits(flags, n, base, mask)), total);
  if (threadIdx.x == 0) tiles[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_kernel(uint64_t* tiles, int64_t n_tiles,
                                                            int32_t* count) {
  __shared__ uint64_t part[kScanThreads];
  const int64_t per = (n_tiles + kScanThreads - 1) / kScanThreads;
  const int64_t lo = threadIdx.x * per, hi = min(lo + per, n_tiles);
  uint64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += tiles[i];
  part[threadIdx.x] = s;
  __syncthreads();
  // inclusive scan of the 1024 partial sums (Hillis-Steele in shared memory)
  for (int d = 1; d < kScanThreads; d <<= 1) {
    const uint64_t t = threadIdx.x >= d ? part[threadIdx.x - d] : 0ull;
    __syncthreads();
    part[threadIdx.x] += t;
    __syncthreads();
  }
  uint64_t run = part[threadIdx.x] - s;  // exclusive prefix of this thread's range
  for (int64_t i = lo; i < hi; ++i) {
    const uint64_t c = tiles[i];
    tiles[i] = run;
    run += c;
  }
  if (threadIdx.x == kScanThreads - 1) *count = static_cast<int32_t>(part[kScanThreads - 1]);
}

__global__ void __launch_bounds__(kCompactThreads) scatter_kernel(const uint8_t* flags, int64_t n,
                                                                  uint32_t mask,
                                                                  const uint64_t* tiles,
                                                                  int32_t* ids) {
  __shared__ int32_t stage[kTile];
  const int64_t tile0 = static_cast<int64_t>(blockIdx.x) * kTile;
  const int64_t base = tile0 + threadIdx.x * kPerThread;
  uint32_t bits = select_bits(flags, n, base, mask);
  uint32_t total;
  uint32_t pos = block_exclusive(__popc(bits), total);
  while (bits) {
    const int j = __ffs(bits) - 1;
    bits &= bits - 1;
    stage[pos++] = static_cast<int32_t>(base + j);
  }
  __syncthreads();
  int32_t* out = ids + tiles[blockIdx.x];
  for (uint32_t i = threadIdx.x; i < total; i += kCompactThreads) out[i] = stage[i];
}

}  // namespace

int64_t compact_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

cudaError_t launch_compact(const uint8_t* flags, int64_t n, uint32_t mask, uint64_t* tiles,
                           int32_t* ids, int32_t* count, cudaStream_t st) {
  const int64_t t = compact_tiles(n);
  if (t == 0) return cudaMemsetAsync(count, 0, sizeof(int32_t), st);
  count_kernel<<<static_cast<unsigned int>(t), kCompactThreads, 0, st>>>(flags, n, mask, tiles);
  scan_kernel<<<1, kScanThreads, 0, st>>>(tiles, t, count);
  scatter_kernel<<<static_cast<unsigned int>(t), kCompactThreads, 0, st>>>(flags, n, mask, tiles,
                                                                           ids);
  return cudaGetLastError();
}

}  // namespace hexval
