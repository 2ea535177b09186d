// hexval_check_soa_noalloc: the FP64 validity check of independent elements
// for callers that cannot allocate device memory (code running where
// cudaMalloc is unavailable or forbidden: inside a host callback or a driver
// layer that owns all allocations, under a memory pool that must not grow,
// or in a process whose allocator is locked after start-up).
//
// It launches the same kernels as hexval_check_soa with a FP64 handle
// (bulk64, then the tail with the exact box check and the exact tier), but
// their scratch -- refinement queue with box positions, exact-check list,
// per-element refinement state, exact-tier list and stacks, counters,
// statistics and status -- lives in one file-scope static device array of
// fixed size, instead of memory allocated by hexval_create.  The caller
// passes only the inputs and the outputs.
//
// Limits: at most kNoallocMaxHex elements per call, a refinement queue of
// kNoallocMaxHex boxes per level (a level that would need more sends the
// elements concerned to the exact tier, whose list holds kNoallocMaxHex
// elements), depth cap 0..15.  The static array takes kScratchBytes (about
// 48 MB) on every device that loads the library, until the process exits.
#include <cstring>
#include <mutex>

#include "hexval_internal.cuh"

namespace {

constexpr uint64_t kNoallocMaxHex = 16384;  // elements per call, boxes per level
constexpr uint64_t kCap = kNoallocMaxHex;

// byte offsets of the parts inside the static array (each 256-byte aligned)
constexpr uint64_t align256(uint64_t x) { return (x + 255) / 256 * 256; }
constexpr uint64_t kOffQcoef0 = 0;
constexpr uint64_t kOffQcoef1 = align256(kOffQcoef0 + 27 * kCap * sizeof(double));
constexpr uint64_t kOffQslot0 = align256(kOffQcoef1 + 27 * kCap * sizeof(double));
constexpr uint64_t kOffQslot1 = align256(kOffQslot0 + kCap * sizeof(uint32_t));
constexpr uint64_t kOffQpos0 = align256(kOffQslot1 + kCap * sizeof(uint32_t));
constexpr uint64_t kOffQpos1 = align256(kOffQpos0 + kCap * sizeof(uint64_t));
constexpr uint64_t kOffXbSlot = align256(kOffQpos1 + kCap * sizeof(uint64_t));
constexpr uint64_t kOffXbQi = align256(kOffXbSlot + hexval::kXbCap * sizeof(uint32_t));
constexpr uint64_t kOffXbPos = align256(kOffXbQi + hexval::kXbCap * sizeof(uint32_t));
constexpr uint64_t kOffElem = align256(kOffXbPos + hexval::kXbCap * sizeof(uint64_t));
constexpr uint64_t kOffState = align256(kOffElem + kCap * sizeof(uint32_t));
constexpr uint64_t kOffLev = align256(kOffState + kCap * sizeof(uint32_t));
constexpr uint64_t kOffE0 = align256(kOffLev + kCap * sizeof(uint32_t));
constexpr uint64_t kOffM0 = align256(kOffE0 + kCap * sizeof(double));
constexpr uint64_t kOffExactList = align256(kOffM0 + kCap * sizeof(double));
constexpr uint64_t kOffCnt = align256(kOffExactList + kCap * sizeof(uint32_t));
constexpr uint64_t kOffStats = align256(kOffCnt + sizeof(hexval::Counters));
constexpr uint64_t kOffStatus = align256(kOffStats + sizeof(hexval::Stats));
constexpr uint64_t kOffExactWork = align256(kOffStatus + sizeof(uint32_t));
// the exact tier's stacks: 592 integers x 32 limbs x 512 workers, 4 bytes each
constexpr uint64_t kExactWorkWords = 592ull * 32ull * 512ull;
constexpr uint64_t kScratchBytes = align256(kOffExactWork + kExactWorkWords * sizeof(uint32_t));

// The scratch.  In host code `scratch` names a host-side stand-in, not the
// device array: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of `scratch` on the current device.  It is looked up on
// every call (a host-side query); when it differs from the one seen before
// on this device (the first call, or a new context after a device reset
// reloaded the module) the counters are zeroed on the caller's stream, ahead
// of the call's kernels.  Later calls find them at zero: every call's tail
// kernel resets them.
int scratch_address(int dev, cudaStream_t st, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return HEXVAL_E_ARG;
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, scratch) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return HEXVAL_E_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_addr[dev] != ptr) {
    if (cudaMemsetAsync(static_cast<unsigned char*>(ptr) + kOffCnt, 0, kOffExactWork - kOffCnt,
                        st) != cudaSuccess) {
      cudaGetLastError();
      return HEXVAL_E_CUDA;
    }
    g_addr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_addr[dev];
  return HEXVAL_OK;
}

}  // namespace

extern "C" int hexval_check_soa_noalloc(int64_t n_hex, const double* corners, uint8_t* flags,
                                        double* bmin, double* bmax, int32_t max_depth,
                                        uint32_t* status_bits, void* stream) {
  if (n_hex < 0 || static_cast<uint64_t>(n_hex) > kNoallocMaxHex) return HEXVAL_E_ARG;
  if (max_depth < 0 || max_depth > hexval::kMaxDepth) return HEXVAL_E_ARG;
  if (n_hex > 0 && (!corners || !flags)) return HEXVAL_E_ARG;
  if (hexval::exact_work_words() != kExactWorkWords) return HEXVAL_E_CUDA;  // layout guard
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HEXVAL_E_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  int rc = scratch_address(dev, st, &base);
  if (rc != HEXVAL_OK) return rc;
  // status of this call starts clean (the array keeps the last call's contents)
  if (cudaMemsetAsync(base + kOffStatus, 0, sizeof(uint32_t), st) != cudaSuccess)
    return HEXVAL_E_CUDA;
  if (n_hex > 0) {
    hexval::Batch p{};
    p.n = n_hex;
    p.base = 0;
    p.soa = corners;
    p.stride = n_hex;
    p.indexed = 0;
    p.flags = flags;
    p.bmin = bmin;
    p.bmax = bmax;
    p.max_depth = max_depth;
    p.esc_in_pass = hexval::kEscInPassDefault;
    p.r32_in_pass = hexval::kR32InPassDefault;
    p.warp_items = hexval::kWarpItemsDefault;
    hexval::Scratch& s = p.s;
    s.qcoef[0] = reinterpret_cast<double*>(base + kOffQcoef0);
    s.qcoef[1] = reinterpret_cast<double*>(base + kOffQcoef1);
    s.qslot[0] = reinterpret_cast<uint32_t*>(base + kOffQslot0);
    s.qslot[1] = reinterpret_cast<uint32_t*>(base + kOffQslot1);
    s.qpos[0] = reinterpret_cast<uint64_t*>(base + kOffQpos0);
    s.qpos[1] = reinterpret_cast<uint64_t*>(base + kOffQpos1);
    s.qcap = kCap;
    s.xb_slot = reinterpret_cast<uint32_t*>(base + kOffXbSlot);
    s.xb_qi = reinterpret_cast<uint32_t*>(base + kOffXbQi);
    s.xb_pos = reinterpret_cast<uint64_t*>(base + kOffXbPos);
    s.xb_cap = hexval::kXbCap;
    s.slot_elem = reinterpret_cast<uint32_t*>(base + kOffElem);
    s.slot_state = reinterpret_cast<uint32_t*>(base + kOffState);
    s.slot_lev = reinterpret_cast<uint32_t*>(base + kOffLev);
    s.slot_e0 = reinterpret_cast<double*>(base + kOffE0);
    s.slot_m0 = reinterpret_cast<double*>(base + kOffM0);
    s.esc = nullptr;  // FP64 form: no escalation list
    s.exact_list = reinterpret_cast<uint32_t*>(base + kOffExactList);
    s.exact_cap = kCap;
    s.exact_work = reinterpret_cast<uint32_t*>(base + kOffExactWork);
    s.exact_work_words = kExactWorkWords;
    s.node32 = nullptr;
    s.max_nodes = 0;
    s.cnt = reinterpret_cast<hexval::Counters*>(base + kOffCnt);
    s.stats = reinterpret_cast<hexval::Stats*>(base + kOffStats);
    s.status = reinterpret_cast<uint32_t*>(base + kOffStatus);
    if (hexval::launch_bulk64(p, st) != cudaSuccess ||
        hexval::launch_tail(p, false, st) != cudaSuccess) {
      cudaGetLastError();
      cudaMemsetAsync(base + kOffCnt, 0, sizeof(hexval::Counters), st);
      return HEXVAL_E_CUDA;
    }
  }
  if (status_bits &&
      cudaMemcpyAsync(status_bits, base + kOffStatus, sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                      st) != cudaSuccess)
    return HEXVAL_E_CUDA;
  return HEXVAL_OK;
}
