// C ABI of libhexval (declared in include/hexval.h): handle management and
// the per-call launch sequence.
//
// One call = one or more batches of at most max_batch elements; per batch:
//   memset(counters)
//   [FP32 form]  bulk32 (all elements) -> bulk64 over the escalation list
//   [FP64 form]  bulk64 (all elements)
//   refine, levels 0 .. D-1 (each launch reads its box count on the device
//                and returns at once when the level is empty)
//   finalize (verdicts of refined elements)
//   exact (elements whose signs could not be certified)
// Nothing synchronises with the host, nothing allocates: a call can be
// enqueued on any stream and captured into a CUDA graph.
#include <cstdio>
#include <cstring>
#include <new>

#include "hexval_internal.cuh"

using hexval::Batch;
using hexval::Scratch;

struct hexval_ctx {
  hexval_config cfg;
  Scratch s;
  void* blocks[24];
  int nblocks;
};

namespace {

int set_device(const hexval_ctx* h) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return HEXVAL_E_CUDA;
  if (cur != h->cfg.device && cudaSetDevice(h->cfg.device) != cudaSuccess) return HEXVAL_E_CUDA;
  return HEXVAL_OK;
}

template <typename T>
bool alloc(hexval_ctx* h, T** out, uint64_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  h->blocks[h->nblocks++] = p;
  *out = static_cast<T*>(p);
  return true;
}

void free_all(hexval_ctx* h) {
  for (int i = 0; i < h->nblocks; ++i) cudaFree(h->blocks[i]);
  h->nblocks = 0;
}

int run_batches(hexval_ctx* h, Batch p, int64_t n_hex, cudaStream_t st) {
  const hexval_config& c = h->cfg;
  for (int64_t base = 0; base < n_hex; base += static_cast<int64_t>(c.max_batch)) {
    p.base = base;
    p.n = n_hex - base < static_cast<int64_t>(c.max_batch) ? n_hex - base
                                                            : static_cast<int64_t>(c.max_batch);
    if (cudaMemsetAsync(h->s.cnt, 0, sizeof(hexval::Counters), st) != cudaSuccess)
      return HEXVAL_E_CUDA;
    cudaError_t e;
    if (c.precision == HEXVAL_FP32_FILTERED) {
      if ((e = hexval::launch_bulk32(p, st)) != cudaSuccess) return HEXVAL_E_CUDA;
      if ((e = hexval::launch_bulk64(p, true, st)) != cudaSuccess) return HEXVAL_E_CUDA;
    } else {
      if ((e = hexval::launch_bulk64(p, false, st)) != cudaSuccess) return HEXVAL_E_CUDA;
    }
    for (int level = 0; level < c.max_depth; ++level)
      if (hexval::launch_refine(p, level, st) != cudaSuccess) return HEXVAL_E_CUDA;
    if (hexval::launch_finalize(p, st) != cudaSuccess) return HEXVAL_E_CUDA;
    if (hexval::launch_exact(p, st) != cudaSuccess) return HEXVAL_E_CUDA;
  }
  return HEXVAL_OK;
}

}  // namespace

extern "C" {

int hexval_config_default(hexval_config* cfg) {
  if (!cfg) return HEXVAL_E_ARG;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->struct_size = sizeof(hexval_config);
  cfg->device = 0;
  cfg->precision = HEXVAL_FP64;
  cfg->max_depth = 8;
  cfg->max_batch = 1ull << 24;
  cfg->queue_capacity = 1ull << 23;
  cfg->max_nodes = 1ull << 24;
  cfg->exact_capacity = 1ull << 16;
  return HEXVAL_OK;
}

int hexval_create(const hexval_config* cfg, hexval_handle* out) {
  if (!cfg || !out || cfg->struct_size != sizeof(hexval_config)) return HEXVAL_E_ARG;
  if (cfg->max_depth < 0 || cfg->max_depth > hexval::kMaxDepth) return HEXVAL_E_ARG;
  if (cfg->precision != HEXVAL_FP64 && cfg->precision != HEXVAL_FP32_FILTERED) return HEXVAL_E_ARG;
  if (cfg->max_batch == 0 || cfg->max_batch > (1ull << 31) || cfg->queue_capacity == 0 ||
      cfg->queue_capacity > (1ull << 31) || cfg->exact_capacity == 0 ||
      cfg->exact_capacity > (1ull << 31) || cfg->max_nodes > (1ull << 31))
    return HEXVAL_E_ARG;
  hexval_ctx* h = new (std::nothrow) hexval_ctx();
  if (!h) return HEXVAL_E_NOMEM;
  h->cfg = *cfg;
  if (set_device(h) != HEXVAL_OK) {
    delete h;
    return HEXVAL_E_CUDA;
  }
  Scratch& s = h->s;
  s.qcap = cfg->queue_capacity;
  s.exact_cap = cfg->exact_capacity;
  s.max_nodes = cfg->max_nodes;
  s.exact_work_words = hexval::exact_work_words_per_worker() * hexval::exact_workers();
  bool ok = alloc(h, &s.qcoef[0], 27 * s.qcap) && alloc(h, &s.qcoef[1], 27 * s.qcap) &&
            alloc(h, &s.qslot[0], s.qcap) && alloc(h, &s.qslot[1], s.qcap) &&
            alloc(h, &s.slot_elem, s.qcap) && alloc(h, &s.slot_state, s.qcap) &&
            alloc(h, &s.slot_lev, s.qcap) && alloc(h, &s.slot_e0, s.qcap) &&
            alloc(h, &s.slot_m0, s.qcap) && alloc(h, &s.esc, cfg->max_batch) &&
            alloc(h, &s.exact_list, s.exact_cap) && alloc(h, &s.exact_work, s.exact_work_words) &&
            alloc(h, &s.node32, 8 * s.max_nodes) && alloc(h, &s.cnt, 1) &&
            alloc(h, &s.stats, 1) && alloc(h, &s.status, 1);
  if (!ok) {
    free_all(h);
    delete h;
    return HEXVAL_E_NOMEM;
  }
  if (cudaMemset(s.cnt, 0, sizeof(hexval::Counters)) != cudaSuccess ||
      cudaMemset(s.stats, 0, sizeof(hexval::Stats)) != cudaSuccess ||
      cudaMemset(s.status, 0, sizeof(uint32_t)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    free_all(h);
    delete h;
    return HEXVAL_E_CUDA;
  }
  *out = h;
  return HEXVAL_OK;
}

int hexval_destroy(hexval_handle h) {
  if (!h) return HEXVAL_E_ARG;
  set_device(h);
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return HEXVAL_OK;
}

int hexval_check_soa(hexval_handle h, int64_t n_hex, const double* corners, uint8_t* flags,
                     double* bmin, double* bmax, void* stream) {
  if (!h || n_hex < 0 || n_hex >= (1ll << 31)) return HEXVAL_E_ARG;
  if (n_hex == 0) return HEXVAL_OK;
  if (!corners || !flags) return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  Batch p{};
  p.soa = corners;
  p.stride = n_hex;
  p.indexed = 0;
  p.flags = flags;
  p.bmin = bmin;
  p.bmax = bmax;
  p.max_depth = h->cfg.max_depth;
  p.s = h->s;
  return run_batches(h, p, n_hex, static_cast<cudaStream_t>(stream));
}

int hexval_check_indexed(hexval_handle h, int64_t n_nodes, const double* nodes, int64_t n_hex,
                         const int32_t* conn, uint8_t* flags, double* bmin, double* bmax,
                         void* stream) {
  if (!h || n_hex < 0 || n_hex >= (1ll << 31) || n_nodes < 0 || n_nodes >= (1ll << 31))
    return HEXVAL_E_ARG;
  if (n_hex == 0) return HEXVAL_OK;
  if (!nodes || !conn || !flags || n_nodes == 0) return HEXVAL_E_ARG;
  if (reinterpret_cast<uintptr_t>(conn) % 16 != 0) return HEXVAL_E_ARG;  // int4 rows
  if (h->cfg.precision == HEXVAL_FP32_FILTERED && static_cast<uint64_t>(n_nodes) > h->s.max_nodes)
    return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Batch p{};
  p.nodes = nodes;
  p.n_nodes = n_nodes;
  p.conn = conn;
  p.indexed = 1;
  p.flags = flags;
  p.bmin = bmin;
  p.bmax = bmax;
  p.max_depth = h->cfg.max_depth;
  p.s = h->s;
  if (h->cfg.precision == HEXVAL_FP32_FILTERED &&
      hexval::launch_nodes32(p, st) != cudaSuccess)
    return HEXVAL_E_CUDA;
  return run_batches(h, p, n_hex, st);
}

int hexval_status(hexval_handle h, void* stream) {
  if (!h) return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return HEXVAL_E_CUDA;
  uint32_t bits = 0;
  if (cudaMemcpy(&bits, h->s.status, sizeof(bits), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HEXVAL_E_CUDA;
  if (bits && cudaMemset(h->s.status, 0, sizeof(uint32_t)) != cudaSuccess) return HEXVAL_E_CUDA;
  if (bits & hexval::kSbIndex) return HEXVAL_E_INDEX;
  if (bits & hexval::kSbQueue) return HEXVAL_E_QUEUE;
  if (bits & hexval::kSbRange) return HEXVAL_E_RANGE;
  if (bits & hexval::kSbTimeout) return HEXVAL_E_TIMEOUT;
  return HEXVAL_OK;
}

int hexval_get_stats(hexval_handle h, hexval_stats* out, int reset, void* stream) {
  if (!h || !out) return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return HEXVAL_E_CUDA;
  hexval::Stats s{};
  if (cudaMemcpy(&s, h->s.stats, sizeof(s), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HEXVAL_E_CUDA;
  out->elements = s.elements;
  out->escalated_fp64 = s.escalated_fp64;
  out->refined = s.refined;
  out->boxes = s.boxes;
  out->exact = s.exact;
  out->max_level_boxes = s.max_level_boxes;
  if (reset && cudaMemset(h->s.stats, 0, sizeof(s)) != cudaSuccess) return HEXVAL_E_CUDA;
  return HEXVAL_OK;
}

const char* hexval_strerror(int code) {
  switch (code) {
    case HEXVAL_OK: return "ok";
    case HEXVAL_E_ARG: return "invalid argument";
    case HEXVAL_E_NOMEM: return "device allocation failed";
    case HEXVAL_E_CUDA: return "CUDA runtime error";
    case HEXVAL_E_INDEX: return "connectivity entry out of range";
    case HEXVAL_E_QUEUE: return "refinement queue or escalation list full";
    case HEXVAL_E_TIMEOUT: return "a bounded device wait gave up";
    case HEXVAL_E_RANGE: return "element outside the range of the exact tier";
    default: return "unknown code";
  }
}

}  // extern "C"
