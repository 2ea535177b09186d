// C ABI of libhexval (declared in include/hexval.h): handle management and
// the per-call launch sequence.
//
// One call = one or more batches of at most max_batch elements; per batch:
//   [FP32 form, indexed]  nodes32 (once per call)
//   bulk32 (FP32 form) or bulk64 (FP64 form) over all elements of the batch
//   [FP32 form, HEXVAL_OPT_DFREDO]  redo_df: double-float redo of escalations
//   [FP32 form, HEXVAL_OPT_PARTIAL64]  redo_partial: FP64 redo of only the
//          signs FP32 left unsettled in each escalation
//   [FP32 form, HEXVAL_OPT_LEVEL1]  level1: first refinement level of the
//          elements listed for the FP32 refinement
//   tail:  one cooperative launch that redoes the FP32 escalations in FP64,
//          refines the undecided elements level by level, runs the exact
//          tier, writes their verdicts and resets the batch counters.
// Nothing synchronises with the host, nothing allocates: a call can be
// enqueued on any stream and captured into a CUDA graph.
//
// Replay: a check call identical to the previous one on the handle (entry
// point, pointers, sizes; profiling off, the stream not capturing) is
// captured once into a CUDA graph on a private stream, and this graph is
// launched for every further identical call (one launch instead of three,
// a few microseconds less per call, as in an optimisation loop that
// re-checks the same mesh buffers).  HEXVAL_OPT_NO_REPLAY turns it off.
#include <cstdio>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "hexval_internal.cuh"

using hexval::Batch;
using hexval::Scratch;

namespace hexval {
// tail.cu: the tail launch with a grid-barrier budget (polls; <= 0: default)
cudaError_t launch_tail(const Batch& p, bool from_list, long long spin_limit, cudaStream_t st);
}  // namespace hexval

// Event pairs for the optional per-phase timing.
struct Profiler {
  static constexpr int kPairs = 2048;
  bool on = false;
  cudaEvent_t ev[kPairs][2] = {};
  int phase[kPairs] = {};
  int head = 0, pending = 0;  // ring of recorded, unread pairs
  hexval_profile acc = {};
};

// What identifies a check call for replay (compared bytewise; padding zeroed).
struct CallKey {
  int kind;  // 0 SoA, 1 indexed
  int64_t n_hex;
  Batch p;
};

struct Replay {
  CallKey last, cached;
  bool have_last = false, have_graph = false;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;  // private capture stream
};

struct hexval_ctx {
  hexval_config cfg;
  long long spin_limit = 0;  // grid-barrier budget of the tail (0: default)
  Scratch s;
  void* blocks[48];
  int nblocks;
  uint64_t scratch_bytes = 0;  // device bytes allocated by hexval_create
  Profiler prof;
  Replay replay;
  // node array recorded by hexval_prepare_nodes (its FP32 records in s.node32
  // with the FP32 form); cleared by hexval_check_indexed
  const double* prep_nodes = nullptr;
  int64_t prep_n = 0;
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
  if (h->nblocks >= static_cast<int>(sizeof(h->blocks) / sizeof(h->blocks[0]))) return false;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  h->blocks[h->nblocks++] = p;
  h->scratch_bytes += count * sizeof(T);
  *out = static_cast<T*>(p);
  return true;
}

void free_all(hexval_ctx* h) {
  for (int i = 0; i < h->nblocks; ++i) cudaFree(h->blocks[i]);
  h->nblocks = 0;
}

void prof_drain(Profiler& P, int keep) {
  while (P.pending > keep) {
    int i = (P.head - P.pending + Profiler::kPairs) % Profiler::kPairs;
    float ms = 0.f;
    if (cudaEventSynchronize(P.ev[i][1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, P.ev[i][0], P.ev[i][1]) == cudaSuccess) {
      P.acc.ms[P.phase[i]] += ms;
      P.acc.launches[P.phase[i]] += 1;
    }
    cudaGetLastError();
    --P.pending;
  }
}

// NVTX range (host side: the enqueue of a phase or call) for timeline tools;
// a no-op without an attached tool.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

const char* phase_name(int ph) {
  switch (ph) {
    case HEXVAL_PH_NODES32: return "hexval nodes32";
    case HEXVAL_PH_BULK32: return "hexval bulk32";
    case HEXVAL_PH_BULK64: return "hexval bulk64";
    case HEXVAL_PH_TAIL: return "hexval tail";
    case HEXVAL_PH_REDODF: return "hexval redo_df";
    case HEXVAL_PH_LEVEL1: return "hexval level1";
    case HEXVAL_PH_PARTIAL: return "hexval redo_partial";
    default: return "hexval";
  }
}

// Launches one phase, bracketed by timing events when profiling is on.
template <typename F>
cudaError_t phase(hexval_ctx* h, int ph, cudaStream_t st, F&& launch) {
  NvtxRange range(phase_name(ph));
  Profiler& P = h->prof;
  if (!P.on) return launch();
  if (P.pending == Profiler::kPairs) prof_drain(P, Profiler::kPairs - 1);
  int i = P.head;
  cudaEventRecord(P.ev[i][0], st);
  cudaError_t e = launch();
  cudaEventRecord(P.ev[i][1], st);
  P.phase[i] = ph;
  P.head = (P.head + 1) % Profiler::kPairs;
  ++P.pending;
  return e;
}

int run_batches(hexval_ctx* h, Batch p, int64_t n_hex, cudaStream_t st) {
  const hexval_config& c = h->cfg;
  for (int64_t base = 0; base < n_hex; base += static_cast<int64_t>(c.max_batch)) {
    p.base = base;
    p.n = n_hex - base < static_cast<int64_t>(c.max_batch) ? n_hex - base
                                                            : static_cast<int64_t>(c.max_batch);
    const bool fp32 = c.precision == HEXVAL_FP32_FILTERED;
    cudaError_t e = fp32 ? phase(h, HEXVAL_PH_BULK32, st, [&] { return hexval::launch_bulk32(p, st); })
                         : phase(h, HEXVAL_PH_BULK64, st, [&] { return hexval::launch_bulk64(p, st); });
    if (e == cudaSuccess && fp32 && p.dfredo)
      e = phase(h, HEXVAL_PH_REDODF, st, [&] { return hexval::launch_redo_df(p, st); });
    if (e == cudaSuccess && fp32 && p.partial64)
      e = phase(h, HEXVAL_PH_PARTIAL, st, [&] { return hexval::launch_redo_partial(p, st); });
    if (e == cudaSuccess && fp32 && p.level1)
      e = phase(h, HEXVAL_PH_LEVEL1, st, [&] { return hexval::launch_level1(p, st); });
    if (e == cudaSuccess)
      e = phase(h, HEXVAL_PH_TAIL, st,
                [&] { return hexval::launch_tail(p, fp32, h->spin_limit, st); });
    if (e != cudaSuccess) {
      // the tail resets the counters; if it could not run, reset them here
      cudaGetLastError();
      cudaMemsetAsync(h->s.cnt, 0, sizeof(hexval::Counters), st);
      return HEXVAL_E_CUDA;
    }
  }
  return HEXVAL_OK;
}

// The launch sequence of one check call (kind 0 SoA, 1 indexed, 2 indexed on
// prepared nodes: no node conversion).
int launch_call(hexval_ctx* h, const Batch& p, int kind, int64_t n_hex, cudaStream_t st) {
  if (kind == 1 && h->cfg.precision == HEXVAL_FP32_FILTERED &&
      phase(h, HEXVAL_PH_NODES32, st, [&] { return hexval::launch_nodes32(p, st); }) !=
          cudaSuccess)
    return HEXVAL_E_CUDA;
  return run_batches(h, p, n_hex, st);
}

// Captures the call's sequence into the handle's graph (updated in place when
// one exists); false when capture or instantiation fails.
bool capture_call(hexval_ctx* h, const Batch& p, int kind, int64_t n_hex) {
  Replay& R = h->replay;
  if (!R.cap && cudaStreamCreateWithFlags(&R.cap, cudaStreamNonBlocking) != cudaSuccess) {
    R.cap = nullptr;
    cudaGetLastError();
    return false;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(R.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int rc = launch_call(h, p, kind, n_hex, R.cap);
  const cudaError_t e = cudaStreamEndCapture(R.cap, &g);
  bool ok = rc == HEXVAL_OK && e == cudaSuccess && g != nullptr;
  if (ok && R.exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(R.exec, g, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(R.exec);
      R.exec = nullptr;
    }
  }
  if (ok && !R.exec && cudaGraphInstantiate(&R.exec, g, 0) != cudaSuccess) {
    R.exec = nullptr;
    ok = false;
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  R.have_graph = ok;
  return ok;
}

// Direct launches, or the replay of a repeated call.
int run_call(hexval_ctx* h, const Batch& p, int kind, int64_t n_hex, cudaStream_t st) {
  NvtxRange range(kind == 0 ? "hexval_check_soa"
                            : kind == 1 ? "hexval_check_indexed" : "hexval_check_indexed_prepared");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if ((h->cfg.options & HEXVAL_OPT_NO_REPLAY) || h->prof.on ||
      cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return launch_call(h, p, kind, n_hex, st);
  }
  Replay& R = h->replay;
  CallKey k;
  std::memset(&k, 0, sizeof(k));
  k.kind = kind;
  k.n_hex = n_hex;
  std::memcpy(&k.p, &p, sizeof(Batch));
  if (R.have_graph && std::memcmp(&k, &R.cached, sizeof(k)) == 0)
    return cudaGraphLaunch(R.exec, st) == cudaSuccess ? HEXVAL_OK : HEXVAL_E_CUDA;
  const bool repeat = R.have_last && std::memcmp(&k, &R.last, sizeof(k)) == 0;
  std::memcpy(&R.last, &k, sizeof(k));
  R.have_last = true;
  if (!repeat || !capture_call(h, p, kind, n_hex)) return launch_call(h, p, kind, n_hex, st);
  std::memcpy(&R.cached, &k, sizeof(k));
  return cudaGraphLaunch(R.exec, st) == cudaSuccess ? HEXVAL_OK : HEXVAL_E_CUDA;
}

// Batch of an indexed check on nodes (n_nodes) and rows conn.
Batch indexed_batch(const hexval_ctx* h, int64_t n_nodes, const double* nodes,
                    const int32_t* conn, uint8_t* flags, double* bmin, double* bmax) {
  Batch p{};
  p.nodes = nodes;
  p.n_nodes = n_nodes;
  p.conn = conn;
  p.indexed = 1;
  p.pair32 = (h->cfg.options & HEXVAL_OPT_PAIR32) != 0;
  p.prefetch32 = (h->cfg.options & HEXVAL_OPT_PREFETCH) != 0;
  p.dfredo = (h->cfg.options & HEXVAL_OPT_DFREDO) != 0;
  p.level1 = (h->cfg.options & HEXVAL_OPT_LEVEL1) != 0;
  p.partial64 = (h->cfg.options & HEXVAL_OPT_PARTIAL64) != 0;
  p.bulk_threads = static_cast<int>(h->cfg.bulk_threads);
  p.esc_in_pass = h->cfg.esc_in_pass;
  p.r32_in_pass = h->cfg.refine_in_pass;
  p.warp_items = h->cfg.tail_warp_items;
  p.flags = flags;
  p.bmin = bmin;
  p.bmax = bmax;
  p.max_depth = h->cfg.max_depth;
  p.s = h->s;
  return p;
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
  cfg->esc_in_pass = hexval::kEscInPassDefault;
  cfg->refine_in_pass = hexval::kR32InPassDefault;
  cfg->tail_warp_items = hexval::kWarpItemsDefault;
  return HEXVAL_OK;
}

int hexval_create(const hexval_config* cfg, hexval_handle* out) {
  if (!cfg || !out || cfg->struct_size != sizeof(hexval_config)) return HEXVAL_E_ARG;
  if (cfg->max_depth < 0 || cfg->max_depth > hexval::kMaxDepth) return HEXVAL_E_ARG;
  if (cfg->precision != HEXVAL_FP64 && cfg->precision != HEXVAL_FP32_FILTERED) return HEXVAL_E_ARG;
  if (cfg->max_batch == 0 || cfg->max_batch > (1ull << 31) || cfg->queue_capacity == 0 ||
      cfg->queue_capacity > (1ull << 31) || cfg->exact_capacity == 0 ||
      cfg->exact_capacity > (1ull << 31) || cfg->max_nodes > (1ull << 31) ||
      (cfg->options & ~static_cast<uint32_t>(HEXVAL_OPT_PAIR32 | HEXVAL_OPT_PREFETCH | HEXVAL_OPT_DFREDO |
                                             HEXVAL_OPT_NO_REPLAY | HEXVAL_OPT_LEVEL1 |
                                             HEXVAL_OPT_PARTIAL64)) ||
      ((cfg->options & HEXVAL_OPT_DFREDO) && (cfg->options & HEXVAL_OPT_PARTIAL64)) ||
      cfg->reserved || cfg->reserved2 || cfg->tail_warp_items < 1 || cfg->tail_warp_items > 64 ||
      (cfg->bulk_threads != 0 && cfg->bulk_threads != 64 && cfg->bulk_threads != 128 &&
       cfg->bulk_threads != 256))
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
  s.exact_work_words = hexval::exact_work_words();
  s.xb_cap = hexval::kXbCap;
  h->spin_limit = cfg->spin_limit;
  bool ok = alloc(h, &s.qcoef[0], 27 * s.qcap) && alloc(h, &s.qcoef[1], 27 * s.qcap) &&
            alloc(h, &s.qslot[0], s.qcap) && alloc(h, &s.qslot[1], s.qcap) &&
            alloc(h, &s.qpos[0], s.qcap) && alloc(h, &s.qpos[1], s.qcap) &&
            alloc(h, &s.xb_slot, s.xb_cap) && alloc(h, &s.xb_qi, s.xb_cap) &&
            alloc(h, &s.xb_pos, s.xb_cap) &&
            alloc(h, &s.slot_elem, s.qcap) && alloc(h, &s.slot_state, s.qcap) &&
            alloc(h, &s.slot_lev, s.qcap) && alloc(h, &s.slot_e0, s.qcap) &&
            alloc(h, &s.slot_m0, s.qcap) && alloc(h, &s.esc, cfg->max_batch) &&
            alloc(h, &s.exact_list, s.exact_cap) && alloc(h, &s.exact_work, s.exact_work_words) &&
            alloc(h, &s.node32, 4 * s.max_nodes) && alloc(h, &s.cnt, 1) &&
            alloc(h, &s.stats, 1) && alloc(h, &s.status, 1) &&
            alloc(h, &s.tiles, static_cast<uint64_t>(hexval::compact_tiles(1ll << 31)));
  s.tiles_cap = static_cast<uint64_t>(hexval::compact_tiles(1ll << 31));
  if (ok && cfg->precision == HEXVAL_FP32_FILTERED) {
    s.q32cap = s.qcap;
    ok = alloc(h, &s.r32, cfg->max_batch) && alloc(h, &s.esc2, cfg->max_batch) &&
         alloc(h, &s.q32coef[0], 27 * s.q32cap) && alloc(h, &s.q32coef[1], 27 * s.q32cap) &&
         alloc(h, &s.q32slot[0], s.q32cap) && alloc(h, &s.q32slot[1], s.q32cap) &&
         alloc(h, &s.s32_elem, cfg->max_batch) && alloc(h, &s.s32_state, cfg->max_batch) &&
         alloc(h, &s.s32_lev, cfg->max_batch) && alloc(h, &s.s32_e0, cfg->max_batch) &&
         alloc(h, &s.s32_m0, cfg->max_batch) &&
         alloc(h, &s.iw, static_cast<uint64_t>(hexval::kIwSlots) * 2 * 27 * hexval::kIwBoxes) &&
         alloc(h, &s.esc3, cfg->max_batch) && alloc(h, &s.r32b, cfg->max_batch);
  }
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
  if (h->prof.ev[0][0])
    for (int i = 0; i < Profiler::kPairs; ++i) {
      cudaEventDestroy(h->prof.ev[i][0]);
      cudaEventDestroy(h->prof.ev[i][1]);
    }
  if (h->replay.exec) cudaGraphExecDestroy(h->replay.exec);
  if (h->replay.cap) cudaStreamDestroy(h->replay.cap);
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
  p.pair32 = (h->cfg.options & HEXVAL_OPT_PAIR32) != 0;
  p.dfredo = (h->cfg.options & HEXVAL_OPT_DFREDO) != 0;
  p.level1 = (h->cfg.options & HEXVAL_OPT_LEVEL1) != 0;
  p.partial64 = (h->cfg.options & HEXVAL_OPT_PARTIAL64) != 0;
  p.bulk_threads = static_cast<int>(h->cfg.bulk_threads);
  p.esc_in_pass = h->cfg.esc_in_pass;
  p.r32_in_pass = h->cfg.refine_in_pass;
  p.warp_items = h->cfg.tail_warp_items;
  p.flags = flags;
  p.bmin = bmin;
  p.bmax = bmax;
  p.max_depth = h->cfg.max_depth;
  p.s = h->s;
  return run_call(h, p, 0, n_hex, static_cast<cudaStream_t>(stream));
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
  h->prep_nodes = nullptr;  // the FP32 node records are replaced
  h->prep_n = 0;
  return run_call(h, indexed_batch(h, n_nodes, nodes, conn, flags, bmin, bmax), 1, n_hex,
                  static_cast<cudaStream_t>(stream));
}

int hexval_prepare_nodes(hexval_handle h, int64_t n_nodes, const double* nodes, void* stream) {
  if (!h || !nodes || n_nodes <= 0 || n_nodes >= (1ll << 31)) return HEXVAL_E_ARG;
  if (h->cfg.precision == HEXVAL_FP32_FILTERED && static_cast<uint64_t>(n_nodes) > h->s.max_nodes)
    return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  h->prep_nodes = nullptr;
  h->prep_n = 0;
  if (h->cfg.precision == HEXVAL_FP32_FILTERED) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Batch p = indexed_batch(h, n_nodes, nodes, nullptr, nullptr, nullptr, nullptr);
    if (phase(h, HEXVAL_PH_NODES32, st, [&] { return hexval::launch_nodes32(p, st); }) !=
        cudaSuccess)
      return HEXVAL_E_CUDA;
  }
  h->prep_nodes = nodes;
  h->prep_n = n_nodes;
  return HEXVAL_OK;
}

int hexval_check_indexed_prepared(hexval_handle h, int64_t n_hex, const int32_t* conn,
                                  uint8_t* flags, double* bmin, double* bmax, void* stream) {
  if (!h || n_hex < 0 || n_hex >= (1ll << 31)) return HEXVAL_E_ARG;
  if (n_hex == 0) return HEXVAL_OK;
  if (!h->prep_nodes || !conn || !flags) return HEXVAL_E_ARG;
  if (reinterpret_cast<uintptr_t>(conn) % 16 != 0) return HEXVAL_E_ARG;  // int4 rows
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  return run_call(h, indexed_batch(h, h->prep_n, h->prep_nodes, conn, flags, bmin, bmax), 2,
                  n_hex, static_cast<cudaStream_t>(stream));
}

int hexval_check_quads(hexval_handle h, int64_t n_quad, const double* corners, uint8_t* flags,
                       double* jmin, double* jmax, void* stream) {
  if (!h || n_quad < 0) return HEXVAL_E_ARG;
  if (n_quad == 0) return HEXVAL_OK;
  if (!corners || !flags) return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  hexval::QuadBatch q{};
  q.n = n_quad;
  q.soa = corners;
  q.stride = n_quad;
  q.indexed = 0;
  q.flags = flags;
  q.jmin = jmin;
  q.jmax = jmax;
  q.status = h->s.status;
  return hexval::launch_quads(q, h->cfg.precision == HEXVAL_FP32_FILTERED,
                              static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? HEXVAL_OK
             : HEXVAL_E_CUDA;
}

int hexval_check_quads_indexed(hexval_handle h, int64_t n_nodes, const double* nodes,
                               int64_t n_quad, const int32_t* conn, uint8_t* flags, double* jmin,
                               double* jmax, void* stream) {
  if (!h || n_quad < 0 || n_nodes < 0 || n_nodes >= (1ll << 31)) return HEXVAL_E_ARG;
  if (n_quad == 0) return HEXVAL_OK;
  if (!nodes || !conn || !flags || n_nodes == 0) return HEXVAL_E_ARG;
  if (reinterpret_cast<uintptr_t>(conn) % 16 != 0 || reinterpret_cast<uintptr_t>(nodes) % 16 != 0)
    return HEXVAL_E_ARG;  // int4 rows, double2 nodes
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  hexval::QuadBatch q{};
  q.n = n_quad;
  q.nodes = nodes;
  q.n_nodes = n_nodes;
  q.conn = conn;
  q.indexed = 1;
  q.flags = flags;
  q.jmin = jmin;
  q.jmax = jmax;
  q.status = h->s.status;
  return hexval::launch_quads(q, h->cfg.precision == HEXVAL_FP32_FILTERED,
                              static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? HEXVAL_OK
             : HEXVAL_E_CUDA;
}

int hexval_corner_quality(hexval_handle h, int64_t n_hex, const double* corners, float* sj_min,
                          void* stream) {
  if (!h || n_hex < 0 || n_hex >= (1ll << 31)) return HEXVAL_E_ARG;
  if (n_hex == 0) return HEXVAL_OK;
  if (!corners || !sj_min) return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  Batch p{};
  p.n = n_hex;
  p.soa = corners;
  p.stride = n_hex;
  p.s = h->s;
  return hexval::launch_quality(p, sj_min, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? HEXVAL_OK
             : HEXVAL_E_CUDA;
}

int hexval_corner_quality_indexed(hexval_handle h, int64_t n_nodes, const double* nodes,
                                  int64_t n_hex, const int32_t* conn, float* sj_min,
                                  void* stream) {
  if (!h || n_hex < 0 || n_hex >= (1ll << 31) || n_nodes < 0 || n_nodes >= (1ll << 31))
    return HEXVAL_E_ARG;
  if (n_hex == 0) return HEXVAL_OK;
  if (!nodes || !conn || !sj_min || n_nodes == 0) return HEXVAL_E_ARG;
  if (reinterpret_cast<uintptr_t>(conn) % 16 != 0) return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  Batch p{};
  p.n = n_hex;
  p.nodes = nodes;
  p.n_nodes = n_nodes;
  p.conn = conn;
  p.indexed = 1;
  p.s = h->s;
  return hexval::launch_quality(p, sj_min, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? HEXVAL_OK
             : HEXVAL_E_CUDA;
}

int hexval_compact(hexval_handle h, int64_t n, const uint8_t* flags, uint32_t verdict_mask,
                   int32_t* ids, int32_t* count, void* stream) {
  if (!h || n < 0 || n >= (1ll << 31) || !count || (verdict_mask & ~0xffu)) return HEXVAL_E_ARG;
  if (n > 0 && (!flags || !ids)) return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  return hexval::launch_compact(flags, n, verdict_mask, h->s.tiles, ids, count,
                                static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? HEXVAL_OK
             : HEXVAL_E_CUDA;
}

int hexval_min_jacobian(hexval_handle h, int64_t n_hex, const double* corners, double rel_tol,
                        int32_t max_depth, double* jmin_lo, double* jmin_hi, uint8_t* depth,
                        void* stream) {
  if (!h || n_hex < 0 || n_hex >= (1ll << 31) || !(rel_tol >= 0.0) || max_depth < 0 ||
      max_depth > hexval::kMaxDepth)
    return HEXVAL_E_ARG;
  if (n_hex == 0) return HEXVAL_OK;
  if (!corners || !jmin_lo || !jmin_hi || !depth) return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  Batch p{};
  p.n = n_hex;
  p.soa = corners;
  p.stride = n_hex;
  p.s = h->s;
  return hexval::launch_minj(p, rel_tol, max_depth, jmin_lo, jmin_hi, depth, &h->s.cnt->minj_next,
                             static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? HEXVAL_OK
             : HEXVAL_E_CUDA;
}

int hexval_min_jacobian_indexed(hexval_handle h, int64_t n_nodes, const double* nodes,
                                int64_t n_hex, const int32_t* conn, double rel_tol,
                                int32_t max_depth, double* jmin_lo, double* jmin_hi,
                                uint8_t* depth, void* stream) {
  if (!h || n_hex < 0 || n_hex >= (1ll << 31) || n_nodes < 0 || n_nodes >= (1ll << 31) ||
      !(rel_tol >= 0.0) || max_depth < 0 || max_depth > hexval::kMaxDepth)
    return HEXVAL_E_ARG;
  if (n_hex == 0) return HEXVAL_OK;
  if (!nodes || !conn || !jmin_lo || !jmin_hi || !depth || n_nodes == 0) return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  Batch p{};
  p.n = n_hex;
  p.nodes = nodes;
  p.n_nodes = n_nodes;
  p.conn = conn;
  p.indexed = 1;
  p.s = h->s;
  return hexval::launch_minj(p, rel_tol, max_depth, jmin_lo, jmin_hi, depth, &h->s.cnt->minj_next,
                             static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? HEXVAL_OK
             : HEXVAL_E_CUDA;
}

int hexval_copy_soa_range(double* dst, const double* src, int64_t n_src, int64_t first,
                          int64_t n, void* stream) {
  if (!dst || !src || n_src < 0 || first < 0 || n < 0 || first + n > n_src) return HEXVAL_E_ARG;
  if (n == 0) return HEXVAL_OK;
  const size_t width = static_cast<size_t>(n) * sizeof(double);
  return cudaMemcpy2DAsync(dst, width, src + first, static_cast<size_t>(n_src) * sizeof(double),
                           width, 24, cudaMemcpyDefault,
                           static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? HEXVAL_OK
             : HEXVAL_E_CUDA;
}

int hexval_scratch_bytes(hexval_handle h, uint64_t* bytes) {
  if (!h || !bytes) return HEXVAL_E_ARG;
  *bytes = h->scratch_bytes;
  return HEXVAL_OK;
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
  out->escalated_df = s.escalated_df;
  out->boxes_fp32 = s.boxes_fp32;
  out->redone_tail = s.redone_tail;
  out->partial_fp64 = s.partial_fp64;
  if (reset && cudaMemset(h->s.stats, 0, sizeof(s)) != cudaSuccess) return HEXVAL_E_CUDA;
  return HEXVAL_OK;
}

int hexval_profile_enable(hexval_handle h, int on) {
  if (!h) return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  Profiler& P = h->prof;
  if (on && !P.ev[0][0]) {
    for (int i = 0; i < Profiler::kPairs; ++i)
      if (cudaEventCreate(&P.ev[i][0]) != cudaSuccess ||
          cudaEventCreate(&P.ev[i][1]) != cudaSuccess)
        return HEXVAL_E_CUDA;
  }
  if (!on) prof_drain(P, 0);
  P.on = on != 0;
  return HEXVAL_OK;
}

int hexval_profile_read(hexval_handle h, hexval_profile* out, int reset) {
  if (!h || !out) return HEXVAL_E_ARG;
  if (set_device(h) != HEXVAL_OK) return HEXVAL_E_CUDA;
  prof_drain(h->prof, 0);
  *out = h->prof.acc;
  if (reset) h->prof.acc = hexval_profile{};
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
