/*
 * hexval.h -- C ABI of the GB300 (sm_103a) validity test of linear hexahedra.
 *
 * Method: Johnen, Weill & Remacle, "Robust and efficient validation of the
 * linear hexahedral element", IMR 2017.  For every hexahedron the library
 * evaluates the Jacobian determinant J at the 8 corners and 12 edge midpoints
 * (Sec. 5: triple products of edge vectors), maps them to the 27 Bezier
 * coefficients of the triquadratic J (Sec. 4, Table t:Tsmall), and classifies
 * the element (Sec. 6): a non-positive sample -> invalid; 27 positive
 * coefficients -> valid; otherwise the coefficients are refined by Bezier
 * subdivision (Sec. 3.1, Sec. 6) until the element is decided or the depth
 * cap is reached.
 *
 * Exactness: every sign decision is certified with a forward-error bound; a
 * decision the bound cannot settle is redone in higher precision (FP32 ->
 * FP64) and finally in exact integer arithmetic on the device (the element
 * at depth 0, or the one refinement box whose sign is uncertain), so the
 * verdicts are those of exact arithmetic on the FP64 inputs.
 *
 * Conventions shared by every entry point:
 *  - array arguments are DEVICE pointers owned by the caller (unless a name
 *    says _host); the library never frees them and never keeps them after
 *    the call has been enqueued;
 *  - calls are stream ordered and enqueue only: no host synchronisation and
 *    no device allocation (all scratch is owned by the handle, allocated in
 *    hexval_create); results are visible once the stream reaches them.  The
 *    one object a call may create is the replay graph of the check calls
 *    (see HEXVAL_OPT_NO_REPLAY), on the second identical call;
 *  - one handle must not be used by two streams at the same time (its
 *    scratch is shared by the calls made on it);
 *  - host-detectable errors return a negative code and enqueue nothing;
 *    device-detected errors (bad connectivity, exhausted work queue, range of
 *    the exact tier) never trap: they set a sticky status read back by
 *    hexval_status, and the affected elements get verdict UNDECIDED.
 */
#ifndef HEXVAL_H
#define HEXVAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hexval_ctx* hexval_handle;

/* return / status codes */
enum {
  HEXVAL_OK = 0,
  HEXVAL_E_ARG = -1,     /* bad argument (null pointer, negative size, ...) */
  HEXVAL_E_NOMEM = -2,   /* device allocation failed in hexval_create */
  HEXVAL_E_CUDA = -3,    /* a CUDA runtime call failed */
  HEXVAL_E_INDEX = -4,   /* device: connectivity entry outside [0, n_nodes) */
  HEXVAL_E_QUEUE = -5,   /* device: refinement queue or escalation list full */
  HEXVAL_E_TIMEOUT = -6, /* device: a bounded wait gave up */
  HEXVAL_E_RANGE = -7    /* device: element outside the exact tier's range */
};

/* precision of the bulk pass */
enum { HEXVAL_FP64 = 0, HEXVAL_FP32_FILTERED = 1 };

/* verdict in bits 0-2 of a flag byte; bits 3-6 hold the decision depth,
 * bit 7 marks an element that needed exact arithmetic: the exact tier, or an
 * exact check of one refinement box (diagnostic only) */
enum {
  HEXVAL_VALID = 1,     /* J > 0 on the whole element */
  HEXVAL_INVALID = 2,   /* J <= 0 somewhere */
  HEXVAL_UNDECIDED = 3, /* depth cap reached, or a device error (see status) */
  HEXVAL_NONFINITE = 4  /* a coordinate is NaN or infinite */
};

typedef struct {
  uint32_t struct_size;    /* sizeof(hexval_config): ABI versioning */
  int32_t device;          /* CUDA device ordinal */
  int32_t precision;       /* HEXVAL_FP64 or HEXVAL_FP32_FILTERED */
  int32_t max_depth;       /* refinement cap D, 0..15 (default 8) */
  uint64_t max_batch;      /* elements per internal batch (default 2^24) */
  uint64_t queue_capacity; /* boxes per refinement level (default 2^23) */
  uint64_t max_nodes;      /* node capacity of the FP32 indexed path (default 2^24) */
  uint64_t exact_capacity; /* elements per batch for the exact tier (default 2^16) */
  uint32_t options;        /* HEXVAL_OPT_* bits (default 0) */
  uint32_t bulk_threads;   /* threads per block of the bulk kernels: 0 (default: 256
                              for FP64, 128 for FP32), 64, 128 or 256 */
  uint32_t spin_limit;     /* polls of the tail kernel's grid barrier before it
                              gives up with HEXVAL_E_TIMEOUT (0: the default,
                              2^24, well over a second); a small value is for
                              testing the timeout path */
  uint32_t reserved;       /* must be 0 */
  /* work placement (tuning knobs; results do not depend on them): */
  uint32_t esc_in_pass;    /* FP32 form: per batch, the first esc_in_pass FP32
                              escalations are redone in FP64 inside the FP32
                              pass by whole warps, the others by the tail
                              kernel (default 4096) */
  uint32_t refine_in_pass; /* FP32 form: per batch, the first refine_in_pass
                              elements that need subdivision are redone and
                              refined in FP64 inside the FP32 pass, the others
                              refined in FP32 by the tail kernel (default 512) */
  uint32_t tail_warp_items; /* a step of the tail kernel with at most this many
                              items per warp runs one item per warp (latency),
                              a larger one one item per thread (throughput);
                              1..64 (default 8) */
  uint32_t reserved2;      /* must be 0 */
} hexval_config;

/* options (tuning knobs; the same flags, and with HEXVAL_OPT_DFREDO or
 * HEXVAL_OPT_PARTIAL64 the bmin / bmax of the escalated elements they decide
 * carry double-float or FP32 error instead of FP64's):
 *  HEXVAL_OPT_PAIR32   the FP32 bulk pass with two elements per thread in
 *                      packed f32x2 arithmetic instead of one per thread;
 *  HEXVAL_OPT_PREFETCH the indexed FP32 bulk pass on a persistent grid that
 *                      stages its inputs through shared memory with
 *                      asynchronous copies: connectivity two tiles ahead,
 *                      node records one tile ahead (ignored with
 *                      HEXVAL_OPT_PAIR32);
 *  HEXVAL_OPT_LEVEL1   FP32 form: the elements listed for the FP32
 *                      refinement get their first refinement level (split
 *                      of the root box, classification of the 8 children,
 *                      Sec. 6) in a full-occupancy kernel of its own, one
 *                      element per thread, before the tail; only elements
 *                      that need deeper levels, or meet a sign FP32 cannot
 *                      settle, go on to the tail's refinement.  Pays when
 *                      many elements are decided on level 1 (boundary
 *                      layers);
 *  HEXVAL_OPT_PARTIAL64  FP32 form: each escalation the FP32 pass lists is
 *                      first redone in part, one per thread in a kernel of
 *                      its own: its FP32 classification is recomputed, and
 *                      only the samples and edge coefficients FP32 left
 *                      unsettled are evaluated in FP64, with the full
 *                      evaluation's bound; a sample certainly <= 0 makes the
 *                      element INVALID, everything certainly positive VALID
 *                      (bmin / bmax then FP32), and whatever this cannot
 *                      decide is redone in full by the tail.  Pays when
 *                      escalations turn on few signs (near-degenerate
 *                      corners); same verdicts.  Not with HEXVAL_OPT_DFREDO
 *                      (hexval_create returns HEXVAL_E_ARG);
 *  HEXVAL_OPT_DFREDO   FP32 form: the escalations the FP32 pass leaves are
 *                      first redone in double-float (pairs of FP32 values,
 *                      about 44 bits, at FP32 throughput) by a kernel of its
 *                      own; those it decides at depth 0 are final (bmin/bmax
 *                      within (2^-31 L + 2^-38 X) L^2 of the exact values, L
 *                      the largest edge-vector component, X the largest
 *                      |coordinate|), the rest go on to FP64.  Pays for one
 *                      more launch per batch; worth it when many elements
 *                      escalate (near-degenerate meshes);
 *  HEXVAL_OPT_NO_REPLAY every check call launched directly.  By default a
 *                      check call identical to the previous one on the
 *                      handle (entry point, pointers, sizes), made with
 *                      profiling off on a stream that is not capturing, is
 *                      captured once into a CUDA graph (on a private
 *                      stream) that further identical calls launch: one
 *                      launch per call instead of three or more.  The
 *                      capture itself costs one host-side graph build. */
enum {
  HEXVAL_OPT_PAIR32 = 1,
  HEXVAL_OPT_PREFETCH = 2,
  HEXVAL_OPT_DFREDO = 4,
  HEXVAL_OPT_NO_REPLAY = 8,
  HEXVAL_OPT_LEVEL1 = 16,
  HEXVAL_OPT_PARTIAL64 = 32
};

typedef struct {
  uint64_t elements;        /* elements processed since the last reset */
  uint64_t escalated_fp64;  /* FP32 decisions redone at higher precision
                               (double-float or FP64) */
  uint64_t refined;         /* elements that needed subdivision */
  uint64_t boxes;           /* boxes split by the refinement (root boxes
                               included; boxes of elements settled on an
                               earlier level are skipped, not counted; the
                               in-warp FP64 refinement of the FP32 pass is
                               not counted) */
  uint64_t exact;           /* elements decided by the exact tier */
  uint64_t max_level_boxes; /* largest refinement level (boxes) */
  uint64_t escalated_df;    /* of escalated_fp64: decided in double-float
                               (pairs of FP32 values, about 44 bits) */
  uint64_t boxes_fp32;      /* of boxes: split by the FP32 refinement */
  uint64_t redone_tail;     /* elements redone in FP64 by the tail kernel
                               (escalations the FP32 pass left) */
  uint64_t partial_fp64;    /* of escalated_fp64: decided by the partial
                               FP64 redo (HEXVAL_OPT_PARTIAL64) */
} hexval_stats;

/* Fills *cfg with the defaults listed above. */
int hexval_config_default(hexval_config* cfg);

/* Creates a handle on cfg->device and allocates all of its device scratch
 * (about 485 B x queue_capacity + 16 B x max_nodes + 4 B x max_batch + 40 MB,
 * ~4.4 GB with the defaults; the FP32-filtered form adds about 225 B x
 * queue_capacity + 36 B x max_batch, ~2.5 GB).  Returns HEXVAL_E_NOMEM if
 * that fails. */
int hexval_create(const hexval_config* cfg, hexval_handle* out);

/* Frees the handle's scratch (synchronises its device). */
int hexval_destroy(hexval_handle h);

/* Copies the elements [first, first + n) of SoA corner planes src (24 planes
 * of n_src values each, laid out as for hexval_check_soa; host -- pinned for
 * an asynchronous copy -- or device memory) into dst, 24 planes of n values
 * (device), with one strided copy on `stream`.  For feeding element ranges
 * of a large input to hexval_check_soa (a server cutting requests, a caller
 * overlapping copies with checks) without a host-side gather.  Not from the
 * paper: data movement of this library.  Stream-ordered, no allocation;
 * HEXVAL_E_ARG for a range outside [0, n_src). */
int hexval_copy_soa_range(double* dst, const double* src, int64_t n_src, int64_t first,
                          int64_t n, void* stream);

/* Device bytes the handle holds (the scratch allocated by hexval_create),
 * for callers that budget device memory, such as a server admitting
 * requests next to a set of handles.  Not from the paper: bookkeeping of
 * this library.  Host only; no synchronisation. */
int hexval_scratch_bytes(hexval_handle h, uint64_t* bytes);

/* Independent elements.
 *   corners: FP64, n_hex*24 values laid out as 24 planes [8][3][n_hex]: value
 *            (k, d, e) at corners[(3*k + d)*n_hex + e] is coordinate d (x,y,z)
 *            of node k (node order of Appendix A) of element e;
 *   flags:   n_hex bytes (verdict | depth << 3 | exact << 7);
 *   bmin, bmax: n_hex FP64 each, the min / max of the element's 27 depth-0
 *            Bezier coefficients (FP32-accurate for elements the FP32 bulk
 *            pass decided); either may be NULL;
 *   stream:  a cudaStream_t (NULL = legacy default stream).
 * n_hex may be 0 (nothing is enqueued) and must be < 2^31. */
int hexval_check_soa(hexval_handle h, int64_t n_hex, const double* corners, uint8_t* flags,
                     double* bmin, double* bmax, void* stream);

/* Elements of an indexed mesh.
 *   nodes: FP64 [n_nodes][3] (x, y, z of each node);
 *   conn:  int32 [n_hex][8], 0-based node ids in Appendix A order.
 * An entry outside [0, n_nodes) gives that element verdict UNDECIDED and the
 * sticky status HEXVAL_E_INDEX.  Other arguments as hexval_check_soa.  With
 * HEXVAL_FP32_FILTERED, n_nodes must not exceed the handle's max_nodes. */
int hexval_check_indexed(hexval_handle h, int64_t n_nodes, const double* nodes, int64_t n_hex,
                         const int32_t* conn, uint8_t* flags, double* bmin, double* bmax,
                         void* stream);

/* The same check in two steps, for many calls on one node array (an indexed
 * mesh checked in ranges of elements whose copies overlap the checks, or
 * candidate element sets sharing one node array): hexval_prepare_nodes
 * records the node array on the handle and, with HEXVAL_FP32_FILTERED,
 * enqueues its conversion to the handle's FP32 node records (once);
 * hexval_check_indexed_prepared then checks n_hex elements (conn as in
 * hexval_check_indexed, any range of the mesh's rows) against it, without
 * converting the nodes again.  Results are those of hexval_check_indexed on
 * the same nodes and rows.  Not from the paper: a data-movement step of
 * this library.  The caller keeps the node array unchanged and orders the
 * prepare call before the checks (same stream, or an event); a later
 * hexval_check_indexed on the handle replaces the FP32 node records, after
 * which hexval_check_indexed_prepared returns HEXVAL_E_ARG until the next
 * prepare.  Argument rules as hexval_check_indexed. */
int hexval_prepare_nodes(hexval_handle h, int64_t n_nodes, const double* nodes, void* stream);
int hexval_check_indexed_prepared(hexval_handle h, int64_t n_hex, const int32_t* conn,
                                  uint8_t* flags, double* bmin, double* bmax, void* stream);

/* Validity of linear quadrangles (Sec. 2.1, Eq. e:determinant2D): the
 * Jacobian determinant of the bilinear map is bilinear, so the element is
 * valid iff its values at the four corners are all positive (strictly).
 * Nodes 1..4 at reference (0,0), (1,0), (1,1), (0,1).
 *
 * corners: device, FP64, planes [4][2][n_quad] (plane 2k + d = coordinate d
 * of node k).  flags: device, n_quad bytes, verdict VALID / INVALID /
 * NONFINITE (or UNDECIDED with status HEXVAL_E_RANGE when an exact test is
 * needed on coordinates spanning more than 120 bits), depth 0, bit 7 set
 * when the exact test decided.  jmin / jmax (device, may be NULL): min / max
 * of the four corner values (FP32-accurate for elements decided by the FP32
 * filter of a HEXVAL_FP32_FILTERED handle, else FP64).  The handle's
 * precision selects the form; the flags are the exact-arithmetic ones in
 * both.  Stream-ordered, no allocation; errors as hexval_check_soa. */
int hexval_check_quads(hexval_handle h, int64_t n_quad, const double* corners, uint8_t* flags,
                       double* jmin, double* jmax, void* stream);

/* The same for an indexed 2D mesh: nodes [n_nodes][2] FP64 and conn
 * [n_quad][4] int32 (0-based, node order as above), both device and 16-byte
 * aligned (else HEXVAL_E_ARG).  An out-of-range entry gives that element
 * UNDECIDED with NaN jmin / jmax and the sticky status HEXVAL_E_INDEX. */
int hexval_check_quads_indexed(hexval_handle h, int64_t n_nodes, const double* nodes,
                               int64_t n_quad, const int32_t* conn, uint8_t* flags, double* jmin,
                               double* jmax, void* stream);

/* Corner scaled Jacobian, the quality measure quoted in Sec. 7 (Fig.
 * f:invalidHighCornerQual): per element the minimum over its 8 corners of
 * the determinant of the three edge vectors leaving the corner, each
 * divided by its length (0 at a corner with a zero-length edge; in [-1, 1]).
 * It is not a validity test: the figure shows an invalid element whose
 * value is 0.64.
 *
 * corners: device FP64 planes [8][3][n_hex] as for hexval_check_soa.
 * sj_min: device, n_hex floats; NaN for non-finite input.  Computed in FP32
 * from the coordinates relative to node 1 (formed in FP64 and scaled by a
 * power of two), so it does not depend on where the element sits; error
 * about 1e-6 for elements of moderate aspect ratio.  Independent of the
 * handle's precision.  Stream-ordered, no allocation. */
int hexval_corner_quality(hexval_handle h, int64_t n_hex, const double* corners, float* sj_min,
                          void* stream);

/* The same on an indexed mesh (nodes [n_nodes][3] FP64, conn [n_hex][8]
 * int32, 16-byte aligned); an out-of-range entry gives NaN and the sticky
 * status HEXVAL_E_INDEX. */
int hexval_corner_quality_indexed(hexval_handle h, int64_t n_nodes, const double* nodes,
                                  int64_t n_hex, const int32_t* conn, float* sj_min,
                                  void* stream);

/* Stream compaction by verdict, for candidate filtering (the paper's
 * motivating use, Sec. 1: indirect hex-dominant meshing builds candidate
 * hexahedra, many more than there are vertices, and keeps the valid ones).
 * Writes to ids (device, capacity n) the indices i, in ascending order, whose
 * verdict flags[i] & 7 has its bit set in verdict_mask (bit 1 = VALID, bit 2
 * = INVALID, ...), and their number to *count (device).  flags: device, n
 * bytes (the output of a check).  n < 2^31.  Stream-ordered, no allocation
 * (the tile sums live in the handle); errors as hexval_check_soa. */
int hexval_compact(hexval_handle h, int64_t n, const uint8_t* flags, uint32_t verdict_mask,
                   int32_t* ids, int32_t* count, void* stream);

/* Minimum of the Jacobian determinant to a tolerance (Sec. 1 and Sec. 3:
 * the smallest Bezier coefficient of a box bounds J from below on it, its
 * smallest corner coefficient bounds the minimum from above, and
 * subdividing sharpens both).  Per element, breadth first: boxes whose lower
 * bound is below U - tol are split in 8, until U - L <= tol with
 * tol = rel_tol * max |b| (b the 27 depth-0 coefficients) or max_depth
 * levels; every value carries a certified FP64 error bound, so the true
 * minimum of J over the reference cube lies in [jmin_lo, jmin_hi].
 *
 * corners: as for hexval_check_soa.  jmin_lo, jmin_hi: device, n_hex
 * doubles (NaN for non-finite input).  depth: device, n_hex bytes, the levels
 * used, bit 7 set when the tolerance was not reached (depth cap, or more
 * boxes on a level than the element's share of the handle's queue).
 * 0 <= max_depth <= 15, rel_tol >= 0.  Stream-ordered, no allocation (the
 * boxes live in the handle's refinement queue); errors as hexval_check_soa. */
int hexval_min_jacobian(hexval_handle h, int64_t n_hex, const double* corners, double rel_tol,
                        int32_t max_depth, double* jmin_lo, double* jmin_hi, uint8_t* depth,
                        void* stream);

/* The same on an indexed mesh (nodes [n_nodes][3] FP64, conn [n_hex][8]
 * int32); an out-of-range entry gives NaN bounds and HEXVAL_E_INDEX. */
int hexval_min_jacobian_indexed(hexval_handle h, int64_t n_nodes, const double* nodes,
                                int64_t n_hex, const int32_t* conn, double rel_tol,
                                int32_t max_depth, double* jmin_lo, double* jmin_hi,
                                uint8_t* depth, void* stream);

/* Synchronises the stream, returns the sticky device status (HEXVAL_OK or
 * the most severe device-detected code) and clears it.  After
 * HEXVAL_E_TIMEOUT the batch that timed out is incomplete: its blocks stopped
 * their work at the barrier (elements not yet decided keep whatever their
 * flags held), while the batch counters were still folded and reset, so the
 * handle stays usable. */
int hexval_status(hexval_handle h, void* stream);

/* Synchronises the stream and copies the counters; reset != 0 zeroes them. */
int hexval_get_stats(hexval_handle h, hexval_stats* out, int reset, void* stream);

/* Per-phase device time, measured with CUDA events recorded on the launch
 * stream around each kernel of the call sequence (diagnostic; adds a few
 * microseconds per call while enabled; do not enable during graph capture). */
enum {
  HEXVAL_PH_NODES32 = 0, /* FP64 nodes -> FP32 copy (FP32 form, indexed input) */
  HEXVAL_PH_BULK32 = 1,  /* FP32 bulk pass */
  HEXVAL_PH_BULK64 = 2,  /* FP64 bulk pass */
  HEXVAL_PH_TAIL = 3,    /* FP64 redo of FP32 escalations, refinement and
                            the exact tier (one launch) */
  HEXVAL_PH_EXACT = 4,   /* unused: the exact tier runs inside the tail */
  HEXVAL_PH_REDODF = 5,  /* double-float redo of escalations (HEXVAL_OPT_DFREDO) */
  HEXVAL_PH_LEVEL1 = 6,  /* first refinement level in its own kernel (HEXVAL_OPT_LEVEL1) */
  HEXVAL_PH_PARTIAL = 7, /* partial FP64 redo of escalations (HEXVAL_OPT_PARTIAL64) */
  HEXVAL_PH_COUNT = 8
};
typedef struct {
  double ms[HEXVAL_PH_COUNT];         /* accumulated device milliseconds */
  uint64_t launches[HEXVAL_PH_COUNT]; /* timed launches */
} hexval_profile;

/* Turns phase timing on (on != 0) or off for the handle. */
int hexval_profile_enable(hexval_handle h, int on);

/* Waits for the recorded events, copies the accumulated times; reset != 0
 * zeroes them. */
int hexval_profile_read(hexval_handle h, hexval_profile* out, int reset);

/* FP64 check of independent elements that allocates nothing, for callers
 * that cannot call cudaMalloc (for instance code running inside a host
 * callback or a driver layer that owns every allocation, or a process whose
 * device memory pool is fixed after start-up).  The paper has no counterpart:
 * this is a packaging of hexval_check_soa (FP64 form) for such callers.
 *
 * It needs no handle.  Its scratch (refinement queue with box positions,
 * exact-check list, refinement state, exact-tier list and stacks, counters,
 * status) is one static device array of about 48 MB that every device which
 * loads the library holds until the process exits; the kernels and the
 * arithmetic are those of hexval_check_soa on a FP64 handle, so flags
 * (exact bit included) and bounds are the same whenever no refinement level
 * exceeds the limit below on either side.  Limits: n_hex <= 16384 per
 * call (larger calls return HEXVAL_E_ARG and enqueue nothing); refinement
 * levels of at most 16384 boxes (more boxes send the elements concerned to
 * the exact tier, which settles them exactly; the call's status then has
 * bit 2 set although the flags are exact, unless the exact tier's list of
 * 16384 elements fills too, which leaves those elements UNDECIDED);
 * max_depth 0..15.  Arguments as hexval_check_soa; status_bits, if not
 * NULL, is a device word that receives the call's device-status bits (1 bad
 * index, 2 queue or list full, 4 bounded wait gave up, 8 exact-tier range),
 * written in stream order.
 *
 * Every call looks the array's device address up (cudaGetSymbolAddress);
 * the first call on a device, and the first after a device reset that
 * reloaded the library's module, also zeroes its counters on the caller's
 * stream.  Make that first call before any stream capture.  All calls share
 * the array and it keeps the last call's contents: calls whose work overlaps
 * on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  No cudaMalloc, cudaFree or allocating library
 * routine is called. */
int hexval_check_soa_noalloc(int64_t n_hex, const double* corners, uint8_t* flags, double* bmin,
                             double* bmax, int32_t max_depth, uint32_t* status_bits,
                             void* stream);

/* Static description of a code. */
const char* hexval_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* HEXVAL_H */
