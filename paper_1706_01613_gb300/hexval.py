"""Thin ctypes binding of libhexval (C ABI in include/hexval.h).

Argument marshalling only: every step of the validity test runs in the CUDA
kernels of the library.  PyTorch provides device memory and streams.  There is
no CPU fallback: if the library is missing or no GPU is present, the calls
raise.

    v = Validator(precision="fp32")          # or "fp64"
    flags, bmin, bmax = v.check_soa(corners)  # corners: (8, 3, n) float64 CUDA
    flags, bmin, bmax = v.check_indexed(nodes, conn)
    v.raise_on_status()                       # sticky device-side errors
"""
import ctypes
import os

from . import _build

HEXVAL_OK = 0
CODES = {0: "HEXVAL_OK", -1: "HEXVAL_E_ARG", -2: "HEXVAL_E_NOMEM", -3: "HEXVAL_E_CUDA",
         -4: "HEXVAL_E_INDEX", -5: "HEXVAL_E_QUEUE", -6: "HEXVAL_E_TIMEOUT",
         -7: "HEXVAL_E_RANGE"}
FP64, FP32_FILTERED = 0, 1
OPT_PAIR32 = 1    # hexval_config.options: packed f32x2 FP32 bulk pass
OPT_PREFETCH = 2  # hexval_config.options: persistent indexed FP32 pass with prefetch
OPT_DFREDO = 4    # hexval_config.options: double-float redo of FP32 escalations
OPT_NO_REPLAY = 8 # hexval_config.options: no graph replay of repeated check calls
OPT_LEVEL1 = 16   # hexval_config.options: first refinement level in a kernel of its own
OPT_PARTIAL64 = 32  # hexval_config.options: the unsettled signs of escalations redone in FP64 first
VALID, INVALID, UNDECIDED, NONFINITE = 1, 2, 3, 4

# every function declared in include/hexval.h (the CPU test checks the list)
EXPORTS = ("hexval_config_default", "hexval_create", "hexval_destroy", "hexval_check_soa",
           "hexval_check_indexed", "hexval_status", "hexval_get_stats", "hexval_profile_enable",
           "hexval_profile_read", "hexval_check_soa_noalloc", "hexval_check_quads",
           "hexval_check_quads_indexed", "hexval_corner_quality",
           "hexval_corner_quality_indexed", "hexval_compact", "hexval_min_jacobian",
           "hexval_min_jacobian_indexed", "hexval_strerror", "hexval_scratch_bytes",
           "hexval_copy_soa_range", "hexval_prepare_nodes", "hexval_check_indexed_prepared")
PHASES = ("nodes32", "bulk32", "bulk64", "tail", "-", "redo_df", "level1", "redo_partial")


class Config(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("device", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("max_batch", ctypes.c_uint64), ("queue_capacity", ctypes.c_uint64),
                ("max_nodes", ctypes.c_uint64), ("exact_capacity", ctypes.c_uint64),
                ("options", ctypes.c_uint32), ("bulk_threads", ctypes.c_uint32),
                ("spin_limit", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("esc_in_pass", ctypes.c_uint32), ("refine_in_pass", ctypes.c_uint32),
                ("tail_warp_items", ctypes.c_uint32), ("reserved2", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("elements", "escalated_fp64", "refined", "boxes", "exact", "max_level_boxes",
                 "escalated_df", "boxes_fp32", "redone_tail", "partial_fp64")]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_uint64 * 8)]


class HexvalError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s%s (%d: %s)" % (what + ": " if what else "", CODES.get(code, "?"),
                                            code, strerror(code)))


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=False):
    """Loads libhexval.so (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libhexval.so is not built (%s); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.hexval_config_default.argtypes = [ctypes.POINTER(Config)]
    lib.hexval_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
    lib.hexval_destroy.argtypes = [vp]
    lib.hexval_check_soa.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    lib.hexval_check_indexed.argtypes = [vp, i64, vp, i64, vp, vp, vp, vp, vp]
    lib.hexval_prepare_nodes.argtypes = [vp, i64, vp, vp]
    lib.hexval_check_indexed_prepared.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    lib.hexval_status.argtypes = [vp, vp]
    lib.hexval_scratch_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.hexval_copy_soa_range.argtypes = [vp, vp, i64, i64, i64, vp]
    lib.hexval_get_stats.argtypes = [vp, ctypes.POINTER(Stats), ctypes.c_int, vp]
    lib.hexval_profile_enable.argtypes = [vp, ctypes.c_int]
    lib.hexval_profile_read.argtypes = [vp, ctypes.POINTER(Profile), ctypes.c_int]
    lib.hexval_check_soa_noalloc.argtypes = [i64, vp, vp, vp, vp, ctypes.c_int32, vp, vp]
    lib.hexval_check_quads.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    lib.hexval_check_quads_indexed.argtypes = [vp, i64, vp, i64, vp, vp, vp, vp, vp]
    lib.hexval_corner_quality.argtypes = [vp, i64, vp, vp, vp]
    lib.hexval_corner_quality_indexed.argtypes = [vp, i64, vp, i64, vp, vp, vp]
    lib.hexval_compact.argtypes = [vp, i64, vp, ctypes.c_uint32, vp, vp, vp]
    f64 = ctypes.c_double
    lib.hexval_min_jacobian.argtypes = [vp, i64, vp, f64, ctypes.c_int32, vp, vp, vp, vp]
    lib.hexval_min_jacobian_indexed.argtypes = [vp, i64, vp, i64, vp, f64, ctypes.c_int32, vp,
                                                vp, vp, vp]
    lib.hexval_strerror.argtypes = [ctypes.c_int]
    lib.hexval_strerror.restype = ctypes.c_char_p
    _lib = lib
    return lib


def strerror(code):
    try:
        return load().hexval_strerror(int(code)).decode()
    except Exception:  # library not loadable: fall back to the code name
        return CODES.get(code, "?")


def default_config():
    cfg = Config()
    rc = load().hexval_config_default(ctypes.byref(cfg))
    if rc != HEXVAL_OK:
        raise HexvalError(rc, "hexval_config_default")
    return cfg


def _check(rc, what):
    if rc != HEXVAL_OK:
        raise HexvalError(rc, what)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Validator:
    """One library handle (its device scratch is allocated here).

    precision: "fp64" (plain FP64 bulk pass) or "fp32" (FP32-filtered bulk
    pass with certified escalation).  The remaining keywords override fields
    of the default configuration (max_depth, queue_capacity, max_batch,
    max_nodes, exact_capacity, bulk_threads, esc_in_pass, refine_in_pass,
    tail_warp_items, options = OPT_* bits: PAIR32, PREFETCH, DFREDO,
    NO_REPLAY, LEVEL1, PARTIAL64).  Repeated identical check calls are
    replayed from a CUDA graph unless NO_REPLAY is set."""

    def __init__(self, precision="fp64", max_depth=8, device=None, **caps):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("hexval needs a CUDA device")
        lib = load()
        cfg = default_config()
        cfg.device = torch.cuda.current_device() if device is None else int(device)
        cfg.precision = {"fp64": FP64, "fp32": FP32_FILTERED}[precision]
        cfg.max_depth = int(max_depth)
        for k, v in caps.items():
            setattr(cfg, k, int(v))
        self.config = cfg
        self.precision = precision
        self.device = torch.device("cuda", cfg.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.hexval_create(ctypes.byref(cfg), ctypes.byref(h)), "hexval_create")
        self._h = h
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hexval_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ calls ----
    def _outputs(self, n, out):
        import torch
        if out is not None:
            return out
        return (torch.empty(n, dtype=torch.uint8, device=self.device),
                torch.empty(n, dtype=torch.float64, device=self.device),
                torch.empty(n, dtype=torch.float64, device=self.device))

    @staticmethod
    def _ptr(t):
        return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p()

    def check_soa(self, corners, out=None, stream=None):
        """corners: contiguous float64 CUDA tensor (8, 3, n).  Returns
        (flags uint8, bmin float64, bmax float64), enqueued on `stream`
        (default: the current stream).  `out` = preallocated triple (bmin
        and bmax may be None)."""
        import torch
        if corners.dtype != torch.float64 or not corners.is_cuda or not corners.is_contiguous():
            raise ValueError("corners must be a contiguous float64 CUDA tensor (8, 3, n)")
        if corners.dim() != 3 or tuple(corners.shape[:2]) != (8, 3):
            raise ValueError("corners must have shape (8, 3, n)")
        n = corners.shape[2]
        flags, bmin, bmax = self._outputs(n, out)
        rc = self._lib.hexval_check_soa(self._h, n, self._ptr(corners), self._ptr(flags),
                                        self._ptr(bmin), self._ptr(bmax), _stream_ptr(stream))
        _check(rc, "hexval_check_soa")
        return flags, bmin, bmax

    def check_indexed(self, nodes, conn, out=None, stream=None):
        """nodes: float64 CUDA (n_nodes, 3); conn: int32 CUDA (n_hex, 8)."""
        import torch
        if nodes.dtype != torch.float64 or not nodes.is_cuda or not nodes.is_contiguous():
            raise ValueError("nodes must be a contiguous float64 CUDA tensor (n_nodes, 3)")
        if conn.dtype != torch.int32 or not conn.is_cuda or not conn.is_contiguous():
            raise ValueError("conn must be a contiguous int32 CUDA tensor (n_hex, 8)")
        if nodes.dim() != 2 or nodes.shape[1] != 3 or conn.dim() != 2 or conn.shape[1] != 8:
            raise ValueError("bad shapes")
        n = conn.shape[0]
        flags, bmin, bmax = self._outputs(n, out)
        rc = self._lib.hexval_check_indexed(self._h, nodes.shape[0], self._ptr(nodes), n,
                                            self._ptr(conn), self._ptr(flags), self._ptr(bmin),
                                            self._ptr(bmax), _stream_ptr(stream))
        _check(rc, "hexval_check_indexed")
        return flags, bmin, bmax

    def prepare_nodes(self, nodes, stream=None):
        """Records `nodes` (float64 CUDA (n_nodes, 3)) for check_indexed_prepared
        and, in the FP32 form, converts them once.  The tensor must stay
        alive and unchanged while it is used."""
        import torch
        if nodes.dtype != torch.float64 or not nodes.is_cuda or not nodes.is_contiguous() or \
                nodes.dim() != 2 or nodes.shape[1] != 3:
            raise ValueError("nodes must be a contiguous float64 CUDA tensor (n_nodes, 3)")
        _check(self._lib.hexval_prepare_nodes(self._h, nodes.shape[0], self._ptr(nodes),
                                              _stream_ptr(stream)), "hexval_prepare_nodes")
        self._prepared = nodes  # kept alive with the handle's record of it

    def check_indexed_prepared(self, conn, out=None, stream=None):
        """check_indexed of rows conn (int32 CUDA (n, 8)) on the nodes of the
        last prepare_nodes."""
        import torch
        if conn.dtype != torch.int32 or not conn.is_cuda or not conn.is_contiguous() or \
                conn.dim() != 2 or conn.shape[1] != 8:
            raise ValueError("conn must be a contiguous int32 CUDA tensor (n_hex, 8)")
        n = conn.shape[0]
        flags, bmin, bmax = self._outputs(n, out)
        rc = self._lib.hexval_check_indexed_prepared(self._h, n, self._ptr(conn), self._ptr(flags),
                                                     self._ptr(bmin), self._ptr(bmax),
                                                     _stream_ptr(stream))
        _check(rc, "hexval_check_indexed_prepared")
        return flags, bmin, bmax

    def check_quads(self, corners, out=None, stream=None):
        """Linear quadrangles: corners contiguous float64 CUDA (4, 2, n).
        Returns (flags uint8, jmin float64, jmax float64)."""
        import torch
        if corners.dtype != torch.float64 or not corners.is_cuda or not corners.is_contiguous():
            raise ValueError("corners must be a contiguous float64 CUDA tensor (4, 2, n)")
        if corners.dim() != 3 or tuple(corners.shape[:2]) != (4, 2):
            raise ValueError("corners must have shape (4, 2, n)")
        n = corners.shape[2]
        flags, jmin, jmax = self._outputs(n, out)
        rc = self._lib.hexval_check_quads(self._h, n, self._ptr(corners), self._ptr(flags),
                                          self._ptr(jmin), self._ptr(jmax), _stream_ptr(stream))
        _check(rc, "hexval_check_quads")
        return flags, jmin, jmax

    def check_quads_indexed(self, nodes, conn, out=None, stream=None):
        """nodes: float64 CUDA (n_nodes, 2); conn: int32 CUDA (n_quad, 4)."""
        import torch
        if nodes.dtype != torch.float64 or not nodes.is_cuda or not nodes.is_contiguous():
            raise ValueError("nodes must be a contiguous float64 CUDA tensor (n_nodes, 2)")
        if conn.dtype != torch.int32 or not conn.is_cuda or not conn.is_contiguous():
            raise ValueError("conn must be a contiguous int32 CUDA tensor (n_quad, 4)")
        if nodes.dim() != 2 or nodes.shape[1] != 2 or conn.dim() != 2 or conn.shape[1] != 4:
            raise ValueError("bad shapes")
        n = conn.shape[0]
        flags, jmin, jmax = self._outputs(n, out)
        rc = self._lib.hexval_check_quads_indexed(self._h, nodes.shape[0], self._ptr(nodes), n,
                                                  self._ptr(conn), self._ptr(flags),
                                                  self._ptr(jmin), self._ptr(jmax),
                                                  _stream_ptr(stream))
        _check(rc, "hexval_check_quads_indexed")
        return flags, jmin, jmax

    def corner_quality(self, corners, out=None, stream=None):
        """Minimum corner scaled Jacobian of each element; corners as for
        check_soa.  Returns a float32 CUDA tensor (n,)."""
        import torch
        if corners.dtype != torch.float64 or not corners.is_cuda or not corners.is_contiguous():
            raise ValueError("corners must be a contiguous float64 CUDA tensor (8, 3, n)")
        if corners.dim() != 3 or tuple(corners.shape[:2]) != (8, 3):
            raise ValueError("corners must have shape (8, 3, n)")
        n = corners.shape[2]
        sj = out if out is not None else torch.empty(n, dtype=torch.float32, device=corners.device)
        rc = self._lib.hexval_corner_quality(self._h, n, self._ptr(corners), self._ptr(sj),
                                             _stream_ptr(stream))
        _check(rc, "hexval_corner_quality")
        return sj

    def corner_quality_indexed(self, nodes, conn, out=None, stream=None):
        """Minimum corner scaled Jacobian on an indexed mesh (float32 (n,))."""
        import torch
        if nodes.dtype != torch.float64 or conn.dtype != torch.int32 or not nodes.is_cuda \
                or not conn.is_cuda or not nodes.is_contiguous() or not conn.is_contiguous():
            raise ValueError("nodes: contiguous float64 CUDA (n_nodes, 3); conn: int32 (n, 8)")
        n = conn.shape[0]
        sj = out if out is not None else torch.empty(n, dtype=torch.float32, device=nodes.device)
        rc = self._lib.hexval_corner_quality_indexed(self._h, nodes.shape[0], self._ptr(nodes), n,
                                                     self._ptr(conn), self._ptr(sj),
                                                     _stream_ptr(stream))
        _check(rc, "hexval_corner_quality_indexed")
        return sj

    def compact(self, flags, verdicts=(VALID,), out=None, stream=None):
        """Ids (int32, ascending) of the elements whose verdict is in
        `verdicts`, enqueued on `stream`.  Returns (ids buffer of len(flags),
        count as a one-element int32 CUDA tensor); ids[:count] are valid."""
        import torch
        if flags.dtype != torch.uint8 or not flags.is_cuda or not flags.is_contiguous():
            raise ValueError("flags must be a contiguous uint8 CUDA tensor")
        n = flags.numel()
        ids, count = out if out is not None else (
            torch.empty(max(n, 1), dtype=torch.int32, device=flags.device),
            torch.empty(1, dtype=torch.int32, device=flags.device))
        mask = 0
        for v in verdicts:
            mask |= 1 << int(v)
        rc = self._lib.hexval_compact(self._h, n, self._ptr(flags), mask, self._ptr(ids),
                                      self._ptr(count), _stream_ptr(stream))
        _check(rc, "hexval_compact")
        return ids, count

    def filter_valid(self, nodes, conn, stream=None):
        """Candidate filtering: checks every candidate of an indexed set and
        returns the ids of the valid ones (synchronises to read the count)."""
        flags, _, _ = self.check_indexed(nodes, conn, out=self._outputs(conn.shape[0], None)[:1]
                                         + (None, None), stream=stream)
        ids, count = self.compact(flags, stream=stream)
        if stream is not None:
            stream.synchronize()
        return ids[:int(count.item())]

    def min_jacobian(self, corners, rel_tol=1e-6, max_depth=12, stream=None):
        """Certified bounds (lo, hi) of the minimum of J of each element
        (corners as for check_soa) and the levels used (uint8, bit 7 = the
        tolerance was not reached)."""
        import torch
        if corners.dtype != torch.float64 or not corners.is_cuda or not corners.is_contiguous():
            raise ValueError("corners must be a contiguous float64 CUDA tensor (8, 3, n)")
        if corners.dim() != 3 or tuple(corners.shape[:2]) != (8, 3):
            raise ValueError("corners must have shape (8, 3, n)")
        n = corners.shape[2]
        lo = torch.empty(n, dtype=torch.float64, device=corners.device)
        hi = torch.empty_like(lo)
        depth = torch.empty(n, dtype=torch.uint8, device=corners.device)
        rc = self._lib.hexval_min_jacobian(self._h, n, self._ptr(corners), float(rel_tol),
                                           int(max_depth), self._ptr(lo), self._ptr(hi),
                                           self._ptr(depth), _stream_ptr(stream))
        _check(rc, "hexval_min_jacobian")
        return lo, hi, depth

    def min_jacobian_indexed(self, nodes, conn, rel_tol=1e-6, max_depth=12, stream=None):
        """As min_jacobian on an indexed mesh."""
        import torch
        if nodes.dtype != torch.float64 or conn.dtype != torch.int32 or not nodes.is_cuda \
                or not conn.is_cuda or not nodes.is_contiguous() or not conn.is_contiguous():
            raise ValueError("nodes: contiguous float64 CUDA (n_nodes, 3); conn: int32 (n, 8)")
        n = conn.shape[0]
        lo = torch.empty(n, dtype=torch.float64, device=nodes.device)
        hi = torch.empty_like(lo)
        depth = torch.empty(n, dtype=torch.uint8, device=nodes.device)
        rc = self._lib.hexval_min_jacobian_indexed(self._h, nodes.shape[0], self._ptr(nodes), n,
                                                   self._ptr(conn), float(rel_tol),
                                                   int(max_depth), self._ptr(lo), self._ptr(hi),
                                                   self._ptr(depth), _stream_ptr(stream))
        _check(rc, "hexval_min_jacobian_indexed")
        return lo, hi, depth

    def host_pipeline(self, kind, *arrays, chunks=4):
        """A HostPipeline of this handle on pinned host inputs (see there)."""
        return HostPipeline(self, kind, *arrays, chunks=chunks)

    def check_host(self, kind, *arrays, chunks=4, stream=None):
        """End-to-end call on host data: pinned host inputs in, pinned host
        outputs (flags, bmin, bmax) back.  kind = "soa" (corners) or
        "indexed" (nodes, conn).  The elements are split into `chunks`
        consecutive ranges whose copies overlap the work on the others:
        host-to-device copies on one stream, the checks on `stream` (default:
        the current stream), device-to-host copies on a third; `stream` waits
        for the last copy, so an event recorded on it after this call marks
        the outputs as ready.  An indexed mesh copies all its nodes first
        (every range may use any node) and prepares them once
        (prepare_nodes)."""
        import torch
        dev = self.device
        main = stream if stream is not None else torch.cuda.current_stream(dev)
        if not hasattr(self, "_copy_streams"):
            self._copy_streams = (torch.cuda.Stream(dev), torch.cuda.Stream(dev))
        cin, cout = self._copy_streams
        cin.wait_stream(main)
        n = arrays[0].shape[2] if kind == "soa" else arrays[1].shape[0]
        host = (torch.empty(n, dtype=torch.uint8, pin_memory=True),
                torch.empty(n, dtype=torch.float64, pin_memory=True),
                torch.empty(n, dtype=torch.float64, pin_memory=True))
        with torch.cuda.stream(main):
            out = (torch.empty(n, dtype=torch.uint8, device=dev),
                   torch.empty(n, dtype=torch.float64, device=dev),
                   torch.empty(n, dtype=torch.float64, device=dev))
        for t in out:  # read by the device-to-host stream too
            t.record_stream(cout)
        k = max(1, min(int(chunks), n))
        bounds = [n * i // k for i in range(k + 1)]
        with torch.cuda.stream(cin):
            if kind == "indexed":
                nodes = arrays[0].to(dev, non_blocking=True)
                conn = torch.empty(arrays[1].shape, dtype=arrays[1].dtype, device=dev)
                nodes.record_stream(main)  # used by the checks on `main`
                conn.record_stream(main)
        if kind == "indexed":  # the nodes are converted once for all ranges
            main.wait_stream(cin)
            self.prepare_nodes(nodes, stream=main)
        for i in range(k):
            lo, hi = bounds[i], bounds[i + 1]
            if hi == lo:
                continue
            with torch.cuda.stream(cin):
                if kind == "indexed":
                    conn[lo:hi].copy_(arrays[1][lo:hi], non_blocking=True)
                else:
                    X = torch.empty((8, 3, hi - lo), dtype=torch.float64, device=dev)
                    X.record_stream(main)
                    copy_soa_range(X, arrays[0], lo, stream=cin)
            main.wait_stream(cin)
            o = tuple(t[lo:hi] for t in out)
            if kind == "indexed":
                self.check_indexed_prepared(conn[lo:hi], out=o, stream=main)
            else:
                self.check_soa(X, out=o, stream=main)
            cout.wait_stream(main)
            with torch.cuda.stream(cout):
                for h, d in zip(host, o):
                    h[lo:hi].copy_(d, non_blocking=True)
        main.wait_stream(cout)
        return host

    def scratch_bytes(self):
        """Device bytes held by this handle's scratch."""
        out = ctypes.c_uint64()
        _check(self._lib.hexval_scratch_bytes(self._h, ctypes.byref(out)), "hexval_scratch_bytes")
        return int(out.value)

    def status(self, stream=None):
        """Synchronises and returns (and clears) the sticky device status."""
        return self._lib.hexval_status(self._h, _stream_ptr(stream))

    def raise_on_status(self, stream=None):
        rc = self.status(stream)
        if rc != HEXVAL_OK:
            raise HexvalError(rc, "device status")

    def profile(self, on=True):
        """Per-phase CUDA-event timing on the launch stream (diagnostic)."""
        _check(self._lib.hexval_profile_enable(self._h, int(bool(on))), "hexval_profile_enable")

    def profile_read(self, reset=False):
        """{phase: (milliseconds, launches)} accumulated while profiling."""
        p = Profile()
        _check(self._lib.hexval_profile_read(self._h, ctypes.byref(p), int(reset)),
               "hexval_profile_read")
        return {name: (p.ms[i], p.launches[i]) for i, name in enumerate(PHASES) if name != "-"}

    def stats(self, reset=False, stream=None):
        s = Stats()
        _check(self._lib.hexval_get_stats(self._h, ctypes.byref(s), int(reset),
                                          _stream_ptr(stream)), "hexval_get_stats")
        return {k: getattr(s, k) for k, _ in Stats._fields_}


def copy_soa_range(dst, src, first, stream=None):
    """dst (8, 3, n) CUDA tensor <- the elements [first, first + n) of the SoA
    planes src (8, 3, N), host (pinned) or device, in one strided copy on
    `stream` (default: the current stream)."""
    n, N = dst.shape[2], src.shape[2]
    if (dst.dtype != src.dtype or not dst.is_cuda or not dst.is_contiguous()
            or not src.is_contiguous() or tuple(src.shape[:2]) != (8, 3)):
        raise ValueError("dst: contiguous CUDA (8, 3, n); src: contiguous (8, 3, N), same dtype")
    rc = load().hexval_copy_soa_range(ctypes.c_void_p(dst.data_ptr()),
                                      ctypes.c_void_p(src.data_ptr()), N, int(first), n,
                                      _stream_ptr(stream))
    _check(rc, "hexval_copy_soa_range")
    return dst


class HostPipeline:
    """End-to-end checks of one set of pinned host inputs, replayed from a
    CUDA graph.

    Validator.check_host issues every copy, wait and check from Python on
    each call; for a mesh checked again and again (its host buffers updated
    in place between runs) that host-side issue cost can exceed the copies.
    Here the whole sequence -- host-to-device copies of `chunks` element
    ranges on one stream, the checks of each range on a second as soon as
    its copy is done (indexed: the nodes first, prepared once), the
    device-to-host copies of flags, bmin and bmax on a third -- is recorded
    once into a CUDA graph; run() replays it, one launch.  Every run copies
    the current contents of the input buffers and overwrites the host
    outputs.  Device and host buffers are allocated here, once."""

    def __init__(self, validator, kind, *arrays, chunks=4):
        import torch
        if kind not in ("soa", "indexed"):
            raise ValueError("kind: soa or indexed")
        for a in arrays:
            if a.is_cuda or not a.is_pinned() or not a.is_contiguous():
                raise ValueError("inputs must be contiguous pinned host tensors")
        self.v, self.kind, self.arrays = validator, kind, arrays
        dev = validator.device
        n = arrays[0].shape[2] if kind == "soa" else arrays[1].shape[0]
        self.n = n
        k = max(1, min(int(chunks), n))
        self.bounds = [n * i // k for i in range(k + 1)]
        self.host = (torch.empty(n, dtype=torch.uint8, pin_memory=True),
                     torch.empty(n, dtype=torch.float64, pin_memory=True),
                     torch.empty(n, dtype=torch.float64, pin_memory=True))
        self.dev_out = (torch.empty(n, dtype=torch.uint8, device=dev),
                        torch.empty(n, dtype=torch.float64, device=dev),
                        torch.empty(n, dtype=torch.float64, device=dev))
        if kind == "indexed":
            self.nodes = torch.empty(arrays[0].shape, dtype=arrays[0].dtype, device=dev)
            self.conn = torch.empty(arrays[1].shape, dtype=arrays[1].dtype, device=dev)
        else:
            self.X = [torch.empty((8, 3, hi - lo), dtype=arrays[0].dtype, device=dev)
                      for lo, hi in zip(self.bounds[:-1], self.bounds[1:])]
        self.streams = (torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev))
        main = self.streams[0]
        main.wait_stream(torch.cuda.current_stream(dev))
        self._enqueue()  # once directly first: lazy initialisation stays out of the capture
        main.synchronize()
        validator.raise_on_status()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=main):
            self._enqueue()

    def _enqueue(self):
        import torch
        main, cin, cout = self.streams
        v = self.v
        cin.wait_stream(main)
        if self.kind == "indexed":
            with torch.cuda.stream(cin):
                self.nodes.copy_(self.arrays[0], non_blocking=True)
            main.wait_stream(cin)
            v.prepare_nodes(self.nodes, stream=main)
        for i, (lo, hi) in enumerate(zip(self.bounds[:-1], self.bounds[1:])):
            if hi == lo:
                continue
            with torch.cuda.stream(cin):
                if self.kind == "indexed":
                    self.conn[lo:hi].copy_(self.arrays[1][lo:hi], non_blocking=True)
                else:
                    copy_soa_range(self.X[i], self.arrays[0], lo, stream=cin)
            main.wait_stream(cin)
            o = tuple(t[lo:hi] for t in self.dev_out)
            if self.kind == "indexed":
                v.check_indexed_prepared(self.conn[lo:hi], out=o, stream=main)
            else:
                v.check_soa(self.X[i], out=o, stream=main)
            cout.wait_stream(main)
            with torch.cuda.stream(cout):
                for h, d in zip(self.host, o):
                    h[lo:hi].copy_(d, non_blocking=True)
        main.wait_stream(cout)

    def run(self, stream=None):
        """Replays the pipeline on `stream` (default: the current stream) and
        returns the pinned host outputs (flags, bmin, bmax), valid once the
        stream reaches this point."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.v.device)
        with torch.cuda.stream(s):
            self.graph.replay()
        return self.host


NOALLOC_MAX_HEX = 16384


def check_soa_noalloc(corners, out, max_depth=8, status_bits=None, stream=None):
    """FP64 check through the allocation-free entry point, for callers that
    cannot allocate device memory (no handle; at most 16384 elements per
    call).  `out` = the caller's (flags, bmin, bmax) CUDA tensors (bmin and
    bmax may be None); `status_bits` = optional int32 CUDA tensor of one
    element that receives the call's device-status bits."""
    lib = load()
    n = corners.shape[2]
    p = Validator._ptr
    rc = lib.hexval_check_soa_noalloc(n, p(corners), p(out[0]), p(out[1]), p(out[2]),
                                      int(max_depth), p(status_bits), _stream_ptr(stream))
    _check(rc, "hexval_check_soa_noalloc")
    return out


def verdict(flags):
    return flags & 7


def depth(flags):
    return (flags >> 3) & 15
