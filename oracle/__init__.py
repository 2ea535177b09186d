"""CPU oracle of the linear-hexahedron validity test (TEST INFRASTRUCTURE ONLY).

Plain FP64 C (``hexval_oracle.c``, loaded through ctypes) for the bulk of the
work, with the exact rational tier of ``exact.py`` for the elements whose
certified FP64 sign decisions are inconclusive.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
this package; the library never imports it and shares no code with it.

Layouts (the same as the library's, Appendix A node order):
  * SoA corners: float64 array of shape (8, 3, n), node-major then x/y/z;
  * indexed: nodes float64 (n_nodes, 3), conn int32 (n_hex, 8), 0-based.
Outputs: flags uint8 (bits 0-2 verdict, 3-6 depth, 7 exact tier used),
bmin/bmax float64 = min/max of the 27 depth-0 Bezier coefficients.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np

from . import exact

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hexval_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

VALID, INVALID, UNDECIDED, NONFINITE = 1, 2, 3, 4


def build(force=False):
    """Compile the C oracle with gcc (OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.oracle_check_soa.argtypes = [i64, vp, i32, i32, vp, vp, vp]
        lib.oracle_check_indexed.argtypes = [i64, vp, i64, vp, i32, i32, vp, vp, vp]
        lib.oracle_coefficients.argtypes = [vp, vp, vp]
        lib.oracle_subdivide.argtypes = [vp, vp]
        lib.oracle_jacobian.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.oracle_jacobian.restype = ctypes.c_double
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_coefficient_bounds.argtypes = [vp, vp, vp]
        lib.oracle_child_bound.argtypes = [ctypes.c_double, vp]
        lib.oracle_child_bound.restype = ctypes.c_double
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads():
    return _load().oracle_max_threads()


def _resolve_exact(flags, gather, max_depth):
    amb = np.nonzero(flags == 0x80)[0]
    for e in amb:
        flags[e] = exact.decide(gather(int(e)), max_depth)
    return flags


def check_soa(corners, max_depth=8, threads=1, exact_tier=True):
    """Verdicts of n independent elements given as (8, 3, n) float64 planes."""
    corners = np.ascontiguousarray(corners, dtype=np.float64)
    assert corners.ndim == 3 and corners.shape[:2] == (8, 3)
    n = corners.shape[2]
    flags = np.zeros(n, np.uint8)
    bmin = np.zeros(n, np.float64)
    bmax = np.zeros(n, np.float64)
    rc = _load().oracle_check_soa(n, _ptr(corners), max_depth, threads,
                                  _ptr(flags), _ptr(bmin), _ptr(bmax))
    if rc != 0:
        raise ValueError("oracle_check_soa: bad arguments (%d)" % rc)
    if exact_tier:
        _resolve_exact(flags, lambda e: corners[:, :, e], max_depth)
    return flags, bmin, bmax


def check_indexed(nodes, conn, max_depth=8, threads=1, exact_tier=True):
    """Verdicts of the elements of an indexed mesh."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    assert nodes.ndim == 2 and nodes.shape[1] == 3
    assert conn.ndim == 2 and conn.shape[1] == 8
    n = conn.shape[0]
    flags = np.zeros(n, np.uint8)
    bmin = np.zeros(n, np.float64)
    bmax = np.zeros(n, np.float64)
    rc = _load().oracle_check_indexed(nodes.shape[0], _ptr(nodes), n, _ptr(conn),
                                      max_depth, threads, _ptr(flags), _ptr(bmin),
                                      _ptr(bmax))
    if rc == -2:
        raise IndexError("connectivity entry out of range")
    if rc != 0:
        raise ValueError("oracle_check_indexed: bad arguments (%d)" % rc)
    if exact_tier:
        _resolve_exact(flags, lambda e: nodes[conn[e]], max_depth)
    return flags, bmin, bmax


def coefficients(X):
    """(c27, b27) of one element given as an (8, 3) array: the 27 samples of J
    at the order-2 nodes and the Bezier coefficients b = T c."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    assert X.shape == (8, 3)
    c = np.zeros(27)
    b = np.zeros(27)
    _load().oracle_coefficients(_ptr(X), _ptr(c), _ptr(b))
    return c, b


def coefficient_bounds(X):
    """(b27, eb27): depth-0 coefficients and their certified error bounds."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    b = np.zeros(27)
    eb = np.zeros(27)
    _load().oracle_coefficient_bounds(_ptr(X), _ptr(b), _ptr(eb))
    return b, eb


def child_bound(e_parent, b):
    """Certified error bound of the children of a box (see the C source)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    return _load().oracle_child_bound(float(e_parent), _ptr(b))


def subdivide(b):
    """The 8 children (8, 27) of a box given by its 27 coefficients."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros((8, 27))
    _load().oracle_subdivide(_ptr(b), _ptr(out))
    return out


def jacobian(X, xi):
    X = np.ascontiguousarray(X, dtype=np.float64)
    return _load().oracle_jacobian(_ptr(X), float(xi[0]), float(xi[1]), float(xi[2]))


def verdict(flags):
    return np.asarray(flags) & 7


def depth(flags):
    return (np.asarray(flags) >> 3) & 15
