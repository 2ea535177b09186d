"""The allocation-free FP64 entry point (for callers that cannot allocate
device memory) against the regular FP64 entry point, through the C ABI.

This file is collected last so that a failure here comes after every other
test has run.  It passes both alone in a fresh process and after the rest
of the suite (the static scratch is looked up on first use and keeps no
state that a later call depends on)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1706_01613_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1706_01613_gb300 import hexval as hv  # noqa: E402

from . import test_oracle_pins as pins  # noqa: E402


def _noalloc(lib, X, depth):
    n = X.shape[2]
    f = torch.empty(n, dtype=torch.uint8, device="cuda")
    lo = torch.empty(n, dtype=torch.float64, device="cuda")
    hi = torch.empty(n, dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.hexval_check_soa_noalloc(n, p(X), p(f), p(lo), p(hi), depth, p(st), stream)
    assert rc == 0, rc
    torch.cuda.synchronize()
    return f.cpu().numpy(), lo.cpu().numpy(), hi.cpu().numpy(), int(st.item())


def _inputs():
    """A refinement-heavy batch with exact zeros, then perturbed cubes."""
    A = synth.twisted_layers(2_500, seed=9090, theta_max_deg=180.0)
    Z = pins._zero_corner_elements(60, 23)
    first = np.ascontiguousarray(np.concatenate([A, Z], axis=2))
    second = synth.perturbed_cubes(16_384, noise=0.45, seed=9191)
    return [torch.from_numpy(first).cuda(), torch.from_numpy(second).cuda()]


def test_noalloc_matches_regular_entry_point_twice_in_a_row():
    """Three calls in a row (the first input twice): all 8 flag bits equal to
    the regular entry point's (the same kernels, the same exact box check),
    bounds within 1e-12; verdict and depth equal to the oracle's too (its
    bit 7 marks a different event, the oracle's own exact tier)."""
    lib = hv.load()
    ref = hv.Validator(precision="fp64", max_depth=10, queue_capacity=1 << 20,
                       max_batch=1 << 20, max_nodes=1 << 10, exact_capacity=1 << 14)
    inputs = _inputs()
    wants = [oracle.check_soa(X.cpu().numpy(), max_depth=10) for X in inputs]
    for X, (of, olo, ohi) in zip(inputs + inputs[:1], wants + wants[:1]):
        want = [t.cpu().numpy() for t in ref.check_soa(X)]
        assert ref.status() == 0
        assert ref.stats(reset=True)["max_level_boxes"] <= hv.NOALLOC_MAX_HEX  # no overflow
        f, lo, hi, st = _noalloc(lib, X, 10)
        assert st == 0
        assert np.array_equal(f, want[0])
        assert np.array_equal(f & 0x7F, of & 0x7F)
        scale = np.maximum(np.abs(want[1]), np.abs(want[2]))
        assert np.all(np.abs(lo - want[1]) <= 1e-12 * scale)
        assert np.all(np.abs(hi - want[2]) <= 1e-12 * scale)
        oscale = np.maximum(np.abs(olo), np.abs(ohi))
        assert np.all(np.abs(lo - olo) <= 1e-12 * oscale)
        assert np.all(np.abs(hi - ohi) <= 1e-12 * oscale)
        assert (f & 7 == 1).any() and (f & 7 == 2).any() and ((f >> 3) & 15).max() >= 1
    ref.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    lib = hv.load()
    X = torch.zeros((8, 3, hv.NOALLOC_MAX_HEX + 1), dtype=torch.float64, device="cuda")
    out = torch.empty(X.shape[2], dtype=torch.uint8, device="cuda")
    rc = lib.hexval_check_soa_noalloc(X.shape[2], ctypes.c_void_p(X.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), None, None, 8, None, None)
    assert rc == -1  # HEXVAL_E_ARG, nothing enqueued
