"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Flags (verdict and decision depth) must be bit-identical; bit 7 (exact tier
used) is diagnostic and masked.  bmin/bmax: the FP64 form within 1e-12 of the
oracle relative to max |coefficient|; the FP32-filtered form, element by
element, within the certified FP32 bound of Sec. 4's coefficients
(fp32_bound below: 256 eps L^2 + 1024 u L^3 with u = 2^-24, eps = 2^-23 X +
2^-24 L, L the largest edge-vector component and X the largest |coordinate|
of the element), which also bounds the elements redone at higher precision.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_1706_01613_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on CPU hosts, skipped there
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1706_01613_gb300 import hexval as hv  # noqa: E402

from . import test_oracle_pins as pins  # noqa: E402

TOL64 = 1e-12
CAPS = dict(queue_capacity=1 << 21, max_batch=1 << 22, max_nodes=1 << 22, exact_capacity=1 << 14)

# edge vectors of the trilinear map (Sec. 5), as pairs of Appendix A nodes
EDGES = [(0, 1), (3, 2), (4, 5), (7, 6), (0, 3), (1, 2), (4, 7), (5, 6),
         (0, 4), (1, 5), (3, 7), (2, 6)]


def fp32_bound(X):
    """Certified bound of the FP32 form's coefficients, per element of the
    corner planes X (8, 3, n): every depth-0 coefficient computed in FP32 is
    within E of its exact value.  L is taken from the exact edges and
    widened by the edges' own FP32 error, as the kernels form it from the
    rounded ones."""
    X = np.asarray(X, np.float64)
    xm = np.abs(X).max(axis=(0, 1))
    L = np.max([np.abs(X[b] - X[a]).max(axis=0) for a, b in EDGES], axis=0)
    L = L * (1 + 2.0 ** -22) + 2.0 ** -22 * xm
    eps = 2.0 ** -23 * xm + 2.0 ** -24 * L
    return (256.0 * eps * L * L + 1024.0 * 2.0 ** -24 * L ** 3) * 1.0001


def _soa(nodes, conn):
    return synth.soa_from_indexed(nodes, conn)


@pytest.fixture(scope="module")
def validators():
    vs = {}
    for prec in ("fp64", "fp32"):
        for d in (8, 12):
            vs[(prec, d)] = hv.Validator(precision=prec, max_depth=d, **CAPS)
    yield vs
    for v in vs.values():
        v.close()


def _run_soa(v, X):
    f, lo, hi = v.check_soa(torch.from_numpy(np.ascontiguousarray(X)).cuda())
    rc = v.status()
    return f.cpu().numpy(), lo.cpu().numpy(), hi.cpu().numpy(), rc


def _compare(prec, got, want, X=None):
    """Flags bit-exact (bit 7 masked); coefficients within 1e-12 (FP64 form)
    or within each element's certified FP32 bound (FP32 form; X = the
    elements' corner planes).  Returns the largest and the 99th percentile
    of the error relative to the element's largest |min/max coefficient|."""
    f, lo, hi = got
    wf, wlo, whi = want
    bad = np.nonzero((f & 0x7F) != (wf & 0x7F))[0]
    assert len(bad) == 0, "flags differ at %s: got %s want %s" % (
        bad[:10], f[bad[:10]] & 0x7F, wf[bad[:10]] & 0x7F)
    assert np.array_equal(np.isnan(lo), np.isnan(wlo))
    fin = np.isfinite(wlo)
    scale = np.maximum(np.abs(wlo), np.abs(whi))[fin]
    err = np.maximum(np.abs(lo[fin] - wlo[fin]), np.abs(hi[fin] - whi[fin]))
    if prec == "fp64":
        assert np.all(err <= TOL64 * scale), "coefficient error %g" % (err / scale).max()
    else:
        assert X is not None and X.shape[2] == len(f)
        E = fp32_bound(X)[fin] + TOL64 * scale  # + the oracle's own rounding
        over = np.nonzero(err > E)[0]
        assert len(over) == 0, "beyond the FP32 bound at %s: error %s bound %s" % (
            np.nonzero(fin)[0][over[:5]], err[over[:5]], E[over[:5]])
    rel = err / np.where(scale > 0, scale, 1.0)
    if not len(rel):
        return 0.0, 0.0
    return float(rel.max()), float(np.percentile(rel, 99))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_paper_worked_examples(validators, prec):
    X = np.stack([np.array(e["nodes"], float) for e in pins._examples()], axis=2)
    got = _run_soa(validators[(prec, 8)], X)
    assert got[3] == 0
    _compare(prec, got[:3], oracle.check_soa(X, max_depth=8), X)
    assert [int(x) & 0x7F for x in got[0]] == [2 | 3 << 3, 1 | 1 << 3, 2]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_perturbed_cubes_10000(validators, prec):
    """10,000 unit cubes with U[-0.3, 0.3] corner noise (seed 20170001)."""
    X = synth.perturbed_cubes(10_000)
    got = _run_soa(validators[(prec, 8)], X)
    rel = _compare(prec, got[:3], oracle.check_soa(X, max_depth=8), X)
    print("%s max / p99 rel coefficient error %.3g / %.3g" % (prec, *rel))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [1, 31, 32, 33, 255, 257, 1000, 4097])
def test_ragged_sizes(validators, prec, n):
    X = synth.perturbed_cubes(n, noise=0.5, seed=1000 + n)
    got = _run_soa(validators[(prec, 8)], X)
    _compare(prec, got[:3], oracle.check_soa(X, max_depth=8), X)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_refinement_heavy(validators, prec):
    """Prisms twisted by up to 180 degrees with aspect ratios up to 1000:
    decisions up to depth 11 (depth cap 12)."""
    X = synth.twisted_layers(20_000, seed=4444, theta_max_deg=180.0)
    v = validators[(prec, 12)]
    v.stats(reset=True)
    got = _run_soa(v, X)
    want = oracle.check_soa(X, max_depth=12)
    _compare(prec, got[:3], want, X)
    assert (want[0] >> 3 & 15).max() >= 6
    st = v.stats()
    assert st["refined"] > 1000 and st["boxes"] > 0


def test_fp32_refinement_keeps_most_elements_off_fp64():
    """Boundary-layer prisms (twist up to 120 degrees, aspect ratio up to
    1000): most need one refinement level, which the FP32 form does in FP32;
    flags equal the oracle's and only a minority is redone in FP64."""
    X = synth.twisted_layers(50_000, seed=4646)
    v = hv.Validator(precision="fp32", max_depth=10, **CAPS)
    v.stats(reset=True)
    got = _run_soa(v, X)
    st = v.stats()
    _compare("fp32", got[:3], oracle.check_soa(X, max_depth=10), X)
    assert st["refined"] > 5000
    assert st["escalated_fp64"] < 0.5 * st["refined"], st
    v.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_depth_caps(prec):
    X = synth.twisted_layers(5000, seed=4545, theta_max_deg=180.0)
    for d in (0, 1, 2, 5):
        v = hv.Validator(precision=prec, max_depth=d, **CAPS)
        got = _run_soa(v, X)
        _compare(prec, got[:3], oracle.check_soa(X, max_depth=d), X)
        v.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_degenerate_go_exact(validators, prec):
    """Exact zeros: collapsed edge, flat element, 180-degree twist, and 200
    elements whose corner-1 J is exactly 0 but rounds to noise of either sign."""
    ref = synth.REF_CORNERS
    X1 = ref.copy()
    X1[1] = X1[0]
    X2 = ref.copy()
    X2[:, 2] = 0.0
    X = np.concatenate([np.stack([X1, X2, pins.TWIST180], axis=2),
                        pins._zero_corner_elements(200, 19)], axis=2)
    got = _run_soa(validators[(prec, 8)], X)
    want = oracle.check_soa(X, max_depth=8)
    _compare(prec, got[:3], want, X)
    assert np.all(got[0] & 0x7F == 2)
    assert np.all(got[0] & 0x80)  # decided by the exact tier


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonfinite_and_empty(validators, prec):
    v = validators[(prec, 8)]
    X = np.stack([synth.REF_CORNERS.copy() for _ in range(3)], axis=2)
    X[2, 1, 0] = np.nan
    X[5, 0, 1] = np.inf
    f, lo, hi, rc = _run_soa(v, X)
    assert rc == 0 and list(f & 7) == [4, 4, 1] and np.isnan(lo[0]) and lo[2] == 1.0
    f, _, _ = v.check_soa(torch.zeros((8, 3, 0), dtype=torch.float64, device="cuda"))
    assert f.numel() == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_indexed_small_grid(validators, prec):
    nodes, conn = synth.structured_grid(24, 20, 16, sigma=0.3, seed=31)
    v = validators[(prec, 8)]
    f, lo, hi = v.check_indexed(torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda())
    assert v.status() == 0
    want = oracle.check_indexed(nodes, conn, max_depth=8)
    _compare(prec, (f.cpu().numpy(), lo.cpu().numpy(), hi.cpu().numpy()), want,
             _soa(nodes, conn))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bad_connectivity_sets_status(validators, prec):
    nodes, conn = synth.structured_grid(6, 5, 4, sigma=0.2, seed=5)
    conn = conn.copy()
    conn[7, 3] = nodes.shape[0]
    conn[9, 0] = -1
    v = validators[(prec, 8)]
    f, lo, _ = v.check_indexed(torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda())
    assert v.status() == -4  # HEXVAL_E_INDEX
    f = f.cpu().numpy()
    assert f[7] & 7 == 3 and f[9] & 7 == 3 and np.isnan(lo.cpu().numpy()[7])
    ok = np.ones(len(conn), bool)
    ok[[7, 9]] = False
    good_conn = conn.copy()
    good_conn[7] = conn[8]
    good_conn[9] = conn[8]
    want = oracle.check_indexed(nodes, good_conn, max_depth=8)[0]
    assert np.array_equal(f[ok] & 0x7F, want[ok] & 0x7F)
    assert v.status() == 0  # the status is cleared once read


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tiny_queue_overflows_into_exact_tier(prec):
    """With a refinement queue of 16 boxes the overflowing elements are
    decided by the exact tier: the flags stay exact and the status says so."""
    X = synth.twisted_layers(3000, seed=4646, theta_max_deg=180.0)
    v = hv.Validator(precision=prec, max_depth=10, queue_capacity=16, max_batch=1 << 16,
                     max_nodes=1 << 10, exact_capacity=1 << 14)
    got = _run_soa(v, X)
    assert got[3] == -5
    _compare(prec, got[:3], oracle.check_soa(X, max_depth=10), X)
    v.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batching_is_invisible(prec):
    X = synth.perturbed_cubes(10_000, noise=0.5, seed=99)
    a = hv.Validator(precision=prec, max_depth=8, **CAPS)
    b = hv.Validator(precision=prec, max_depth=8, queue_capacity=1 << 16, max_batch=777,
                     max_nodes=1 << 10, exact_capacity=1 << 10)
    ga, gb = _run_soa(a, X), _run_soa(b, X)
    for x, y in zip(ga[:3], gb[:3]):
        assert np.array_equal(x, y, equal_nan=True)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_affine_mixture_escalation(validators, prec):
    """Precision-stress mixture: 5% near-degenerate elements (|min J/max J|
    <= 1e-6) must be escalated by the FP32 form and still get exact flags."""
    X, kind, r = synth.affine_mixture(200_000, seed=20170003)
    v = validators[(prec, 8)]
    v.stats(reset=True)
    got = _run_soa(v, X)
    rel = _compare(prec, got[:3], oracle.check_soa(X, max_depth=8), X)
    st = v.stats()
    print("%s: %s max / p99 rel coefficient error %.3g / %.3g" % (prec, st, *rel))
    if prec == "fp32":
        assert st["escalated_fp64"] >= (kind == 1).sum()


@pytest.mark.parametrize("kind", ["soa", "indexed"])
def test_double_float_redo_of_many_escalations(kind):
    """About 26,000 near-degenerate elements in one batch of 2^19, with
    HEXVAL_OPT_DFREDO: the escalations beyond the FP32 pass's own FP64 redo
    are redone one per thread in double-float (about 44 bits, so nearly all
    of |min J / max J| <= 1e-6 are decided there), FP64 for the rest.  Flags
    identical to the run without the option and exact against the oracle on
    every near-degenerate element and a sample of the others; their
    coefficient bounds within 1e-6 of the oracle's.  The indexed form gives
    every element its own 8 nodes."""
    X, deg_kind, _ = synth.affine_mixture(1 << 19, seed=20170005)
    n = X.shape[2]
    runs = []
    for opt in (hv.OPT_DFREDO, 0):
        v = hv.Validator(precision="fp32", max_depth=8, options=opt)
        v.stats(reset=True)
        if kind == "soa":
            got = _run_soa(v, X)
        else:
            nodes = np.ascontiguousarray(X.transpose(2, 0, 1).reshape(8 * n, 3))
            conn = np.arange(8 * n, dtype=np.int32).reshape(n, 8)
            got = [t.cpu().numpy() for t in v.check_indexed(torch.from_numpy(nodes).cuda(),
                                                            torch.from_numpy(conn).cuda())]
            got.append(v.status())
        runs.append((got, v.stats()))
        v.close()
    (f, lo, hi, rc), st = runs[0]
    assert rc == 0 and runs[1][0][3] == 0
    assert np.array_equal(f, runs[1][0][0])
    deg = np.nonzero(deg_kind == 1)[0]
    rest = np.random.default_rng(5).choice(np.nonzero(deg_kind != 1)[0], 20_000, replace=False)
    for idx in (deg, rest):
        Xi = np.ascontiguousarray(X[:, :, idx])
        want = oracle.check_soa(Xi, max_depth=8)
        rel = _compare("fp32", (f[idx], lo[idx], hi[idx]), want, Xi)
        if idx is deg:  # double-float or FP64: far tighter than the FP32 bound
            assert rel[0] <= 1e-6
    print(kind, st, runs[1][1])
    assert st["escalated_fp64"] >= len(deg)
    assert st["escalated_df"] >= 0.5 * (len(deg) - 4096)
    assert runs[1][1]["escalated_df"] == 0


@pytest.mark.parametrize("kind", ["soa", "indexed"])
def test_partial_fp64_redo_of_escalations(kind):
    """HEXVAL_OPT_PARTIAL64, no escalation redone inside the FP32 pass
    (esc_in_pass 0): the partial redo evaluates in FP64 only the samples
    and edge coefficients FP32 left unsettled, the tail redoes the rest.  About 25,000 near-degenerate
    elements in 500,000 (one corner moved: few signs open) and twisted
    boundary-layer prisms (refinement in the same batch), depth caps 0, 1
    and 8: flags identical to the run without the option, exact against the
    oracle on every near-degenerate element, every prism and a sample of the
    others, and the statistics count the elements the partial redo decided."""
    X, deg_kind, _ = synth.affine_mixture(500_000, seed=20170021)
    T = synth.twisted_layers(20_000, seed=20170022, theta_max_deg=150.0)
    X = np.ascontiguousarray(np.concatenate([X, T], axis=2))
    deg_kind = np.concatenate([deg_kind, np.full(T.shape[2], 3, np.int8)])
    n = X.shape[2]
    nodes = np.ascontiguousarray(X.transpose(2, 0, 1).reshape(8 * n, 3))
    conn = np.arange(8 * n, dtype=np.int32).reshape(n, 8)
    for depth in (8, 1, 0):
        runs = []
        for opt in (hv.OPT_PARTIAL64, 0):
            v = hv.Validator(precision="fp32", max_depth=depth, options=opt, esc_in_pass=0,
                             **CAPS)
            v.stats(reset=True)
            if kind == "soa":
                got = _run_soa(v, X)
            else:
                got = [t.cpu().numpy() for t in v.check_indexed(torch.from_numpy(nodes).cuda(),
                                                                torch.from_numpy(conn).cuda())]
                got.append(v.status())
            runs.append((got, v.stats()))
            v.close()
        (f, lo, hi, rc), st = runs[0]
        assert rc == 0 and runs[1][0][3] == 0
        assert np.array_equal(f, runs[1][0][0])
        print(kind, depth, st)
        # the partial redo's leftovers are the tail's to redo in full
        assert 0 < st["partial_fp64"]
        assert st["partial_fp64"] + st["redone_tail"] <= st["escalated_fp64"]
        assert runs[1][1]["partial_fp64"] == 0
        if depth != 8:
            continue
        deg = np.nonzero(deg_kind == 1)[0]
        rest = np.random.default_rng(6).choice(np.nonzero((deg_kind != 1) & (deg_kind != 3))[0],
                                               20_000, replace=False)
        for idx in (deg, rest, np.nonzero(deg_kind == 3)[0]):
            Xi = np.ascontiguousarray(X[:, :, idx])
            _compare("fp32", (f[idx], lo[idx], hi[idx]), oracle.check_soa(Xi, max_depth=8), Xi)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_repeated_calls_replay_a_graph(prec):
    """Identical calls are replayed from a graph the library captures on the
    second one: results equal the direct launches', in-place changes of the
    inputs between calls are seen, and other pointers fall back to direct
    launches (and then a new graph)."""
    nodes, conn = synth.structured_grid(40, 30, 20, sigma=0.3, seed=91)
    N, C = torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda()
    n = len(conn)
    direct = hv.Validator(precision=prec, max_depth=8, options=hv.OPT_NO_REPLAY, **CAPS)
    v = hv.Validator(precision=prec, max_depth=8, **CAPS)
    out = tuple(torch.empty(n, dtype=d, device="cuda") for d in (torch.uint8, torch.float64, torch.float64))
    ref = [t.cpu().numpy() for t in direct.check_indexed(N, C)]
    for _ in range(4):  # direct, capture + replay, replay, replay
        got = [t.cpu().numpy() for t in v.check_indexed(N, C, out=out)]
        for a, b in zip(got, ref):
            assert np.array_equal(a, b, equal_nan=True)
    N[conn[7, 6]] += torch.tensor([0.0, 0.0, -3.0], dtype=torch.float64, device="cuda")  # inverts element 7
    ref2 = [t.cpu().numpy() for t in direct.check_indexed(N, C)]
    got = [t.cpu().numpy() for t in v.check_indexed(N, C, out=out)]
    assert got[0][7] & 7 == 2
    for a, b in zip(got, ref2):
        assert np.array_equal(a, b, equal_nan=True)
    X = synth.perturbed_cubes(3001, noise=0.5, seed=92)
    want = oracle.check_soa(X, max_depth=8)
    Xd = torch.from_numpy(X).cuda()
    for _ in range(3):
        _compare(prec, [t.cpu().numpy() for t in v.check_soa(Xd)], want, X)
    assert v.status() == 0 and direct.status() == 0
    v.close()
    direct.close()


def test_exact_box_checks_settle_deep_uncertain_boxes():
    """65,536 prisms twisted by up to 180 degrees (depth cap 10), where some
    boxes deep in the refinement have coefficients within the FP64 error
    bound of zero.  Each such box is checked exactly on its own (the root
    coefficients as integers, subdivided to the box by the exact Bernstein
    formulas) instead of sending its element through the full exact tier.
    Flags equal the oracle's on every element that used an exact box check
    and on a sample of the others, in both forms, and a call takes seconds."""
    import time
    X = synth.twisted_layers(65536, seed=20170004, theta_max_deg=180.0)
    got = {}
    for prec in ("fp64", "fp32"):
        v = hv.Validator(precision=prec, max_depth=10)
        Xd = torch.from_numpy(X).cuda()
        v.check_soa(Xd)
        torch.cuda.synchronize()
        t0 = time.time()
        f = v.check_soa(Xd)[0].cpu().numpy()
        dt = time.time() - t0
        assert v.status() == 0
        v.close()
        assert dt < 5.0, dt
        got[prec] = f
    used = np.union1d(np.nonzero(got["fp64"] & 0x80)[0], np.nonzero(got["fp32"] & 0x80)[0])
    print("elements with an exact box check:", len(used))
    assert len(used) > 0
    rest = np.random.default_rng(6).choice(X.shape[2], 3000, replace=False)
    idx = np.union1d(used, rest)
    wf, _, _ = oracle.check_soa(np.ascontiguousarray(X[:, :, idx]), max_depth=10)
    for prec in ("fp64", "fp32"):
        bad = np.nonzero((got[prec][idx] & 0x7F) != (wf & 0x7F))[0]
        assert len(bad) == 0, (prec, idx[bad[:10]], got[prec][idx[bad[:10]]], wf[bad[:10]])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_barrier_wait_budget_runs_out_cleanly(prec):
    """Failure detection without a fault: with a grid-barrier budget of one
    poll the tail kernel's barriers give up, the status reads
    HEXVAL_E_TIMEOUT, and the blocks stop their work and end the kernel; the
    counters are still folded and reset, so the context and the handle stay
    usable, and a handle with the default budget then gives the oracle's
    flags on the same input."""
    X = synth.twisted_layers(20_000, seed=4444, theta_max_deg=180.0)  # deep refinement
    v = hv.Validator(precision=prec, max_depth=8, spin_limit=1, **CAPS)
    rcs = [_run_soa(v, X)[3] for _ in range(5)]
    v.close()
    assert set(rcs) <= {0, -6} and -6 in rcs, rcs
    w = hv.Validator(precision=prec, max_depth=8, **CAPS)
    got = _run_soa(w, X)
    assert got[3] == 0
    _compare(prec, got[:3], oracle.check_soa(X, max_depth=8), X)
    w.close()


def test_cuda_graph_capture_replays():
    X = torch.from_numpy(synth.perturbed_cubes(5000, noise=0.5, seed=3)).cuda()
    v = hv.Validator(precision="fp32", max_depth=8, **CAPS)
    out = (torch.empty(5000, dtype=torch.uint8, device="cuda"),
           torch.empty(5000, dtype=torch.float64, device="cuda"),
           torch.empty(5000, dtype=torch.float64, device="cuda"))
    ref = [t.clone() for t in v.check_soa(X)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        v.check_soa(X, out=out, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        v.check_soa(X, out=out)
    for t in out:
        t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
    v.close()


# ----------------------------------------- full-size inputs, every element ----
# The oracle runs once per input on all host cores and is shared by both forms.

@functools.lru_cache(maxsize=1)
def _full_mesh_128():
    nodes, conn = synth.structured_grid(128)
    return nodes, conn, oracle.check_indexed(nodes, conn, max_depth=8,
                                             threads=oracle.max_threads())


@functools.lru_cache(maxsize=1)
def _full_twisted():
    X = synth.twisted_layers(4_194_304)
    return X, oracle.check_soa(X, max_depth=10, threads=oracle.max_threads())


@functools.lru_cache(maxsize=1)
def _full_affine():
    X, kind, _ = synth.affine_mixture(16_777_216)
    return X, kind, oracle.check_soa(X, max_depth=8, threads=oracle.max_threads())


def _fp32_error_line(name, prec, rel):
    print("coefficient error %s %s: max %.3g p99 %.3g" % (name, prec, rel[0], rel[1]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_structured_mesh_128_cubed(prec):
    """The 128^3 indexed mesh (2,097,152 elements) with the library's default
    launch configuration; every element against the oracle."""
    nodes, conn, want = _full_mesh_128()
    v = hv.Validator(precision=prec, max_depth=8)
    f, lo, hi = v.check_indexed(torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda())
    assert v.status() == 0
    got = (f.cpu().numpy(), lo.cpu().numpy(), hi.cpu().numpy())
    _fp32_error_line("mesh128", prec, _compare(prec, got, want, _soa(nodes, conn)))
    v.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_twisted_layers(prec):
    """4,194,304 boundary-layer elements (depth cap 10); every element."""
    X, want = _full_twisted()
    v = hv.Validator(precision=prec, max_depth=10)
    f, lo, hi = v.check_soa(torch.from_numpy(X).cuda())
    assert v.status() == 0
    got = (f.cpu().numpy(), lo.cpu().numpy(), hi.cpu().numpy())
    _fp32_error_line("twisted", prec, _compare(prec, got, want, X))
    v.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_affine_mixture(prec):
    """16,777,216 precision-stress elements (5% near-degenerate, 5%
    inverted); every element."""
    X, kind, want = _full_affine()
    v = hv.Validator(precision=prec, max_depth=8)
    f, lo, hi = v.check_soa(torch.from_numpy(X).cuda())
    assert v.status() == 0
    got = (f.cpu().numpy(), lo.cpu().numpy(), hi.cpu().numpy())
    _fp32_error_line("affine", prec, _compare(prec, got, want, X))
    v.close()


@pytest.mark.parametrize("kind", ["soa", "indexed"])
def test_fp32_variants_agree(kind):
    """The FP32 pass with one element per thread (scalar), two per thread
    (packed f32x2) and on a persistent staging grid give identical flags and
    coefficients that match the oracle; odd sizes exercise the idle second
    lane and a ragged last tile."""
    vs = [hv.Validator(precision="fp32", max_depth=8, options=o, **CAPS)
          for o in (0, hv.OPT_PAIR32, hv.OPT_PREFETCH)]
    if kind == "soa":
        X = synth.perturbed_cubes(20_001, noise=0.45, seed=77)
        got = [_run_soa(v, X)[:3] for v in vs]
        want = oracle.check_soa(X, max_depth=8)
    else:
        nodes, conn = synth.structured_grid(31, 17, 13, sigma=0.3, seed=78)
        N, C = torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda()
        got = [[t.cpu().numpy() for t in v.check_indexed(N, C)] for v in vs]
        want = oracle.check_indexed(nodes, conn, max_depth=8)
        X = _soa(nodes, conn)
    for other in got[1:]:
        for x, y in zip(got[0], other):
            assert np.array_equal(x, y, equal_nan=True)
    _compare("fp32", got[0], want, X)
    for v in vs:
        v.close()


@pytest.mark.parametrize("opt,threads", [("PREFETCH", 64), ("PREFETCH", 128), ("PREFETCH", 256)])
def test_persistent_indexed_pass_many_tiles(opt, threads):
    """The indexed FP32 pass on a persistent grid staged through shared
    memory (several tiles per block, a ragged last tile): flags equal to the
    oracle's, bad connectivity rows flagged, escalations beyond the in-pass
    share (more than 4096) left to the tail kernel."""
    nodes, conn = synth.structured_grid(100, 97, 61, sigma=0.3, seed=81)
    conn = conn.copy()
    bad_rows = [5, 123_457, len(conn) - 1]
    good = conn[[6, 123_458, len(conn) - 2]].copy()
    conn[bad_rows[0], 2] = -7
    conn[bad_rows[1], 5] = nodes.shape[0]
    conn[bad_rows[2], 7] = 1 << 30
    options = 0
    for o in opt.split("|"):
        options |= getattr(hv, "OPT_" + o)
    v = hv.Validator(precision="fp32", max_depth=8, options=options, bulk_threads=threads, **CAPS)
    v.stats(reset=True)
    f, lo, hi = [t.cpu().numpy() for t in v.check_indexed(torch.from_numpy(nodes).cuda(),
                                                          torch.from_numpy(conn).cuda())]
    assert v.status() == -4  # HEXVAL_E_INDEX
    st = v.stats()
    assert st["escalated_fp64"] > 4096
    assert all(f[r] & 7 == 3 and np.isnan(lo[r]) for r in bad_rows)
    fixed = conn.copy()
    fixed[bad_rows] = good
    want = oracle.check_indexed(nodes, fixed, max_depth=8)
    ok = np.ones(len(conn), bool)
    ok[bad_rows] = False
    _compare("fp32", (f[ok], lo[ok], hi[ok]), tuple(w[ok] for w in want),
             np.ascontiguousarray(_soa(nodes, fixed)[:, :, ok]))
    v.close()


def test_autotuner_picks_a_candidate_and_stays_exact(tmp_path):
    from paper_1706_01613_gb300 import tune
    nodes, conn = synth.structured_grid(40, 40, 40, sigma=0.15, seed=80)
    dev = (torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda())
    cache = str(tmp_path / "tune.json")
    best = tune.best_config("fp32", "indexed", len(conn), dev, cache=cache, reps=3, **CAPS)
    launch = {"options": best["options"] & ~(hv.OPT_DFREDO | hv.OPT_LEVEL1 | hv.OPT_PARTIAL64),
              "bulk_threads": best["bulk_threads"]}
    assert launch in tune.candidates("fp32")
    assert tune.best_config("fp32", "indexed", len(conn), dev, cache=cache, **CAPS) == best
    v = hv.Validator(precision="fp32", max_depth=8, **best, **CAPS)
    got = [t.cpu().numpy() for t in v.check_indexed(*dev)]
    _compare("fp32", got, oracle.check_indexed(nodes, conn, max_depth=8), _soa(nodes, conn))
    v.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_indexed_nodes_not_16_byte_aligned(validators, prec):
    """A node array that starts 8 bytes past a 16-byte boundary (odd node
    count too) takes the scalar conversion path and gives the same flags."""
    nodes, conn = synth.structured_grid(12, 9, 7, sigma=0.3, seed=33)
    buf = torch.zeros(nodes.size + 1, dtype=torch.float64, device="cuda")
    buf[1:] = torch.from_numpy(nodes.reshape(-1)).cuda()
    N = buf[1:].view(-1, 3)
    assert N.data_ptr() % 16 == 8
    v = validators[(prec, 8)]
    f, lo, hi = v.check_indexed(N, torch.from_numpy(conn).cuda())
    assert v.status() == 0
    _compare(prec, (f.cpu().numpy(), lo.cpu().numpy(), hi.cpu().numpy()),
             oracle.check_indexed(nodes, conn, max_depth=8), _soa(nodes, conn))


@pytest.mark.parametrize("opt", [0, hv.OPT_PAIR32, hv.OPT_PREFETCH])
def test_nodes_outside_fp32_range_escalate(opt):
    """Nodes with a coordinate FP32 cannot hold get +inf records in the FP32
    form; every element touching one goes to FP64 and the results are the
    oracle's.  Two cases: three nodes of the face y = 0 moved to y = 1e-300,
    below FP32's normal range but a negligible move (elements with some
    records infinite), and the whole mesh scaled by 2^130 (every record
    infinite; J scales by 2^390, exactly)."""
    nodes, conn = synth.structured_grid(9, 8, 7, sigma=0.2, seed=91)
    mixed = nodes.copy()
    tiny = [0, 5, 4 + 10 * 9 * 3]  # node ids i + 10 (j + 9 k) with j = 0
    assert np.all(nodes[tiny, 1] == 0.0)
    mixed[tiny, 1] = 1e-300
    scaled = nodes * 2.0 ** 130
    v = hv.Validator(precision="fp32", max_depth=8, options=opt, **CAPS)
    for X, touching in ((mixed, np.isin(conn, tiny).any(axis=1).sum()), (scaled, len(conn))):
        v.stats(reset=True)
        got = [t.cpu().numpy() for t in v.check_indexed(torch.from_numpy(X).cuda(),
                                                        torch.from_numpy(conn).cuda())]
        assert v.status() == 0
        assert v.stats()["escalated_fp64"] >= touching
        _compare("fp32", got, oracle.check_indexed(X, conn, max_depth=8), _soa(X, conn))
    v.close()


@pytest.mark.parametrize("kind", ["affine", "twisted"])
def test_placement_knobs_do_not_change_results(kind):
    """All escalations and refinements left to the tail kernel (esc_in_pass =
    refine_in_pass = 0), or kept in the bulk pass, with the tail's warp
    threshold at both ends: flags identical to the defaults' and the
    oracle's, bounds within each element's certified bound (an element
    refined in FP32 rather than redone in FP64 reports FP32 bounds)."""
    if kind == "affine":
        X, _, _ = synth.affine_mixture(100_000, seed=20170013)
        depth = 8
    else:
        X = synth.twisted_layers(60_000, seed=20170014, theta_max_deg=180.0)
        depth = 10
    runs = []
    for knobs in ({}, dict(esc_in_pass=0, refine_in_pass=0, tail_warp_items=1),
                  dict(esc_in_pass=1 << 20, refine_in_pass=1 << 20, tail_warp_items=64)):
        for prec in ("fp32", "fp64"):
            if prec == "fp64" and "esc_in_pass" in knobs and knobs["esc_in_pass"]:
                continue
            v = hv.Validator(precision=prec, max_depth=depth, **knobs, **CAPS)
            runs.append((prec, _run_soa(v, X)))
            v.close()
    want = oracle.check_soa(X, max_depth=depth)
    for prec, got in runs:
        assert got[3] == 0
        _compare(prec, got[:3], want, X)
    base = {"fp32": runs[0][1], "fp64": runs[1][1]}
    for prec, got in runs[2:]:
        assert np.array_equal(got[0] & 0x7F, base[prec][0] & 0x7F)


@pytest.mark.parametrize("kind,chunks", [("indexed", 1), ("indexed", 4), ("soa", 3)])
def test_host_buffers_pipeline(kind, chunks):
    """The end-to-end call on pinned host buffers (inputs copied in chunk by
    chunk while earlier chunks are checked, all three outputs copied back)
    gives the device-resident call's flags and the oracle's, with bounds
    within each element's certified bound."""
    v = hv.Validator(precision="fp32", max_depth=8, **CAPS)
    if kind == "indexed":
        nodes, conn = synth.structured_grid(30, 21, 17, sigma=0.3, seed=95)
        host = (torch.from_numpy(nodes).pin_memory(), torch.from_numpy(conn).pin_memory())
        want = [t.cpu().numpy() for t in v.check_indexed(host[0].cuda(), host[1].cuda())]
        oracle_out, X = oracle.check_indexed(nodes, conn, max_depth=8), _soa(nodes, conn)
    else:
        X = synth.perturbed_cubes(10_007, noise=0.45, seed=96)
        host = (torch.from_numpy(X).pin_memory(),)
        want = [t.cpu().numpy() for t in v.check_soa(host[0].cuda())]
        oracle_out = oracle.check_soa(X, max_depth=8)
    got = v.check_host(kind, *host, chunks=chunks)
    torch.cuda.synchronize()
    got = [t.numpy() for t in got]
    assert np.array_equal(got[0] & 0x7F, want[0] & 0x7F)
    _compare("fp32", got, oracle_out, X)
    assert v.status() == 0
    v.close()


@pytest.mark.parametrize("kind", ["indexed", "soa"])
def test_host_pipeline_graph_replay(kind):
    """HostPipeline (the chunked host call recorded into a CUDA graph): each
    run gives the device-resident call's verdicts on the current contents of
    the pinned inputs (changed in place between runs), with bounds within
    each element's certified bound."""
    v = hv.Validator(precision="fp32", max_depth=8, **CAPS)
    if kind == "indexed":
        nodes, conn = synth.structured_grid(30, 21, 17, sigma=0.3, seed=99)
        host = (torch.from_numpy(nodes).pin_memory(), torch.from_numpy(conn).pin_memory())
    else:
        X = synth.perturbed_cubes(10_007, noise=0.45, seed=100)
        host = (torch.from_numpy(X).pin_memory(),)
    pipe = v.host_pipeline(kind, *host, chunks=3)
    for step in range(2):
        if step == 1:  # new contents in the same pinned buffers
            if kind == "indexed":
                host[0][::7] *= 1.01
                host[0][5::11] += 0.2
            else:
                host[0][:, :, ::5] = host[0][:, :, ::5].flip(0)  # reversed node order: inverted
        res = pipe.run()
        torch.cuda.synchronize()  # the host outputs are written by the replay
        got = [t.numpy().copy() for t in res]
        if kind == "indexed":
            a, c = host[0].numpy(), host[1].numpy()
            want = [t.cpu().numpy() for t in v.check_indexed(host[0].cuda(), host[1].cuda())]
            oracle_out, Xs = oracle.check_indexed(a, c, max_depth=8), _soa(a, c)
        else:
            Xs = host[0].numpy()
            want = [t.cpu().numpy() for t in v.check_soa(host[0].cuda())]
            oracle_out = oracle.check_soa(Xs, max_depth=8)
        assert np.array_equal(got[0] & 0x7F, want[0] & 0x7F)
        _compare("fp32", got, oracle_out, Xs)
    assert v.status() == 0
    v.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_prepared_nodes_in_ranges(prec):
    """hexval_prepare_nodes + hexval_check_indexed_prepared over ranges of
    rows give hexval_check_indexed's outputs on the whole mesh, every bit; a
    check_indexed on the handle drops the prepared nodes (E_ARG until the
    next prepare)."""
    nodes, conn = synth.structured_grid(40, 23, 19, sigma=0.35, seed=98)
    N, C = torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda()
    v = hv.Validator(precision=prec, max_depth=8, options=hv.OPT_NO_REPLAY, **CAPS)
    want = [t.cpu().numpy() for t in v.check_indexed(N, C)]
    v.prepare_nodes(N)
    n = len(conn)
    cuts = [0, 1, 777, n // 2, n - 5, n]
    got = [np.empty_like(w) for w in want]
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        part = v.check_indexed_prepared(C[lo:hi])
        for g, t in zip(got, part):
            g[lo:hi] = t.cpu().numpy()
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    assert v.status() == 0
    v.check_indexed(N, C[:10])
    with pytest.raises(hv.HexvalError):
        v.check_indexed_prepared(C[:10])
    v.close()


def test_copy_soa_range_from_host_and_device():
    """One strided copy of an element range of SoA planes, from pinned host
    memory and from device memory, equals the slice."""
    X = torch.from_numpy(synth.perturbed_cubes(5000, seed=97)).pin_memory()
    for src in (X, X.cuda()):
        dst = torch.empty((8, 3, 1234), dtype=torch.float64, device="cuda")
        hv.copy_soa_range(dst, src, 2345)
        torch.cuda.synchronize()
        assert torch.equal(dst.cpu(), X[:, :, 2345:2345 + 1234])
    with pytest.raises(hv.HexvalError):
        hv.copy_soa_range(torch.empty((8, 3, 10), dtype=torch.float64, device="cuda"), X, 4995)


@pytest.mark.parametrize("opt", [hv.OPT_LEVEL1, hv.OPT_LEVEL1 | hv.OPT_PAIR32,
                                 hv.OPT_LEVEL1 | hv.OPT_PREFETCH])
def test_first_level_in_the_fp32_pass(opt):
    """HEXVAL_OPT_LEVEL1: elements decided on level 1 by the first-level
    kernel (boundary-layer prisms, about a quarter need one level), the
    others by the tail as before; flags equal to the default's and the
    oracle's, depth caps 1 and 10; the statistics count them as refined."""
    X = synth.twisted_layers(30_000, seed=20170015, theta_max_deg=150.0)
    for depth in (1, 10):
        base = hv.Validator(precision="fp32", max_depth=depth, **CAPS)
        want = _run_soa(base, X)
        v = hv.Validator(precision="fp32", max_depth=depth, options=opt, **CAPS)
        v.stats(reset=True)
        got = _run_soa(v, X)
        st = v.stats()
        assert got[3] == 0
        assert np.array_equal(got[0] & 0x7F, want[0] & 0x7F)
        _compare("fp32", got[:3], oracle.check_soa(X, max_depth=depth), X)
        assert st["refined"] >= ((want[0] >> 3 & 15) >= 1).sum()
        base.close()
        v.close()
    nodes, conn = synth.structured_grid(20, 18, 16, sigma=0.35, seed=20170016)
    v = hv.Validator(precision="fp32", max_depth=8, options=opt, **CAPS)
    got = [t.cpu().numpy() for t in v.check_indexed(torch.from_numpy(nodes).cuda(),
                                                    torch.from_numpy(conn).cuda())]
    _compare("fp32", got, oracle.check_indexed(nodes, conn, max_depth=8), _soa(nodes, conn))
    v.close()
