"""Parity of the quadrangle kernels (through the C ABI) with the quadrangle
oracle: flags bit-identical (bit 7, "decided exactly", masked), jmin/jmax
within 1e-12 (FP64 form) or 2e-3 (FP32-decided elements) relative to the
largest |corner value|."""
import numpy as np
import pytest

from oracle import quad
from paper_1706_01613_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on CPU hosts, skipped there
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1706_01613_gb300 import hexval as hv  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 2e-3}


@pytest.fixture(scope="module")
def validators():
    vs = {p: hv.Validator(precision=p, max_depth=8, queue_capacity=1 << 16, max_batch=1 << 20,
                          max_nodes=1 << 20, exact_capacity=1 << 10) for p in ("fp64", "fp32")}
    yield vs
    for v in vs.values():
        v.close()


def _fp32_bound(X):
    """Certified FP32 error bound of the corner values (see quad.cu): inputs
    rounded within 2^-24 X, differences within eps = 2^-23 X + 2^-24 L."""
    X = np.asarray(X, float)
    Xm = np.abs(X).reshape(8, -1).max(axis=0)
    d = [X[1] - X[0], X[2] - X[3], X[3] - X[0], X[2] - X[1]]
    L = np.max([np.abs(v).max(axis=0) for v in d], axis=0) * (1 + 2.0 ** -20) + 2.0 ** -23 * Xm
    eps = 2.0 ** -23 * Xm + 2.0 ** -24 * L
    return (4 * eps * (L + eps) + 2 * eps * eps + 4 * 2.0 ** -24 * (L + eps) ** 2) * 1.01


def _compare(prec, got, want, X=None):
    """Flags bit-identical; jmin/jmax within 1e-12 relative (FP64) or within
    the certified FP32 bound of each element (FP32 form, X given)."""
    f, lo, hi = got
    wf, wlo, whi = want
    bad = np.nonzero((f & 0x7F) != (wf & 0x7F))[0]
    assert len(bad) == 0, "flags differ at %s: %s vs %s" % (bad[:8], f[bad[:8]], wf[bad[:8]])
    fin = np.isfinite(wlo)
    err = np.maximum(np.abs(lo[fin] - wlo[fin]), np.abs(hi[fin] - whi[fin]))
    if prec == "fp64" or X is None:
        scale = np.maximum(np.abs(wlo), np.abs(whi))[fin]
        scale = np.where(scale > 0, scale, 1.0)
        assert np.all(err / scale <= TOL[prec]), (err / scale).max()
    else:
        bound = _fp32_bound(X)[fin]
        assert np.all(err <= bound), (err / bound).max()
    assert np.array_equal(np.isnan(lo), np.isnan(wlo))


def _soa(v, X):
    out = v.check_quads(torch.from_numpy(np.ascontiguousarray(X)).cuda())
    return [t.cpu().numpy() for t in out], v.status()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("noise", [0.3, 0.45])
def test_perturbed_squares(validators, prec, noise):
    X = synth.perturbed_squares(200_003, noise=noise, seed=11)
    got, rc = _soa(validators[prec], X)
    assert rc == 0
    want = quad.check(X)
    _compare(prec, got, want, X)
    frac = np.mean((want[0] & 7) == quad.INVALID)
    assert 0.0 < frac < 0.5


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [1, 31, 33, 257, 1000])
def test_ragged_sizes(validators, prec, n):
    X = synth.perturbed_squares(n, noise=0.45, seed=n)
    got, _ = _soa(validators[prec], X)
    _compare(prec, got, quad.check(X), X)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_special_shapes_and_exact_decisions(validators, prec):
    d = 2.0 ** -100
    shapes = [
        [[0, 0], [1, 0], [1, 1], [0, 1]],
        [[0, 0], [1, 0], [0, 1], [1, 1]],          # bow-tie
        [[0, 0], [2, 0], [0.5, 0.5], [0, 2]],      # dart
        [[0, 0], [0, 1], [1, 1], [1, 0]],          # clockwise
        [[0, 0], [1, 0], [2, 0], [0, 1]],          # three collinear nodes: J = 0
        # a straight angle at node 1 tilted by d: J1 = x12 y14 - y12 x14 = d exactly,
        # far inside every floating-point bound; the other corners are ~1
        [[0, 0], [1, 0], [0, 1], [-1, d]],
        [[0, 0], [1, 0], [0, 1], [-1, -d]],
        [[0, 0], [1, 0], [0, 1], [-1, 0]],
    ]
    X = np.transpose(np.array(shapes, float), (1, 2, 0)).copy()
    got, rc = _soa(validators[prec], X)
    assert rc == 0
    want = quad.check(X)
    _compare(prec, got, want, X)
    assert list(got[0] & 7) == [1, 2, 2, 2, 2, 1, 2, 2]
    assert all(got[0][5:] & 0x80)  # decided by the exact test


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonfinite_and_empty(validators, prec):
    X = synth.perturbed_squares(64, seed=3)
    X[1, 0, 5] = np.nan
    X[3, 1, 9] = -np.inf
    got, _ = _soa(validators[prec], X)
    _compare(prec, got, quad.check(X), X)
    assert got[0][5] & 7 == 4 and got[0][9] & 7 == 4
    empty = torch.empty((4, 2, 0), dtype=torch.float64, device="cuda")
    f, _, _ = validators[prec].check_quads(empty)
    assert f.numel() == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_indexed_grid(validators, prec):
    nodes, conn = synth.structured_grid_2d(700, 600, sigma=0.3, seed=12)
    v = validators[prec]
    out = v.check_quads_indexed(torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda())
    assert v.status() == 0
    _compare(prec, [t.cpu().numpy() for t in out], quad.check_indexed(nodes, conn),
             np.transpose(nodes[conn], (1, 2, 0)))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_indexed_bad_entries(validators, prec):
    nodes, conn = synth.structured_grid_2d(20, 10, seed=13)
    conn = conn.copy()
    conn[3, 1] = -1
    conn[17, 2] = nodes.shape[0]
    v = validators[prec]
    f, lo, _ = [t.cpu().numpy() for t in
                v.check_quads_indexed(torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda())]
    assert v.status() == -4
    assert f[3] & 7 == 3 and f[17] & 7 == 3 and np.isnan(lo[3])
    ok = np.ones(len(conn), bool)
    ok[[3, 17]] = False
    fixed = conn.copy()
    fixed[[3, 17]] = conn[[4, 18]]
    assert np.array_equal(f[ok] & 0x7F, quad.check_indexed(nodes, fixed)[0][ok] & 0x7F)


def test_indexed_misaligned_is_rejected(validators):
    nodes, conn = synth.structured_grid_2d(8, seed=14)
    N = torch.from_numpy(nodes).cuda()
    buf = torch.empty(N.numel() + 1, dtype=torch.float64, device="cuda")
    shifted = buf[1:].view(-1, 2)
    shifted.copy_(N)
    with pytest.raises(RuntimeError):
        validators["fp64"].check_quads_indexed(shifted, torch.from_numpy(conn).cuda())


def test_span_beyond_exact_range_is_undecided(validators):
    """Coordinates spanning 131 bits with a corner value inside the FP64 bound:
    the exact test is out of range, so the element is UNDECIDED with status
    HEXVAL_E_RANGE (the oracle, with unbounded rationals, says VALID)."""
    P = [[0.0, 0.0], [2.0 ** 100, 0.0], [2.0 ** 100, 2.0 ** -30], [0.0, 2.0 ** -30]]
    X = np.transpose(np.array([P], float), (1, 2, 0)).copy()
    got, rc = _soa(validators["fp64"], X)
    assert got[0][0] & 7 == 3 and rc == -7
    assert quad.check(X)[0][0] & 7 == quad.VALID


def test_full_grid_4096_sampled():
    """The benchmark's 2D workload (4096^2 quads), every flag against the oracle."""
    nodes, conn = synth.structured_grid_2d(4096)
    want = quad.check_indexed(nodes, conn)
    for prec in ("fp32", "fp64"):
        v = hv.Validator(precision=prec, max_depth=8, queue_capacity=1 << 16)
        out = v.check_quads_indexed(torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda())
        assert v.status() == 0
        _compare(prec, [t.cpu().numpy() for t in out], want, np.transpose(nodes[conn], (1, 2, 0)))
        v.close()
