"""Corner scaled Jacobian on the GPU (through the C ABI) against the FP64
oracle.  Tolerance per element: the FP32 evaluation on coordinates relative to
node 1 moves each unit edge vector by about 2^-21 x (largest relative
coordinate / that edge's length), so the test allows 2e-6 x (longest /
shortest edge) + 1e-6."""
import math

import numpy as np
import pytest

from oracle import quality
from paper_1706_01613_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on CPU hosts, skipped there
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1706_01613_gb300 import hexval as hv  # noqa: E402

from . import test_oracle_pins as pins  # noqa: E402


@pytest.fixture(scope="module")
def v():
    h = hv.Validator(precision="fp64", queue_capacity=1 << 12, max_batch=1 << 20,
                     max_nodes=1 << 20, exact_capacity=1 << 10)
    yield h
    h.close()


def _tol(X):
    X = np.asarray(X, float)
    lens = []
    for k in range(8):
        for m, _ in quality.NBR[k]:
            lens.append(np.linalg.norm(X[m] - X[k], axis=0))
    lens = np.array(lens)
    ar = lens.max(axis=0) / np.maximum(lens.min(axis=0), 1e-300)
    return 2e-6 * ar + 1e-6


def _check(got, X):
    want = quality.min_scaled_jacobian(X)
    fin = np.isfinite(want)
    assert np.array_equal(np.isnan(got), ~fin)
    err = np.abs(got[fin] - want[fin])
    assert np.all(err <= _tol(X)[fin]), err.max()


@pytest.mark.parametrize("noise", [0.3, 0.6])
def test_perturbed_cubes(v, noise):
    X = synth.perturbed_cubes(100_001, noise=noise, seed=21)
    got = v.corner_quality(torch.from_numpy(X).cuda()).cpu().numpy()
    _check(got, X)


def test_independent_of_position(v):
    X = synth.perturbed_cubes(20_000, noise=0.3, seed=22)
    a = v.corner_quality(torch.from_numpy(X).cuda()).cpu().numpy()
    b = v.corner_quality(torch.from_numpy(X + 1e6).cuda()).cpu().numpy()
    assert np.max(np.abs(a - b)) <= 2e-5
    _check(b, X + 1e6)


def test_paper_example_and_degenerate_corners(v):
    e = pins._examples()[2]
    X = np.stack([np.array(e["nodes"], float), synth.REF_CORNERS.copy(), synth.REF_CORNERS.copy()],
                 axis=2)
    X[1, :, 2] = X[0, :, 2]  # nodes 1 and 2 coincide: value 0
    X[3, 1, 1] = np.nan
    got = v.corner_quality(torch.from_numpy(np.ascontiguousarray(X)).cuda()).cpu().numpy()
    assert math.floor(got[0] * 100) / 100 == e["min_corner_scaled_jacobian_2dp"]
    assert np.isnan(got[1]) and got[2] == 0.0


def test_indexed_mesh(v):
    nodes, conn = synth.structured_grid(64, 48, 40, sigma=0.2, seed=23)
    got = v.corner_quality_indexed(torch.from_numpy(nodes).cuda(),
                                   torch.from_numpy(conn).cuda()).cpu().numpy()
    assert v.status() == 0
    _check(got, np.transpose(nodes[conn], (1, 2, 0)))


def test_indexed_bad_entry(v):
    nodes, conn = synth.structured_grid(6, 5, 4, seed=24)
    conn = conn.copy()
    conn[11, 6] = -3
    got = v.corner_quality_indexed(torch.from_numpy(nodes).cuda(),
                                   torch.from_numpy(conn).cuda()).cpu().numpy()
    assert v.status() == -4 and np.isnan(got[11])
    assert np.all(np.isfinite(np.delete(got, 11)))
