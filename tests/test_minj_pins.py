"""Pins of the minimum-of-J oracle (branch and bound on the Bezier
coefficients, Sec. 1 and 3) against facts outside it: constant J on
parallelepipeds, the minimum of J sampled on the dyadic grid that contains
every box corner it can visit, the twisted prism's closed form, and sign
agreement with the validity verdict."""
import numpy as np
import pytest

import oracle
from oracle import minj
from paper_1706_01613_gb300 import synth

REF = synth.REF_CORNERS


def _grid_min(X, n=33):
    g = np.linspace(0.0, 1.0, n)
    return min(oracle.jacobian(X, (a, b, c)) for a in g for b in g for c in g)


@pytest.mark.parametrize("seed", range(3))
def test_parallelepiped_is_decided_at_depth_0(seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(3, 3))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    X = REF @ A.T + rng.normal(size=3)
    L, U, d, conv = minj.min_jacobian(X, 1e-9)
    assert conv and d == 0 and L <= np.linalg.det(A) <= U and U - L < 1e-9


@pytest.mark.parametrize("seed", range(6))
def test_interval_brackets_the_dyadic_grid_minimum(seed):
    """Boxes of depth <= 5 have their corners on the 33^3 grid, so the grid
    minimum lies in [L, U] (L bounds the true minimum from below, U is at
    least J at some grid point)."""
    X = synth.perturbed_cubes(1, noise=0.35, seed=100 + seed)[:, :, 0]
    L, U, d, conv = minj.min_jacobian(X, 1e-3, max_depth=5)
    m = _grid_min(X)
    assert L <= m + 1e-12 and m <= U + 1e-12
    if conv:
        assert U - L <= 1e-3 * np.abs(oracle.coefficients(X)[1]).max() + 1e-15


@pytest.mark.parametrize("theta", [30.0, 75.0, 110.0])
def test_twisted_prism_closed_form(theta):
    """Bottom face (+-1/2, +-1/2, 0), top face turned by theta at height t:
    the minimum of J is t (1 + cos theta) / 2 (closed form)."""
    t = 0.3
    c, s = np.cos(np.radians(theta)), np.sin(np.radians(theta))
    bottom = REF[:4, :2] - 0.5
    top = bottom @ np.array([[c, s], [-s, c]])
    X = np.concatenate([np.c_[bottom, np.zeros(4)], np.c_[top, np.full(4, t)]])
    L, U, _, conv = minj.min_jacobian(X, 1e-6, max_depth=14)
    want = t * (1 + c) / 2
    assert conv and L <= want <= U and U - L <= 1e-6 * np.abs(oracle.coefficients(X)[1]).max()


def test_sign_agrees_with_the_verdict():
    X = synth.perturbed_cubes(150, noise=0.55, seed=7)
    f, _, _ = oracle.check_soa(X, max_depth=12)
    for e in range(X.shape[2]):
        L, U, _, conv = minj.min_jacobian(X[:, :, e], 1e-6, max_depth=12)
        v = f[e] & 7
        if L > 0:
            assert v == oracle.VALID
        if U <= 0:
            assert v == oracle.INVALID
