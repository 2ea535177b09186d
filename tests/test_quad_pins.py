"""Pins of the quadrangle oracle (Sec. 2.1) against facts the paper and the
mathematics fix, none of which re-types the oracle's formula:

* the bilinear interpolation of the corner values reproduces J computed by
  central differences of the map at interior points (this fixes which value
  belongs to which corner);
* J1 + J3 = J2 + J4 (Fig. f:areas), exactly on integer inputs;
* the mean of the corner values is the area (shoelace formula, Green);
* J at corner k is twice the signed area of the triangle of corner k;
* special shapes: unit square, parallelograms, bow-tie, dart, clockwise,
  three collinear nodes (J = 0 exactly), translation/scaling laws;
* the minimum of J over a dense grid is attained at a corner;
* the exact tier decides constructed elements whose corner value is known in
  closed form but lies far inside the FP64 error bound.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import quad

REF = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)


def _map(P, xi, eta):
    L = np.array([(1 - xi) * (1 - eta), xi * (1 - eta), xi * eta, (1 - xi) * eta])
    return L @ P


def _fd_jacobian(P, xi, eta, h=1e-6):
    dxi = (_map(P, xi + h, eta) - _map(P, xi - h, eta)) / (2 * h)
    deta = (_map(P, xi, eta + h) - _map(P, xi, eta - h)) / (2 * h)
    return dxi[0] * deta[1] - deta[0] * dxi[1]


def _one(P):
    return np.asarray(P, float).reshape(4, 2, 1)


def _random_quads(n, seed, noise=0.3):
    rng = np.random.default_rng(seed)
    return REF[:, :, None] + rng.uniform(-noise, noise, size=(4, 2, n))


def test_bilinear_interpolation_of_corner_values_is_the_jacobian():
    X = _random_quads(50, 1)
    J, _ = quad.corner_jacobians(X)
    rng = np.random.default_rng(2)
    for e in range(X.shape[2]):
        for _ in range(5):
            xi, eta = rng.uniform(0.05, 0.95, 2)
            L = np.array([(1 - xi) * (1 - eta), xi * (1 - eta), xi * eta, (1 - xi) * eta])
            assert abs(L @ J[:, e] - _fd_jacobian(X[:, :, e], xi, eta)) < 1e-7


def test_area_relation_exact_on_integers():
    rng = np.random.default_rng(3)
    X = rng.integers(-1000, 1000, size=(4, 2, 500)).astype(float)
    J, _ = quad.corner_jacobians(X)  # exact: integer products below 2^53
    assert np.array_equal(J[0] + J[2], J[1] + J[3])


def test_mean_corner_value_is_the_shoelace_area():
    X = _random_quads(200, 4)
    J, _ = quad.corner_jacobians(X)
    x, y = X[:, 0], X[:, 1]
    area = 0.5 * (x * np.roll(y, -1, axis=0) - np.roll(x, -1, axis=0) * y).sum(axis=0)
    assert np.allclose(J.mean(axis=0), area, rtol=0, atol=1e-14)


def test_corner_value_is_twice_the_corner_triangle_area():
    X = _random_quads(100, 5)
    J, _ = quad.corner_jacobians(X)
    for k in range(4):
        p, nxt, prv = X[k], X[(k + 1) % 4], X[(k - 1) % 4]
        a, b = nxt - p, prv - p
        tri = a[0] * b[1] - a[1] * b[0]  # 2 x signed area of (p, next, previous)
        assert np.allclose(J[k], tri, atol=1e-14)


@pytest.mark.parametrize("A", [np.eye(2), [[2.0, 0.5], [-0.3, 1.5]], [[0.1, 3.0], [-2.0, 0.2]]])
def test_parallelograms_have_equal_corner_values(A):
    A = np.asarray(A, float)
    X = _one(REF @ A.T + np.array([3.0, -7.0]))
    f, lo, hi = quad.check(X)
    assert lo[0] == pytest.approx(np.linalg.det(A), abs=1e-14)
    assert hi[0] == pytest.approx(np.linalg.det(A), abs=1e-14)
    assert f[0] & 7 == quad.VALID


def test_translation_and_scaling():
    X = _random_quads(100, 6)
    J, _ = quad.corner_jacobians(X)
    J2, _ = quad.corner_jacobians(3.0 * X + 11.0)
    assert np.allclose(J2, 9.0 * J, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("name,P,want", [
    ("square", [[0, 0], [1, 0], [1, 1], [0, 1]], quad.VALID),
    ("bow-tie", [[0, 0], [1, 0], [0, 1], [1, 1]], quad.INVALID),
    ("dart", [[0, 0], [2, 0], [0.5, 0.5], [0, 2]], quad.INVALID),
    ("clockwise", [[0, 0], [0, 1], [1, 1], [1, 0]], quad.INVALID),
    ("collinear", [[0, 0], [1, 0], [2, 0], [0, 1]], quad.INVALID),
    ("kite", [[0, 0], [2, -1], [3, 2], [-1, 2]], quad.VALID),
])
def test_shapes(name, P, want):
    f, lo, _ = quad.check(_one(P))
    assert f[0] & 7 == want, name
    if name == "collinear":
        assert lo[0] == 0.0  # J = 0 exactly at node 2: not strictly positive


def test_minimum_over_a_grid_is_at_a_corner():
    X = _random_quads(30, 7, noise=0.45)
    J, _ = quad.corner_jacobians(X)
    g = np.linspace(0.0, 1.0, 41)
    for e in range(X.shape[2]):
        vals = [sum(w * J[k, e] for k, w in enumerate(
            [(1 - a) * (1 - b), a * (1 - b), a * b, (1 - a) * b])) for a in g for b in g]
        assert min(vals) >= J[:, e].min() - 1e-14


@pytest.mark.parametrize("s", [2.0 ** -12, -(2.0 ** -12), 0.0])
def test_exact_tier_decides_inside_the_bound(s):
    """A unit square translated to 2^40 whose node 3 is shifted by s along x:
    J at corner 4 is exactly s + 1 - 1 = s (closed form: (x3 - x4) (y4 - y1)
    with x3 - x4 = 1 + s - 1 by construction below), far inside the FP64
    bound of the translated coordinates."""
    t = 2.0 ** 40
    P = np.array([[t, t], [t + 1, t], [t + s, t + 1], [t, t + 1]])
    # corner 4 (0,1): d/dxi = n3 - n4 = (s, 0), d/deta = n4 - n1 = (0, 1) -> J4 = s
    f, _, _ = quad.check(_one(P))
    _, E = quad.corner_jacobians(_one(P))
    assert E[3, 0] > abs(s)  # undecidable in FP64
    assert f[0] & 0x80
    assert f[0] & 7 == (quad.VALID if s > 0 else quad.INVALID)


def test_nonfinite():
    X = _random_quads(5, 8)
    X[2, 1, 3] = np.nan
    X[0, 0, 4] = np.inf
    f, lo, _ = quad.check(X)
    assert list(f[3:] & 7) == [quad.NONFINITE, quad.NONFINITE]
    assert np.isnan(lo[3]) and np.isnan(lo[4])


def test_indexed_matches_soa():
    rng = np.random.default_rng(9)
    nodes = rng.uniform(-1, 1, size=(50, 2))
    nodes[:4] = REF
    conn = rng.integers(0, 50, size=(300, 4)).astype(np.int32)
    conn[0] = [0, 1, 2, 3]
    a = quad.check_indexed(nodes, conn)
    b = quad.check(np.transpose(nodes[conn], (1, 2, 0)))
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=True)
    assert a[0][0] & 7 == quad.VALID


def test_printed_corner_expressions():
    """Eq. e:determinant2D attaches x43 y14 - y43 x14 to L3 and x43 y23 -
    y43 x23 to L4; evaluating both at a non-symmetric quadrangle shows that
    the first is J at (0,1) (node 4) and the second J at (1,1) (node 3), i.e.
    the printed L3/L4 labels are swapped; the text's definition (J_k = J at
    corner k) is what the oracle follows."""
    P = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 2.0], [0.0, 1.0]])
    d = lambda i, j, c: P[j - 1][c] - P[i - 1][c]  # noqa: E731
    printed_L3 = d(4, 3, 0) * d(1, 4, 1) - d(4, 3, 1) * d(1, 4, 0)
    printed_L4 = d(4, 3, 0) * d(2, 3, 1) - d(4, 3, 1) * d(2, 3, 0)
    assert printed_L3 == pytest.approx(_fd_jacobian(P, 0.0 + 1e-9, 1.0 - 1e-9), abs=1e-5)
    assert printed_L4 == pytest.approx(_fd_jacobian(P, 1.0 - 1e-9, 1.0 - 1e-9), abs=1e-5)
    J, _ = quad.corner_jacobians(_one(P))
    assert (J[2, 0], J[3, 0]) == (printed_L4, printed_L3)
    assert Fraction(J[0, 0]) + Fraction(J[2, 0]) == Fraction(J[1, 0]) + Fraction(J[3, 0])
