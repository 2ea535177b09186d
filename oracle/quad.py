"""Oracle of the validity test of the linear quadrangle (TEST INFRASTRUCTURE ONLY).

Sec. 2.1 of the paper: the map of a linear quadrangle with the shape
functions L1 = (1-xi)(1-eta), L2 = xi(1-eta), L3 = xi eta, L4 = (1-xi) eta
(nodes 1..4 at (0,0), (1,0), (1,1), (0,1)) is bilinear, so its Jacobian
determinant J = sum_k L_k J_k is bilinear too, with J_k the value of J at
corner k.  Its minimum is therefore one of the four J_k, and the element is
valid iff all four are positive (strictly, as for the hexahedron).

Plain numpy in FP64: J at each corner from the derivatives of the shape
functions (Eq. e:determinant2D's Jacobian matrix), each sign certified by a
forward-error bound of the expression tree on absolute values; a corner
whose sign the bound cannot settle sends the element to exact rational
arithmetic (``fractions``).  Flags (the hexahedron's byte): verdict in bits
0-2 (1 valid, 2 invalid, 4 non-finite input), depth 0, bit 7 = decided
exactly.  jmin/jmax = min/max of the four J_k (the Bezier coefficients of a
bilinear J are its corner values).

Layouts: corners float64 (4, 2, n) (node-major, then x/y); indexed: nodes
float64 (n_nodes, 2), conn int32 (n, 4).  Only tests, the smoke check and
the benchmark's CPU baseline may use this module.
"""
from fractions import Fraction

import numpy as np

VALID, INVALID, NONFINITE = 1, 2, 4

# reference coordinates of nodes 1..4
REF = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float64)


def dshape(xi, eta):
    """d L_k / d xi and d L_k / d eta at (xi, eta), k = 1..4."""
    dxi = np.array([-(1 - eta), (1 - eta), eta, -eta], dtype=object)
    deta = np.array([-(1 - xi), -xi, xi, (1 - xi)], dtype=object)
    return dxi, deta


# derivative weights at the four corners (exact small integers)
_W = [dshape(int(x), int(y)) for x, y in REF]


def corner_jacobians(X):
    """J at the four corners, float64 (4, n), with their error bounds (4, n)."""
    X = np.asarray(X, dtype=np.float64)
    u = 2.0 ** -53
    J = np.empty((4, X.shape[2]))
    E = np.empty_like(J)
    for k, (wx, we) in enumerate(_W):
        wx = np.array(wx, dtype=np.float64)
        we = np.array(we, dtype=np.float64)
        # Jacobian matrix entries: sums of 4 weighted coordinates (3 roundings)
        xx = sum(wx[m] * X[m, 0] for m in range(4))
        yx = sum(wx[m] * X[m, 1] for m in range(4))
        xe = sum(we[m] * X[m, 0] for m in range(4))
        ye = sum(we[m] * X[m, 1] for m in range(4))
        ax = sum(abs(wx[m]) * np.abs(X[m, 0]) for m in range(4))
        ay = sum(abs(wx[m]) * np.abs(X[m, 1]) for m in range(4))
        bx = sum(abs(we[m]) * np.abs(X[m, 0]) for m in range(4))
        by = sum(abs(we[m]) * np.abs(X[m, 1]) for m in range(4))
        J[k] = xx * ye - xe * yx
        # each product term passes through <= 3 + 1 + 1 roundings
        E[k] = 8 * u * (ax * by + bx * ay) + 4.9e-324
    return J, E


def _exact_corners(X):
    """Exact J at the four corners of one element (4, 2) as Fractions."""
    P = [[Fraction(float(v)) for v in row] for row in X]
    out = []
    for wx, we in _W:
        xx = sum(Fraction(int(wx[m])) * P[m][0] for m in range(4))
        yx = sum(Fraction(int(wx[m])) * P[m][1] for m in range(4))
        xe = sum(Fraction(int(we[m])) * P[m][0] for m in range(4))
        ye = sum(Fraction(int(we[m])) * P[m][1] for m in range(4))
        out.append(xx * ye - xe * yx)
    return out


def check(X):
    """Verdicts of n quadrangles given as (4, 2, n) float64 planes."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    assert X.ndim == 3 and X.shape[:2] == (4, 2)
    n = X.shape[2]
    flags = np.zeros(n, np.uint8)
    with np.errstate(all="ignore"):
        J, E = corner_jacobians(X)
    finite = np.all(np.isfinite(X.reshape(8, n)), axis=0)
    nonpos = np.any(J <= -E, axis=0)
    amb = np.any(np.abs(J) <= E, axis=0)
    flags[:] = np.where(nonpos, INVALID, np.where(amb, 0x80, VALID))
    for e in np.nonzero(finite & ~nonpos & amb)[0]:
        Jx = _exact_corners(X[:, :, e])
        flags[e] = (INVALID if any(v <= 0 for v in Jx) else VALID) | 0x80
    flags[~finite] = NONFINITE
    jmin = np.where(finite, J.min(axis=0), np.nan)
    jmax = np.where(finite, J.max(axis=0), np.nan)
    return flags, jmin, jmax


def check_indexed(nodes, conn):
    """Verdicts of the quadrangles of an indexed 2D mesh."""
    nodes = np.asarray(nodes, dtype=np.float64)
    conn = np.asarray(conn)
    X = np.transpose(nodes[conn], (1, 2, 0))  # (4, 2, n)
    return check(X)
