"""Corner scaled Jacobian of the linear hexahedron (TEST INFRASTRUCTURE ONLY).

The quality measure the paper quotes in Sec. 7 (Fig. f:invalidHighCornerQual,
after Knupp and Yamakawa-Shimada): at each of the 8 corners, the determinant
of the three edge vectors leaving the corner, each divided by its length, in
the (xi, eta, zeta) orientation of the corner's Jacobian matrix; the element
measure is the minimum over the corners.  A corner with a zero-length edge
has the value 0.  Plain numpy in FP64.

Layout: corners float64 (8, 3, n) in the node order of Appendix A.  Only the
tests, the smoke check and the benchmark's CPU baseline may use this module.
"""
import numpy as np

# Appendix A reference corners
REF = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])


def _neighbours():
    """For corner k, the nodes one step away along xi, eta, zeta, and the
    sign that turns each edge into a column of the Jacobian at k (+1 if the
    step goes towards increasing reference coordinate)."""
    out = []
    for k in range(8):
        cols = []
        for d in range(3):
            t = REF[k].copy()
            t[d] = 1 - t[d]
            m = int(np.nonzero((REF == t).all(axis=1))[0][0])
            cols.append((m, 1.0 if REF[k][d] == 0 else -1.0))
        out.append(cols)
    return out


NBR = _neighbours()


def corner_scaled_jacobians(X):
    """(8, n) array: the scaled Jacobian at each corner."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[2]
    out = np.empty((8, n))
    for k in range(8):
        cols = []
        zero = np.zeros(n, bool)
        for m, s in NBR[k]:
            v = s * (X[m] - X[k])  # (3, n)
            ln = np.sqrt((v * v).sum(axis=0))
            zero |= ln == 0
            cols.append(v / np.where(ln > 0, ln, 1.0))
        a, b, c = cols
        det = (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0])
               + a[2] * (b[0] * c[1] - b[1] * c[0]))
        out[k] = np.where(zero, 0.0, det)
    return out


def min_scaled_jacobian(X):
    """(n,) minimum corner scaled Jacobian; NaN for non-finite input."""
    X = np.asarray(X, dtype=np.float64)
    with np.errstate(all="ignore"):
        q = corner_scaled_jacobians(X).min(axis=0)
    finite = np.all(np.isfinite(X.reshape(24, -1)), axis=0)
    return np.where(finite, q, np.nan)
