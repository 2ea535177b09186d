"""Independent mathematics used to pin the oracle (tests only).

Nothing here is shared with the oracle or the CUDA path, and it follows
different routes to the same quantities:
  * the trilinear map x(xi) of Appendix A evaluated directly, and its
    derivatives by central differences (exact for a map that is affine in
    each variable separately), J by a generic determinant;
  * Bezier coefficients by collocation: solving the Bernstein system
    A b = c with A built from the Bernstein polynomials of Sec. 3.1, instead
    of the printed Table t:Tb;
  * sub-box coefficients by collocation on the sub-box instead of de
    Casteljau;
  * the decision depth of an INVALID element from its characterisation on
    dyadic grids (see ``invalid_depth_bruteforce``).
"""
from fractions import Fraction
from math import comb

import numpy as np

# Appendix A: node k sits at these reference coordinates.
CORNERS = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
           (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]


def shape_values(xi, eta, zeta):
    """The eight trilinear shape functions of Appendix A, written out."""
    return [(1 - xi) * (1 - eta) * (1 - zeta), xi * (1 - eta) * (1 - zeta),
            xi * eta * (1 - zeta), (1 - xi) * eta * (1 - zeta),
            (1 - xi) * (1 - eta) * zeta, xi * (1 - eta) * zeta,
            xi * eta * zeta, (1 - xi) * eta * zeta]


def map_point(X, p):
    L = shape_values(*p)
    return [sum(L[k] * X[k][d] for k in range(8)) for d in range(3)]


def det3(m):
    """Cofactor expansion along the first row (works on Fractions)."""
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
            - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


def jac_exact(X, p, h=Fraction(1, 2)):
    """J at p from central differences of the map, exact on Fractions."""
    cols = []
    for j in range(3):
        pp = list(p)
        pm = list(p)
        pp[j] += h
        pm[j] -= h
        xp, xm = map_point(X, pp), map_point(X, pm)
        cols.append([(xp[d] - xm[d]) / (2 * h) for d in range(3)])
    # matrix with columns d/dxi, d/deta, d/dzeta
    m = [[cols[j][i] for j in range(3)] for i in range(3)]
    return det3(m)


def jac_numpy(X, pts, h=0.5):
    """J at many points (P, 3) in float64: central differences + numpy det."""
    X = np.asarray(X, float)
    pts = np.asarray(pts, float)

    def mp(q):
        x, y, z = q[:, 0], q[:, 1], q[:, 2]
        L = np.stack(shape_values(x, y, z), axis=1)  # (P, 8)
        return L @ X

    cols = []
    for j in range(3):
        dp = np.zeros(3)
        dp[j] = h
        cols.append((mp(pts + dp) - mp(pts - dp)) / (2 * h))
    M = np.stack(cols, axis=2)  # (P, 3 comps, 3 derivs)
    return np.linalg.det(M)


# ---- Bernstein basis and collocation (Sec. 3.1, 3.2) ------------------------

def bernstein(i, t):
    return comb(2, i) * t ** i * (1 - t) ** (2 - i)


# the paper's Greek ordering of the 27 coefficients (Fig. f:ordercoeff),
# tensor indices (i, j, k) = 2 * node coordinates
ORDER = [(0, 0, 0), (2, 0, 0), (2, 2, 0), (0, 2, 0), (0, 0, 2), (2, 0, 2), (2, 2, 2), (0, 2, 2),
         (1, 0, 0), (2, 1, 0), (1, 2, 0), (0, 1, 0), (0, 0, 1), (2, 0, 1), (2, 2, 1), (0, 2, 1),
         (1, 0, 2), (2, 1, 2), (1, 2, 2), (0, 1, 2),
         (1, 1, 0), (1, 0, 1), (2, 1, 1), (1, 2, 1), (0, 1, 1), (1, 1, 2),
         (1, 1, 1)]


def bezier_eval(b, pts):
    """sum_alpha b_alpha B_alpha(xi) at points (P, 3), float64."""
    pts = np.asarray(pts, float)
    out = np.zeros(len(pts))
    for a, (i, j, k) in enumerate(ORDER):
        out += (b[a] * bernstein(i, pts[:, 0]) * bernstein(j, pts[:, 1])
                * bernstein(k, pts[:, 2]))
    return out


def collocation_matrix():
    """A[alpha][beta] = B_beta(xi_alpha) with xi_alpha the order-2 nodes."""
    A = []
    for (ia, ja, ka) in ORDER:
        p = (Fraction(ia, 2), Fraction(ja, 2), Fraction(ka, 2))
        A.append([bernstein(i, p[0]) * bernstein(j, p[1]) * bernstein(k, p[2])
                  for (i, j, k) in ORDER])
    return A


def invert(A):
    """Gauss-Jordan inverse over Fractions."""
    n = len(A)
    M = [list(map(Fraction, row)) + [Fraction(int(i == j)) for j in range(n)]
         for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [v / pv for v in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * b for a, b in zip(M[r], M[col])]
    return [row[n:] for row in M]


_AINV = None


def ainv():
    global _AINV
    if _AINV is None:
        _AINV = invert(collocation_matrix())
    return _AINV


def box_coefficients_exact(X, lo, size):
    """Exact Bezier coefficients of J restricted to the box lo + [0,size]^3
    (reparametrised to the unit cube), by collocation."""
    c = [jac_exact(X, (lo[0] + size * Fraction(i, 2), lo[1] + size * Fraction(j, 2),
                       lo[2] + size * Fraction(k, 2))) for (i, j, k) in ORDER]
    Ai = ainv()
    return [sum(Ai[r][a] * c[a] for a in range(27)) for r in range(27)]


def to_fractions(X):
    return [[Fraction(float(v)) for v in row] for row in np.asarray(X, float)]


def verdict_bruteforce(X, max_depth):
    """Reference verdict and depth by collocation on sub-boxes (exact).

    Level 0: the 20 samples at corners and edge midpoints decide INVALID,
    all 27 root coefficients positive decide VALID.  Level d >= 1: every
    uncertified box of level d-1 is split into 8 boxes whose coefficients
    are obtained by collocation on the box itself; a non-positive corner
    coefficient anywhere on the level means INVALID@d, no uncertified box
    left means VALID@d, the cap means UNDECIDED@max_depth.
    Returns (verdict, depth) with verdict 1 valid, 2 invalid, 3 undecided."""
    Xf = to_fractions(X)
    samples = [jac_exact(Xf, (Fraction(i, 2), Fraction(j, 2), Fraction(k, 2)))
               for (i, j, k) in ORDER[:20]]
    if any(v <= 0 for v in samples):
        return 2, 0
    root = box_coefficients_exact(Xf, (0, 0, 0), Fraction(1))
    if all(v > 0 for v in root):
        return 1, 0
    if max_depth == 0:
        return 3, 0
    live = [(0, 0, 0)]  # integer box origins at the current level
    for level in range(1, max_depth + 1):
        size = Fraction(1, 2 ** level)
        kids = [(2 * x + dx, 2 * y + dy, 2 * z + dz) for (x, y, z) in live
                for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
        coeffs = [box_coefficients_exact(Xf, tuple(size * v for v in o), size) for o in kids]
        if any(v <= 0 for cf in coeffs for v in cf[:8]):
            return 2, level
        live = [o for o, cf in zip(kids, coeffs) if not all(v > 0 for v in cf[8:])]
        if not live:
            return 1, level
        if level == max_depth:
            return 3, level
    raise AssertionError


def invalid_depth_bruteforce(X, max_depth):
    """For an element with a non-positive J somewhere on a dyadic grid: the
    smallest d <= max_depth such that J <= 0 at a point of G_d, where G_0 is
    the 8 corners + 12 edge midpoints and G_d (d >= 1) the grid of spacing
    2^-d; None if no such d.  Every box containing such a point cannot be
    certified (its coefficients bound J from below), so the refinement
    reaches a box having the point as a corner at level d; hence INVALID@d
    holds exactly for this d."""
    Xf = to_fractions(X)
    g0 = [jac_exact(Xf, (Fraction(i, 2), Fraction(j, 2), Fraction(k, 2)))
          for (i, j, k) in ORDER[:20]]
    if any(v <= 0 for v in g0):
        return 0
    for d in range(1, max_depth + 1):
        m = 2 ** d
        for i in range(m + 1):
            for j in range(m + 1):
                for k in range(m + 1):
                    if jac_exact(Xf, (Fraction(i, m), Fraction(j, m), Fraction(k, m))) <= 0:
                        return d
    return None


_AINV_F = None


def verdict_collocation_float(X, max_depth, margin=1e-9):
    """Fast float64 version of ``verdict_bruteforce`` (collocation on every
    box, numpy).  Returns (verdict, depth), or None when a decisive value lies
    within margin * scale of zero (then only the exact check can tell)."""
    global _AINV_F
    if _AINV_F is None:
        _AINV_F = np.array([[float(v) for v in row] for row in ainv()])
    X = np.asarray(X, float)
    lat = np.array(ORDER, float) / 2.0
    scale = np.abs(jac_numpy(X, lat)).max()
    tol = margin * scale

    def box_coeffs(origins, size):
        pts = (origins[:, None, :] + size * lat[None, :, :]).reshape(-1, 3)
        c = jac_numpy(X, pts).reshape(len(origins), 27)
        return c @ _AINV_F.T * (size ** 3) / (size ** 3)

    c0 = jac_numpy(X, lat[:20])
    if np.any(np.abs(c0) <= tol):
        return None
    if np.any(c0 <= 0):
        return 2, 0
    b = box_coeffs(np.zeros((1, 3)), 1.0)
    if np.any(np.abs(b) <= tol):
        return None
    if np.all(b > 0):
        return 1, 0
    if max_depth == 0:
        return 3, 0
    live = np.zeros((1, 3))
    offs = np.array([[dx, dy, dz] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)], float)
    for level in range(1, max_depth + 1):
        size = 0.5 ** level
        kids = (live[:, None, :] + offs[None, :, :] * size).reshape(-1, 3)
        cf = box_coeffs(kids, size)
        if np.any(np.abs(cf) <= tol):
            return None
        if np.any(cf[:, :8] <= 0):
            return 2, level
        keep = ~np.all(cf[:, 8:] > 0, axis=1)
        live = kids[keep]
        if len(live) == 0:
            return 1, level
        if level == max_depth:
            return 3, level
    raise AssertionError
