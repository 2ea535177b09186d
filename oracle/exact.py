"""Exact-arithmetic tier of the CPU oracle (TEST INFRASTRUCTURE ONLY).

The FP64 oracle (``hexval_oracle.c``) certifies every sign decision with a
forward-error bound.  An element whose verdict depends on a value inside its
bound is recomputed here with ``fractions.Fraction``: every FP64 input is a
dyadic rational, J is a cubic polynomial in the inputs, and the Bezier
coefficients and their de Casteljau refinements are dyadic combinations of J
samples, so rational arithmetic gives the exact verdict.

It follows the same statement of the method as the C oracle:
  * J from Eq. e:det3d with the shape-function derivatives of Appendix A,
  * the 27 samples in the order of Fig. f:ordercoeff and b = T c (Table t:Tb),
  * the decision of Sec. 6 evaluated breadth first with a depth cap.
Only tests, the smoke check and the benchmark's CPU baseline may call it.
"""
from fractions import Fraction

VALID, INVALID, UNDECIDED, NONFINITE = 1, 2, 3, 4

# Appendix A node order, reference coordinates.
REF_NODE = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
            (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]

# Fig. f:ordercoeff: order-2 nodes, coordinates x2.
LAT2 = [(0, 0, 0), (2, 0, 0), (2, 2, 0), (0, 2, 0), (0, 0, 2), (2, 0, 2), (2, 2, 2), (0, 2, 2),
        (1, 0, 0), (2, 1, 0), (1, 2, 0), (0, 1, 0), (0, 0, 1), (2, 0, 1), (2, 2, 1), (0, 2, 1),
        (1, 0, 2), (2, 1, 2), (1, 2, 2), (0, 1, 2),
        (1, 1, 0), (1, 0, 1), (2, 1, 1), (1, 2, 1), (0, 1, 1), (1, 1, 2),
        (1, 1, 1)]

EDGE_END = [(1, 2), (2, 3), (3, 4), (1, 4), (1, 5), (2, 6),
            (3, 7), (4, 8), (5, 6), (6, 7), (7, 8), (5, 8)]
FACE_CORNER = [(1, 2, 3, 4), (1, 2, 5, 6), (2, 3, 6, 7),
               (3, 4, 7, 8), (1, 4, 5, 8), (5, 6, 7, 8)]
FACE_EDGE = [(9, 10, 11, 12), (9, 13, 14, 17), (10, 14, 15, 18),
             (11, 15, 16, 19), (12, 13, 16, 20), (17, 18, 19, 20)]


def table_T():
    """Table t:Tb as exact rationals, block by block."""
    T = [[Fraction(0)] * 27 for _ in range(27)]
    for r in range(8):
        T[r][r] = Fraction(1)
    for e, (a, b) in enumerate(EDGE_END):
        r = 8 + e
        T[r][a - 1] = Fraction(-1, 2)
        T[r][b - 1] = Fraction(-1, 2)
        T[r][r] = Fraction(2)
    for f in range(6):
        r = 20 + f
        for q in range(4):
            T[r][FACE_CORNER[f][q] - 1] = Fraction(1, 4)
            T[r][FACE_EDGE[f][q] - 1] = Fraction(-1)
        T[r][r] = Fraction(4)
    for a in range(8):
        T[26][a] = Fraction(-1, 8)
    for a in range(8, 20):
        T[26][a] = Fraction(1, 2)
    for a in range(20, 26):
        T[26][a] = Fraction(-2)
    T[26][26] = Fraction(8)
    return T


_T = table_T()
_ALPHA = {lat: a for a, lat in enumerate(LAT2)}


def _dshape(k, j, xi):
    v = Fraction(1)
    for d in range(3):
        on = REF_NODE[k][d]
        l = xi[d] if on else 1 - xi[d]
        dl = 1 if on else -1
        v *= dl if d == j else l
    return v


def jacobian(X, xi):
    """Eq. e:det3d at the reference point xi (exact)."""
    Jm = [[sum(X[k][i] * _dshape(k, j, xi) for k in range(8)) for j in range(3)]
          for i in range(3)]
    perms = [((0, 1, 2), 1), ((1, 2, 0), 1), ((2, 0, 1), 1),
             ((0, 2, 1), -1), ((2, 1, 0), -1), ((1, 0, 2), -1)]
    return sum(s * Jm[p[0]][0] * Jm[p[1]][1] * Jm[p[2]][2] for p, s in perms)


def samples_and_coefficients(X):
    """c (27 samples at the order-2 nodes) and b = T c, exact."""
    c = [jacobian(X, tuple(Fraction(v, 2) for v in lat)) for lat in LAT2]
    b = [sum(_T[r][a] * c[a] for a in range(27) if _T[r][a]) for r in range(27)]
    return c, b


def subdivide(b):
    """Quadratic de Casteljau split at 1/2 along each axis -> 8 children
    (child o = sx + 2 sy + 4 sz), each in the Fig. f:ordercoeff order."""
    A = {}
    for a, (i, j, k) in enumerate(LAT2):
        A[(i, j, k)] = b[a]

    def split(p0, p1, p2):
        l1 = (p0 + p1) / 2
        r1 = (p1 + p2) / 2
        return [p0, l1, (l1 + r1) / 2, r1, p2]

    A1 = {}
    for j in range(3):
        for k in range(3):
            for i, v in enumerate(split(A[(0, j, k)], A[(1, j, k)], A[(2, j, k)])):
                A1[(i, j, k)] = v
    A2 = {}
    for i in range(5):
        for k in range(3):
            for j, v in enumerate(split(A1[(i, 0, k)], A1[(i, 1, k)], A1[(i, 2, k)])):
                A2[(i, j, k)] = v
    G = {}
    for i in range(5):
        for j in range(5):
            for k, v in enumerate(split(A2[(i, j, 0)], A2[(i, j, 1)], A2[(i, j, 2)])):
                G[(i, j, k)] = v
    out = []
    for o in range(8):
        sx, sy, sz = o & 1, (o >> 1) & 1, (o >> 2) & 1
        child = [None] * 27
        for (i, j, k), a in _ALPHA.items():
            child[a] = G[(2 * sx + i, 2 * sy + j, 2 * sz + k)]
        out.append(child)
    return out


def decide(X_float, max_depth):
    """Exact verdict of one element: returns the flag byte (bit 7 set to mark
    that the exact tier produced it)."""
    X = [[Fraction(float(v)) for v in row] for row in X_float]
    c, b = samples_and_coefficients(X)
    if any(v <= 0 for v in c[:20]):
        return INVALID | 0x80
    if all(v > 0 for v in b):
        return VALID | 0x80
    if max_depth == 0:
        return UNDECIDED | 0x80
    boxes = [b]
    for level in range(1, max_depth + 1):
        kids = [ch for box in boxes for ch in subdivide(box)]
        if any(v <= 0 for box in kids for v in box[:8]):
            return INVALID | (level << 3) | 0x80
        boxes = [box for box in kids if not all(v > 0 for v in box[8:])]
        if not boxes:
            return VALID | (level << 3) | 0x80
        if level == max_depth:
            return UNDECIDED | (level << 3) | 0x80
    raise AssertionError("unreachable")
