"""Minimum of the Jacobian determinant to a tolerance (TEST INFRASTRUCTURE ONLY).

Sec. 1 and Sec. 3 of the paper (after [johnen2013]): by the convex hull
property the smallest Bezier coefficient of a box is a lower bound of J on
it, and the smallest corner coefficient (a value of J, at a corner of the
box) is an upper bound of the minimum; subdividing sharpens both.  Statement
followed here, breadth first with a depth cap D and an absolute tolerance
tol = rel_tol * max |b| (b the depth-0 coefficients):

    boxes = {root}; U = min of the root's corner coefficients; L = min of b
    level by level, while U - L > tol and the depth is below D:
        every box whose lower bound is below U - tol is split in 8 (the
        others cannot lower the answer by more than tol); U takes the
        smallest corner coefficient of the children; children whose lower
        bound is at least U are dropped; L = the smallest lower bound left
        (at most U).

Every value carries the oracle's certified error bound (coefficient_bounds at
depth 0, child_bound below): lower bounds are "coefficient - bound", upper
bounds "coefficient + bound", so the true minimum lies in [L, U].  Returns
(L, U, depth, converged).  Uses the C oracle's coefficients, subdivision and
bounds; only tests and the benchmark's CPU baseline may call it.
"""
import numpy as np

import oracle

CORNERS = list(range(8))  # the oracle's order: the 8 corner coefficients first


def min_jacobian(X, rel_tol=1e-6, max_depth=12):
    X = np.ascontiguousarray(X, dtype=np.float64)
    b, eb = oracle.coefficient_bounds(X)
    if not np.all(np.isfinite(X)):
        return np.nan, np.nan, 0, False
    E = float(eb.max())
    tol = rel_tol * float(np.abs(b).max())
    U = float(b[CORNERS].min()) + E
    L = min(U, float(b.min()) - E)
    boxes = [(b, E)]
    depth = 0
    settled = np.inf  # smallest lower bound of the boxes left unsplit so far
    while U - L > tol and depth < max_depth:
        u0 = U  # classification uses the level's starting U (order-free)
        kids = []
        for bb, e in boxes:
            lo = float(bb.min()) - e
            if lo >= u0:
                continue
            if lo >= u0 - tol:
                settled = min(settled, lo)
                continue
            ec = oracle.child_bound(e, bb)
            for ch in oracle.subdivide(bb):
                kids.append((ch, ec))
                U = min(U, float(ch[CORNERS].min()) + ec)
        depth += 1
        boxes = [(ch, ec) for ch, ec in kids if float(ch.min()) - ec < U]
        L = min([U, settled] + [float(ch.min()) - ec for ch, ec in boxes])
        if not kids:
            break
    return L, U, depth, U - L <= tol
