"""Pins of the oracle's exact rational tier below depth 0 (Sec. 6 subdivision).

``oracle/exact.py`` settles the elements whose certified FP64 signs are
inconclusive.  Its depth-0 part is pinned elsewhere; here its subdivision
(``subdivide``) and its breadth-first refinement loop (``decide`` at depth >=
1) are checked against the independent collocation route of ``_indep``:
Bezier coefficients of J on each sub-box obtained by solving the Bernstein
system on that box, and the collocation tree of verdicts built from them.
Every comparison is exact (``fractions.Fraction``).
"""
from fractions import Fraction

import numpy as np

import oracle
from oracle import exact
from paper_1706_01613_gb300 import synth

from . import _indep as ind

REF = synth.REF_CORNERS


def _coarse_dyadic(n, seed):
    """Unit cubes with every coordinate moved by a multiple of 1/4 in
    [-0.5, 0.5]: J takes small-denominator values, so exact zeros at box
    corners below depth 0 are common and the FP64 bound cannot settle them."""
    rng = np.random.default_rng(seed)
    return REF[:, :, None] + np.round(rng.uniform(-0.6, 0.6, size=(8, 3, n)) * 4) / 4


def _box_origin(path):
    """Lower corner of the box reached by child indices `path` (o = sx + 2 sy
    + 4 sz at each level), and its size."""
    lo = [Fraction(0)] * 3
    size = Fraction(1)
    for o in path:
        size /= 2
        for d in range(3):
            lo[d] += size * ((o >> d) & 1)
    return tuple(lo), size


def test_exact_subdivide_is_restriction_over_two_levels():
    """Children and grandchildren of the exact de Casteljau split equal the
    collocation coefficients of J on the same boxes, exactly."""
    rng = np.random.default_rng(41)
    for _ in range(2):
        X = np.round((REF + rng.uniform(-0.4, 0.4, size=(8, 3))) * 16) / 16
        Xf = ind.to_fractions(X)
        _, b = exact.samples_and_coefficients(Xf)
        assert b == ind.box_coefficients_exact(Xf, (0, 0, 0), Fraction(1))
        kids = exact.subdivide(b)
        for o in range(8):
            lo, size = _box_origin([o])
            assert kids[o] == ind.box_coefficients_exact(Xf, lo, size), o
        o1 = int(rng.integers(8))
        grand = exact.subdivide(kids[o1])
        for o2 in range(8):
            lo, size = _box_origin([o1, o2])
            assert grand[o2] == ind.box_coefficients_exact(Xf, lo, size), (o1, o2)


def test_exact_refinement_matches_collocation_tree():
    """Elements the C oracle hands to the exact tier with a verdict below
    depth 0 (coarse dyadic coordinates, exact zeros or near-ties on box
    corners): the exact tier's verdict and depth, reached through its
    refinement loop, equal the collocation tree's, for VALID and INVALID at
    depths 1 to 3; and with a cap below that depth the element is
    UNDECIDED at the cap in both."""
    X = _coarse_dyadic(8000, 33)
    flags, _, _ = oracle.check_soa(X, max_depth=4)
    deep = np.nonzero(((flags & 0x80) != 0) & (((flags >> 3) & 15) >= 1))[0]
    by_class = {}
    for e in deep:
        by_class.setdefault((int(flags[e]) & 7, int(flags[e]) >> 3 & 15), []).append(int(e))
    assert {(1, 1), (1, 2), (1, 3), (2, 2)} <= set(by_class), by_class.keys()
    for (v, d), elems in sorted(by_class.items()):
        for e in elems[:3]:
            f = exact.decide(X[:, :, e], 4)
            assert f & 0x80 and (f & 7, f >> 3 & 15) == (v, d)
            assert (v, d) == ind.verdict_bruteforce(X[:, :, e], 4), e
    e = by_class[(1, 3)][0]
    for cap in (1, 2):
        f = exact.decide(X[:, :, e], cap)
        assert (f & 7, f >> 3 & 15) == (3, cap) == ind.verdict_bruteforce(X[:, :, e], cap)
