"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle: J is evaluated from the map by central
differences, coefficients by collocation with the Bernstein basis, sub-box
coefficients by collocation on the sub-box, verdicts and depths by the
characterisations in ``_indep``.  A dropped term, a wrong sign or index, a
transposed operand or a wrong comparison in the oracle fails at least one of
them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1706_01613_gb300 import synth

from . import _indep as ind

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")
REF = synth.REF_CORNERS


def _examples():
    with open(GOLDEN) as f:
        return json.load(f)["examples"]


def _rand_hex(rng, noise=0.3):
    return REF + rng.uniform(-noise, noise, size=(8, 3))


# ---------------------------------------------------------------- tables ----

def test_table_T_is_inverse_of_bernstein_collocation():
    """Sec. 3.2: T = A^-1 with A_ab = B_b(xi_a).  Table t:Tb as transcribed
    must equal the inverse computed from the Bernstein polynomials."""
    Ai = ind.ainv()
    T = exact.table_T()
    assert all(T[r][c] == Ai[r][c] for r in range(27) for c in range(27))


def test_table_Q_reproduces_T_route_exactly():
    """Table t:Tsmall: b = Q c20 must equal T c27 (Sec. 4).  Q is transcribed
    here from the paper; rational check on random rational hexes."""
    h, q, e = Fraction(1, 2), Fraction(3, 4), Fraction(5, 8)
    Q = [[Fraction(0)] * 20 for _ in range(27)]
    for r in range(8):
        Q[r][r] = Fraction(1)
    for e_, (a, b) in enumerate(exact.EDGE_END):
        Q[8 + e_][a - 1] = -h
        Q[8 + e_][b - 1] = -h
        Q[8 + e_][8 + e_] = Fraction(2)
    for f in range(6):
        for k in range(4):
            Q[20 + f][exact.FACE_CORNER[f][k] - 1] = -q
            Q[20 + f][exact.FACE_EDGE[f][k] - 1] = Fraction(1)
    for a in range(8):
        Q[26][a] = -e
    for a in range(8, 20):
        Q[26][a] = h
    rng = np.random.default_rng(1)
    for _ in range(3):
        X = [[Fraction(int(v), 64) for v in row] for row in rng.integers(-80, 80, (8, 3))]
        c, b = exact.samples_and_coefficients(X)
        bq = [sum(Q[r][a] * c[a] for a in range(20)) for r in range(27)]
        assert bq == b


def test_seven_linear_relations_with_corrected_sign():
    """Sec. 4 (Corollary, Table t:7LinRel): b21..b27 depend linearly on
    b1..b20.  The relation that holds is b21 = 1/2 sum(b9..b12) - 1/4
    sum(b1..b4) (and b27 = 1/4 sum(edges) - 1/4 sum(corners)); the table
    prints the opposite overall sign, which a constant J = 1 rules out."""
    rng = np.random.default_rng(2)
    X = [[Fraction(int(v), 16) for v in row] for row in rng.integers(-20, 20, (8, 3))]
    _, b = exact.samples_and_coefficients(X)
    for f in range(6):
        lhs = b[20 + f]
        rhs = (Fraction(1, 2) * sum(b[k - 1] for k in exact.FACE_EDGE[f])
               - Fraction(1, 4) * sum(b[k - 1] for k in exact.FACE_CORNER[f]))
        assert lhs == rhs
    assert b[26] == Fraction(1, 4) * sum(b[8:20]) - Fraction(1, 4) * sum(b[:8])


# ------------------------------------------------------ J and coefficients --

def test_samples_are_J_at_order2_nodes():
    rng = np.random.default_rng(3)
    for _ in range(20):
        X = _rand_hex(rng)
        c, _ = oracle.coefficients(X)
        pts = np.array(ind.ORDER, float) / 2.0
        ref = ind.jac_numpy(X, pts)
        np.testing.assert_allclose(c, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_bezier_expansion_reproduces_J():
    """Eq. e:bezExpansion: sum b B must equal J everywhere (random points)."""
    rng = np.random.default_rng(4)
    for _ in range(30):
        X = _rand_hex(rng, noise=0.45)
        _, b = oracle.coefficients(X)
        pts = rng.uniform(0, 1, size=(200, 3))
        ref = ind.jac_numpy(X, pts)
        got = ind.bezier_eval(b, pts)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(b).max())


def test_corner_coefficients_are_corner_tetrahedra():
    """Sec. 3.1 / Sec. 5: b_1..b_8 are J at the corners = 6 vol of the corner
    tetrahedra, e.g. J_1 = det(v12, v14, v15)."""
    nbr = {0: (1, 3, 4), 1: (0, 2, 5), 2: (3, 1, 6), 3: (2, 0, 7),
           4: (5, 7, 0), 5: (4, 6, 1), 6: (7, 5, 2), 7: (6, 4, 3)}
    rng = np.random.default_rng(5)
    for _ in range(20):
        X = _rand_hex(rng)
        _, b = oracle.coefficients(X)
        for k in range(8):
            cols = []
            for d, m in enumerate(nbr[k]):
                v = X[m] - X[k]
                # the corner's xi_d coordinate is 1 when the neighbour lies below
                cols.append(v if REF[m][d] > REF[k][d] else -v)
            ref = np.linalg.det(np.stack(cols, axis=1))
            assert abs(b[k] - ref) <= 1e-13 * max(1.0, abs(ref))


def test_parallelepiped_gives_equal_coefficients():
    """An affine map has constant J = det(A): all 27 coefficients equal it."""
    rng = np.random.default_rng(6)
    for _ in range(20):
        A = rng.normal(size=(3, 3))
        t = rng.normal(size=3) * 5
        X = REF @ A.T + t
        _, b = oracle.coefficients(X)
        d = np.linalg.det(A)
        np.testing.assert_allclose(b, d, rtol=1e-12, atol=1e-12)
    _, b = oracle.coefficients(REF)
    assert np.all(b == 1.0)


def test_affine_transform_scales_and_translation_invariant():
    rng = np.random.default_rng(7)
    for _ in range(10):
        X = _rand_hex(rng)
        A = rng.normal(size=(3, 3))
        _, b0 = oracle.coefficients(X)
        _, b1 = oracle.coefficients(X @ A.T + rng.normal(size=3))
        np.testing.assert_allclose(b1, np.linalg.det(A) * b0, rtol=0,
                                   atol=1e-11 * np.abs(b0).max() * abs(np.linalg.det(A)))


def test_mean_coefficient_is_volume():
    """Each quadratic Bernstein polynomial integrates to 1/3, so sum(b)/27 =
    integral of J = volume; the volume here comes from 2x2x2 Gauss quadrature
    (exact for the triquadratic J)."""
    g = np.array([0.5 - 0.5 / math.sqrt(3), 0.5 + 0.5 / math.sqrt(3)])
    pts = np.array([[a, b, c] for a in g for b in g for c in g])
    rng = np.random.default_rng(8)
    for _ in range(20):
        X = _rand_hex(rng)
        _, b = oracle.coefficients(X)
        vol = ind.jac_numpy(X, pts).sum() / 8.0
        assert abs(b.sum() / 27.0 - vol) <= 1e-13 * max(1.0, abs(vol))


def test_closed_form_moved_corner():
    """Moving corner k towards the centre by 2s(centre - C_k) gives
    J = 1 - s(P2 P3 + P1 P3 + P1 P2) with P_d the affine coordinate equal to 1
    at that corner, hence b = 1 - s (i2 i3 + i1 i3 + i1 i2)/4 with i_d the
    tensor index counted from the far face; min J = 1 - 3s at the corner."""
    for k in range(8):
        for s in (0.1, 0.3, 1.0 / 3.0, 0.45):
            X = REF.copy()
            X[k] = REF[k] + 2 * s * (0.5 - REF[k])
            _, b = oracle.coefficients(X)
            for a, (i, j, l) in enumerate(ind.ORDER):
                loc = [t if REF[k][d] == 1 else 2 - t for d, t in enumerate((i, j, l))]
                want = 1 - s * (loc[1] * loc[2] + loc[0] * loc[2] + loc[0] * loc[1]) / 4.0
                assert abs(b[a] - want) < 1e-14
            assert abs(b[k] - (1 - 3 * s)) < 1e-14


def test_closed_form_twisted_prism():
    """Bottom square at z = 0, top square turned by theta at z = t:
    J = t (1 - 2 zeta (1 - zeta)(1 - cos theta)), whose Bezier coefficients
    are t (zeta index 0 or 2) and t cos(theta) (zeta index 1)."""
    for theta_deg in (10.0, 60.0, 100.0, 150.0, 179.0):
        th = math.radians(theta_deg)
        for t in (1.0, 0.01):
            X = synth.twisted_layers(1, noise=0.0)[:, :, 0]
            base = np.array([[-0.5, -0.5], [0.5, -0.5], [0.5, 0.5], [-0.5, 0.5]])
            X[4:8, 0] = base[:, 0] * math.cos(th) - base[:, 1] * math.sin(th)
            X[4:8, 1] = base[:, 0] * math.sin(th) + base[:, 1] * math.cos(th)
            X[4:8, 2] = t
            X[0:4, 2] = 0.0
            _, b = oracle.coefficients(X)
            for a, (i, j, l) in enumerate(ind.ORDER):
                want = t * (math.cos(th) if l == 1 else 1.0)
                assert abs(b[a] - want) < 1e-13
            for z in (0.0, 0.25, 0.5, 0.9):
                want = t * (1 - 2 * z * (1 - z) * (1 - math.cos(th)))
                assert abs(oracle.jacobian(X, (0.3, 0.7, z)) - want) < 1e-13


def test_convex_hull_on_dense_grid():
    """Sec. 3.1: min b <= min J and max J <= max b; checked on the 33^3 grid,
    for the root and for the 8 children of one subdivision on their boxes."""
    rng = np.random.default_rng(9)
    g = np.linspace(0.0, 1.0, 33)
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    for _ in range(4):
        X = _rand_hex(rng, noise=0.45)
        _, b = oracle.coefficients(X)
        J = ind.jac_numpy(X, P)
        tol = 1e-12 * np.abs(b).max()
        assert b.min() <= J.min() + tol and J.max() <= b.max() + tol
        kids = oracle.subdivide(b)
        for o in range(8):
            lo = np.array([o & 1, (o >> 1) & 1, (o >> 2) & 1]) * 0.5
            Jc = ind.jac_numpy(X, lo + 0.5 * P)
            assert kids[o].min() <= Jc.min() + tol and Jc.max() <= kids[o].max() + tol


def test_subdivision_is_restriction():
    """Children of the de Casteljau split are the Bezier coefficients of J on
    the sub-boxes: compared with collocation on each sub-box (exact input)."""
    rng = np.random.default_rng(10)
    for _ in range(2):
        X = np.round(_rand_hex(rng) * 64) / 64
        _, b = oracle.coefficients(X)
        kids = oracle.subdivide(b)
        Xf = ind.to_fractions(X)
        for o in range(8):
            lo = (Fraction(o & 1, 2), Fraction((o >> 1) & 1, 2), Fraction((o >> 2) & 1, 2))
            want = ind.box_coefficients_exact(Xf, lo, Fraction(1, 2))
            np.testing.assert_allclose(kids[o], [float(w) for w in want], rtol=0, atol=1e-13)


def test_exact_coefficients_on_dyadic_inputs():
    """Coordinates on a 1/16 grid: the exact coefficients (collocation over
    Fractions) must be matched by the FP64 oracle to within a few ulps."""
    rng = np.random.default_rng(11)
    for _ in range(5):
        X = np.round(_rand_hex(rng, noise=0.4) * 16) / 16
        _, b = oracle.coefficients(X)
        want = ind.box_coefficients_exact(ind.to_fractions(X), (0, 0, 0), Fraction(1))
        assert np.allclose(b, [float(w) for w in want], rtol=0, atol=1e-14)


# ----------------------------------------------------------- verdicts ------

def test_paper_worked_examples():
    """Sec. 7: the three printed hexahedra are invalid, valid, invalid."""
    exs = _examples()
    X = np.stack([np.array(e["nodes"], float) for e in exs], axis=2)
    flags, _, _ = oracle.check_soa(X, max_depth=8)
    want = {"valid": 1, "invalid": 2}
    assert [int(f) & 7 for f in flags] == [want[e["verdict"]] for e in exs]


def test_paper_worked_examples_depths_bruteforce():
    """Decision depths of the worked examples against the independent
    characterisations (collocation tree / dyadic-grid search)."""
    exs = _examples()
    X = np.stack([np.array(e["nodes"], float) for e in exs], axis=2)
    flags, _, _ = oracle.check_soa(X, max_depth=8)
    for e, f in zip(exs, flags):
        Xe = np.array(e["nodes"], float)
        if e["verdict"] == "invalid":
            assert int(f) >> 3 & 15 == ind.invalid_depth_bruteforce(Xe, 4)
        else:
            assert (int(f) & 7, int(f) >> 3 & 15) == ind.verdict_bruteforce(Xe, 3)


def test_third_example_corner_scaled_jacobian():
    """Fig. f:invalidHighCornerQual: min corner scaled Jacobian prints as 0.64."""
    e = _examples()[2]
    X = np.array(e["nodes"], float)
    nbr = {0: (1, 3, 4), 1: (2, 0, 5), 2: (3, 1, 6), 3: (0, 2, 7),
           4: (7, 5, 0), 5: (4, 6, 1), 6: (5, 7, 2), 7: (6, 4, 3)}
    q = []
    for k in range(8):
        v = [X[m] - X[k] for m in nbr[k]]
        v = [w / np.linalg.norm(w) for w in v]
        q.append(np.linalg.det(np.stack(v, axis=1)))
    assert math.floor(min(q) * 100) / 100 == e["min_corner_scaled_jacobian_2dp"]


def test_verdicts_match_bruteforce_on_random_small():
    """Random elements near the validity boundary; verdict and depth against
    the collocation tree (exact arithmetic, small cap)."""
    rng = np.random.default_rng(12)
    seen = set()
    cnt = 0
    while cnt < 40:
        X = np.round(_rand_hex(rng, noise=0.55) * 32) / 32
        f, _, _ = oracle.check_soa(X[:, :, None], max_depth=3)
        v, d = int(f[0]) & 7, int(f[0]) >> 3 & 15
        if (v, d) in seen and rng.uniform() < 0.8:
            continue
        seen.add((v, d))
        cnt += 1
        assert (v, d) == ind.verdict_bruteforce(X, 3), X
    assert {(1, 0), (2, 0)} <= seen and len(seen) >= 4


def test_verdicts_match_float_collocation_tree_many():
    """Hundreds of elements that need refinement (picked from strongly
    perturbed cubes and from prisms twisted by up to 180 degrees), against
    the collocation tree in float64; elements with a decisive value within
    1e-9 of zero are left to the exact checks."""
    rng = np.random.default_rng(17)
    A = np.stack([_rand_hex(rng, noise=0.6) for _ in range(12000)], axis=2)
    B = synth.twisted_layers(6000, seed=4242, theta_max_deg=180.0)
    X = np.concatenate([A, B], axis=2)
    flags, _, _ = oracle.check_soa(X, max_depth=6)
    deep = np.nonzero((flags >> 3) & 15 >= 1)[0]
    assert len(deep) > 300
    compared = 0
    for e in deep[:700]:
        want = ind.verdict_collocation_float(X[:, :, e], 6)
        if want is None:
            continue
        compared += 1
        assert (int(flags[e]) & 7, int(flags[e]) >> 3 & 15) == want, e
    assert compared > 250


def test_invalid_depth_characterisation():
    """INVALID@d iff d is the first dyadic level holding a point with J <= 0."""
    rng = np.random.default_rng(13)
    done = 0
    while done < 25:
        X = _rand_hex(rng, noise=0.6)
        f, _, _ = oracle.check_soa(X[:, :, None], max_depth=4)
        if int(f[0]) & 7 != 2:
            continue
        done += 1
        assert int(f[0]) >> 3 & 15 == ind.invalid_depth_bruteforce(X, 4)


def test_dense_sampling_agrees_with_verdict():
    """Brute force on a dense grid: a sampled J <= 0 forces INVALID, and a
    VALID element has J > 0 at every sample."""
    rng = np.random.default_rng(14)
    g = np.linspace(0.0, 1.0, 17)
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    X = np.stack([_rand_hex(rng, noise=0.5) for _ in range(300)], axis=2)
    flags, _, _ = oracle.check_soa(X, max_depth=8)
    for e in range(X.shape[2]):
        J = ind.jac_numpy(X[:, :, e], P)
        if J.min() <= -1e-12:
            assert flags[e] & 7 == 2
        if flags[e] & 7 == 1:
            assert J.min() > 0


# ------------------------------------------------- degenerate and edge cases

TWIST180 = np.array([[-0.5, -0.5, 0], [0.5, -0.5, 0], [0.5, 0.5, 0], [-0.5, 0.5, 0],
                     [0.5, 0.5, 1], [-0.5, 0.5, 1], [-0.5, -0.5, 1], [0.5, -0.5, 1]], float)


def test_degenerate_cases_go_exact():
    """Cases whose values are exactly zero need the exact tier: a collapsed
    edge (J = 0 at two corners), a flat element (J = 0 everywhere), and a
    prism twisted by exactly 180 degrees (J = (1 - 2 zeta)^2, zero at the
    midpoints of the four vertical edges).  All are INVALID@0."""
    X1 = REF.copy()
    X1[1] = X1[0]
    X2 = REF.copy()
    X2[:, 2] = 0.0
    X = np.stack([X1, X2, TWIST180], axis=2)
    flags, _, _ = oracle.check_soa(X, max_depth=6)
    assert [int(f) & 0x7F for f in flags] == [2, 2, 2]
    assert all(int(f) & 0x80 for f in flags)  # decided by the exact tier


def test_nonfinite_inputs():
    X = np.stack([REF.copy() for _ in range(3)], axis=2)
    X[2, 1, 0] = np.nan
    X[5, 0, 1] = np.inf
    flags, bmin, bmax = oracle.check_soa(X)
    assert list(flags & 7) == [4, 4, 1]
    assert np.isnan(bmin[0]) and np.isnan(bmax[1]) and bmin[2] == 1.0


def test_empty_and_indexed_agree_with_soa():
    flags, _, _ = oracle.check_soa(np.zeros((8, 3, 0)))
    assert flags.shape == (0,)
    nodes, conn = synth.structured_grid(6, 5, 4, sigma=0.3, seed=77)
    fi, lo_i, hi_i = oracle.check_indexed(nodes, conn, max_depth=8)
    fs, lo_s, hi_s = oracle.check_soa(synth.soa_from_indexed(nodes, conn), max_depth=8)
    assert np.array_equal(fi, fs) and np.array_equal(lo_i, lo_s) and np.array_equal(hi_i, hi_s)
    with pytest.raises(IndexError):
        bad = conn.copy()
        bad[3, 2] = nodes.shape[0]
        oracle.check_indexed(nodes, bad)


def test_undecided_at_cap():
    """An element that needs three or more levels to be certified stays
    UNDECIDED when the cap is two (checked against the collocation tree)."""
    rng = np.random.default_rng(15)
    for _ in range(20000):
        X = np.round(_rand_hex(rng, noise=0.5) * 64) / 64
        f, _, _ = oracle.check_soa(X[:, :, None], max_depth=8)
        if int(f[0]) & 7 == 1 and int(f[0]) >> 3 & 15 >= 3:
            break
    else:
        pytest.fail("no deep element found")
    f2, _, _ = oracle.check_soa(X[:, :, None], max_depth=2)
    assert (int(f2[0]) & 7, int(f2[0]) >> 3 & 15) == (3, 2) == ind.verdict_bruteforce(X, 2)


def test_twist_below_180_is_valid_at_level_1():
    """The prism twisted by theta < 180 degrees has zeta coefficients
    t (1, cos theta, 1); one split gives t (1, (1+cos)/2, (1+cos)/2) > 0, so
    it is VALID@1 whenever cos theta <= 0 (collocation tree agrees)."""
    th = math.radians(179.0)
    X = TWIST180.copy()
    base = X[0:4, 0:2].copy()
    X[4:8, 0] = base[:, 0] * math.cos(th) - base[:, 1] * math.sin(th)
    X[4:8, 1] = base[:, 0] * math.sin(th) + base[:, 1] * math.cos(th)
    f, _, _ = oracle.check_soa(X[:, :, None], max_depth=4)
    assert (int(f[0]) & 7, int(f[0]) >> 3 & 15) == (1, 1) == ind.verdict_bruteforce(X, 2)


def _cube_rotations():
    mats = []
    import itertools
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            M = np.zeros((3, 3))
            for r, c in enumerate(perm):
                M[r, c] = signs[r]
            if round(np.linalg.det(M)) == 1:
                mats.append(M)
    return mats


def _relabel(X, R):
    """Node k of the new element sits where the old map puts the rotated
    reference corner: X'[k] = X[index of R (C_k - 1/2) + 1/2]."""
    idx = {tuple(c): k for k, c in enumerate(REF.astype(int))}
    perm = [idx[tuple(np.rint(R @ (REF[k] - 0.5) + 0.5).astype(int))] for k in range(8)]
    return X[perm], perm


def test_verdict_invariant_under_cube_rotations():
    """Relabelling the nodes by one of the 24 rotations of the reference cube
    reparametrises J by that rotation; the dyadic subdivision grid is
    invariant, so verdict and depth must not change, and the coefficients
    must be permuted accordingly."""
    rng = np.random.default_rng(16)
    rots = _cube_rotations()
    assert len(rots) == 24
    lat = {tuple(v): a for a, v in enumerate(ind.ORDER)}
    picked = 0
    while picked < 30:
        X = _rand_hex(rng, noise=0.5)
        f, _, _ = oracle.check_soa(X[:, :, None], max_depth=6)
        if int(f[0]) >> 3 & 15 == 0 and picked >= 4:
            continue
        picked += 1
        Xs = np.stack([_relabel(X, R)[0] for R in rots], axis=2)
        fs, _, _ = oracle.check_soa(Xs, max_depth=6)
        assert np.all(fs == f[0])
        _, b = oracle.coefficients(X)
        for R in rots[:6]:
            _, b2 = oracle.coefficients(_relabel(X, R)[0])
            for a, v in enumerate(ind.ORDER):
                w = np.rint(R @ (np.array(v) - 1) + 1).astype(int)
                assert abs(b2[a] - b[lat[tuple(w)]]) <= 1e-13 * np.abs(b).max()


def test_error_bounds_hold_against_exact_values():
    """The certified bounds are upper bounds of the actual error: depth-0
    coefficients and two levels of children, against exact collocation
    (Fractions), on elements far from the origin (large rounding)."""
    rng = np.random.default_rng(18)
    for _ in range(4):
        X = _rand_hex(rng, noise=0.45) * rng.uniform(0.3, 3.0) + rng.uniform(-1e3, 1e3, 3)
        Xf = ind.to_fractions(X)
        b, eb = oracle.coefficient_bounds(X)
        ex = ind.box_coefficients_exact(Xf, (0, 0, 0), Fraction(1))
        err = [abs(Fraction(float(v)) - w) for v, w in zip(b, ex)]
        assert all(e <= Fraction(float(t)) for e, t in zip(err, eb))
        assert max(err) > 0  # the check is not vacuous
        level = [(b, float(eb.max()), (Fraction(0),) * 3, Fraction(1))]
        for _lv in range(2):
            nxt = []
            for bb, e, lo, size in level[:2]:
                ec = oracle.child_bound(e, bb)
                for o, kid in enumerate(oracle.subdivide(bb)):
                    h = size / 2
                    lo2 = (lo[0] + (o & 1) * h, lo[1] + ((o >> 1) & 1) * h,
                           lo[2] + ((o >> 2) & 1) * h)
                    ex = ind.box_coefficients_exact(Xf, lo2, h)
                    err = [abs(Fraction(float(v)) - w) for v, w in zip(kid, ex)]
                    assert max(err) <= Fraction(ec)
                    nxt.append((kid, ec, lo2, h))
            level = nxt


def _zero_corner_elements(n, seed):
    """Elements whose corner-1 Jacobian is exactly 0 (v15 = -(v12 + v14)/8
    with an exact sum) while J > 0 elsewhere near it; with full-mantissa
    coordinates the FP64 value of that sample is rounding noise of either
    sign, so only a certified comparison gets the exact verdict INVALID@0."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        a = np.array([1 + rng.uniform(0, .25), rng.uniform(0, .25), rng.uniform(0, .25)])
        b = np.array([rng.uniform(0, .25), 1 + rng.uniform(0, .25), rng.uniform(0, .25)])
        s = a + b
        if not (np.all(s - a == b) and np.all(s - b == a)):
            continue
        X = REF.copy()
        X[1], X[3], X[2] = a, b, s
        X[4] = -s * 0.125
        X[5], X[7], X[6] = a + [0, 0, 1.0], b + [0, 0, 1.0], s + [0, 0, 1.0]
        out.append(X)
    return np.stack(out, axis=2)


def test_exact_zero_sample_is_invalid():
    X = _zero_corner_elements(200, 19)
    c0 = np.array([oracle.coefficients(X[:, :, e])[0][0] for e in range(X.shape[2])])
    assert (c0 > 0).sum() > 20 and (c0 < 0).sum() > 20  # noise of both signs
    flags, _, _ = oracle.check_soa(X, max_depth=6)
    assert np.all(flags & 0x7F == 2)


def test_certified_bounds_never_violated():
    """The FP64 oracle's decisions never disagree with exact arithmetic on
    inputs built to sit close to the validity boundary."""
    X, kind, r = synth.affine_mixture(400, seed=99, r_max=1e-13)
    flags, _, _ = oracle.check_soa(X, max_depth=4)
    for e in np.nonzero(kind == 1)[0][:40]:
        want = exact.decide(X[:, :, e], 4) & 0x7F
        assert int(flags[e]) & 0x7F == want
