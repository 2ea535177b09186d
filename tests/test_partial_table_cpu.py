"""The FP64 expressions of the partial redo (element64.cuh: sample64,
edge64), read from the CUDA source as text and evaluated here in numpy on
random elements, against the oracle.

The partial redo of an FP32 escalation evaluates single samples and edge
coefficients in FP64 by index: sample q < 8 is J at corner node q, sample
8 + e is C = 4 J at the midpoint of edge e (Sec. 5), and edge coefficient e
(scaled by 2) is that sample less the corner samples at the edge's two ends
(Sec. 4, Table t:Tsmall).  A wrong edge-vector index, a wrong end node or an
edge mapped to the wrong midpoint in these tables changes which sign is
redone, which the GPU parity tests catch only if such an element comes up;
here every entry is checked on every run.  The edge vectors follow the
element map of Appendix A: a[y + 2z] along xi at (eta, zeta) = (y, z),
b[x + 2z] along eta at (xi, zeta) = (x, z), g[x + 2y] along zeta at
(xi, eta) = (x, y).
"""
import os
import re

import numpy as np

import oracle
from paper_1706_01613_gb300 import synth

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1706_01613_gb300", "csrc")

# Appendix A: the reference-cube corner of each node
CORNER = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]


def node_at(x, y, z):
    return CORNER.index((x, y, z))


def edge_midpoint(e):
    """Midpoint of edge e in the numbering of the kernels: xi-edges at
    (eta, zeta) = (e & 1, e >> 1), then eta-edges at (xi, zeta), then
    zeta-edges at (xi, eta)."""
    if e < 4:
        return (0.5, e & 1, e >> 1)
    if e < 8:
        return ((e - 4) & 1, 0.5, (e - 4) >> 1)
    return ((e - 8) & 1, (e - 8) >> 1, 0.5)


def _function(name):
    src = open(os.path.join(CSRC, "element64.cuh")).read()
    start = src.index("double %s(" % name)
    return src[start:src.index("\n}\n", start)]


def _edges(X):
    a = [X[node_at(1, y, z)] - X[node_at(0, y, z)] for z in (0, 1) for y in (0, 1)]
    b = [X[node_at(x, 1, z)] - X[node_at(x, 0, z)] for z in (0, 1) for x in (0, 1)]
    g = [X[node_at(x, y, 1)] - X[node_at(x, y, 0)] for y in (0, 1) for x in (0, 1)]
    return a, b, g


def _samples(X):
    """The 20 cases of sample64, evaluated from their source text."""
    cases = re.findall(r"case (\d+): return (.*?);", _function("sample64"))
    assert sorted(int(q) for q, _ in cases) == list(range(20))
    a, b, g = _edges(X)
    env = {"a": a, "b": b, "g": g, "vadd": lambda u, v: u + v,
           "det3": lambda u, v, w: float(np.dot(u, np.cross(v, w)))}
    return {int(q): eval(expr, {"__builtins__": {}}, env) for q, expr in cases}


def _edge_ends():
    """The end nodes (ca, cb) of each edge as edge64 computes them, from its
    source text: three branches, e < 4, e < 8, else."""
    body = _function("edge64")
    pairs = re.findall(r"ca = node_at\((.*?)\);\s*cb = node_at\((.*?)\);", body)
    assert len(pairs) == 3
    ends = []
    for e in range(12):
        ca, cb = pairs[0 if e < 4 else 1 if e < 8 else 2]
        ev = lambda s: node_at(*eval("(%s)" % s, {"__builtins__": {}}, {"e": e}))
        ends.append((ev(ca), ev(cb)))
    return ends


def _lattice_index(X, c27, xi):
    """Index of the oracle's order-2 node at reference point xi, found by
    value (the oracle's samples are J at its 27 nodes)."""
    J = oracle.jacobian(X, xi)
    r = np.nonzero(c27 == J)[0]
    assert len(r) == 1
    return int(r[0])


def test_sample_table_is_J_at_corners_and_4J_at_edge_midpoints():
    rng = np.random.default_rng(20170030)
    for _ in range(20):
        X = synth.REF_CORNERS + rng.uniform(-0.3, 0.3, size=(8, 3))
        s = _samples(X)
        for q in range(8):
            J = oracle.jacobian(X, CORNER[q])
            assert abs(s[q] - J) <= 1e-12 * max(1.0, abs(J))
        for e in range(12):
            J = oracle.jacobian(X, edge_midpoint(e))
            assert abs(s[8 + e] - 4.0 * J) <= 1e-12 * max(1.0, abs(J))


def test_edge_coefficients_are_twice_the_oracle_bezier_coefficients():
    """edge64(e) = sample(8 + e) - corner(ca) - corner(cb) with edge64's own
    end nodes: twice the Bezier coefficient at the edge's midpoint lattice
    node (Table t:Tsmall's edge rows)."""
    rng = np.random.default_rng(20170031)
    ends = _edge_ends()
    for e, (ca, cb) in enumerate(ends):
        # the ends: the midpoint with its 0.5 coordinate set to 0 and to 1
        m = edge_midpoint(e)
        k = [i for i in range(3) if m[i] == 0.5][0]
        lo, hi = list(m), list(m)
        lo[k], hi[k] = 0, 1
        assert {ca, cb} == {node_at(*lo), node_at(*hi)}, e
    for _ in range(20):
        X = synth.REF_CORNERS + rng.uniform(-0.3, 0.3, size=(8, 3))
        s = _samples(X)
        c27, b27 = oracle.coefficients(X)
        for e, (ca, cb) in enumerate(ends):
            r = _lattice_index(X, c27, edge_midpoint(e))
            edge = s[8 + e] - s[ca] - s[cb]
            assert abs(edge - 2.0 * b27[r]) <= 1e-11 * max(1.0, abs(b27[r]))
