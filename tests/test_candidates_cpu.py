"""The candidate-set generator against the oracle: a candidate is a grid cell
with its corner labels permuted by a cube symmetry, so its map is the cell's
map composed with that symmetry and J changes by the factor det = +-1.  A
rotated candidate therefore has the cell's verdict and depth (the
subdivision at 1/2 commutes with the cube's symmetries); a reflected one is
INVALID at depth 0 (J changes sign everywhere, and a valid cell has positive
corners)."""
import numpy as np

import oracle
from paper_1706_01613_gb300 import synth


def test_symmetries_form_the_cube_group():
    perm, sign = synth.cube_symmetries()
    assert len({tuple(p) for p in perm}) == 48
    assert sorted(sign.tolist()) == [-1] * 24 + [1] * 24
    assert list(perm[np.argmax((perm == np.arange(8)).all(axis=1))]) == list(range(8))


def test_rotated_candidates_keep_the_cell_verdict_reflected_ones_are_invalid():
    nodes, conn, cell, sym = synth.hex_candidates(6, 6, sigma=0.3, seed=5)
    _, cells = synth.structured_grid(6, sigma=0.3, seed=5)
    fc, _, _ = oracle.check_indexed(nodes, conn, max_depth=8)
    fcell, _, _ = oracle.check_indexed(nodes, cells, max_depth=8)
    _, sign = synth.cube_symmetries()
    rot = sign[sym] > 0
    assert np.array_equal(fc[rot] & 0x7F, fcell[cell[rot]] & 0x7F)
    valid_cell = (fcell[cell] & 7) == oracle.VALID
    refl = ~rot & valid_cell
    assert np.all((fc[refl] & 0x7F) == oracle.INVALID)
    assert rot.sum() > 100 and refl.sum() > 100
