"""Pins of the corner scaled Jacobian oracle: the paper's printed value for
Fig. f:invalidHighCornerQual, closed forms (unit cube, parallelepipeds),
invariances, Hadamard's inequality, degenerate corners, and agreement of its
sign with the corner Bezier coefficients of the validity oracle."""
import math

import numpy as np
import pytest

import oracle
from oracle import quality
from paper_1706_01613_gb300 import synth

from . import test_oracle_pins as pins

REF = quality.REF.astype(float)


def test_paper_example_prints_as_0_64():
    e = pins._examples()[2]
    X = np.array(e["nodes"], float)[:, :, None]
    q = quality.min_scaled_jacobian(X)[0]
    assert math.floor(q * 100) / 100 == e["min_corner_scaled_jacobian_2dp"]
    f, _, _ = oracle.check_soa(X, max_depth=8)
    assert f[0] & 7 == oracle.INVALID  # high corner quality, yet invalid


def test_unit_cube_is_one_everywhere():
    assert np.allclose(quality.corner_scaled_jacobians(REF[:, :, None]), 1.0, atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_parallelepiped_closed_form(seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(3, 3))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    X = (REF @ A.T + rng.normal(size=3))[:, :, None]
    want = np.linalg.det(A) / np.prod(np.linalg.norm(A, axis=0))
    assert np.allclose(quality.corner_scaled_jacobians(X)[:, 0], want, atol=1e-12)


def test_invariances():
    X = synth.perturbed_cubes(200, noise=0.3, seed=3)
    q = quality.corner_scaled_jacobians(X)
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    Y = np.einsum("ij,kjn->kin", Q, X) * 7.5 + np.array([100.0, -3.0, 2.0])[None, :, None]
    assert np.allclose(quality.corner_scaled_jacobians(Y), q, atol=1e-12)
    Z = X.copy()
    Z[:, 0, :] *= -1  # reflection: every corner changes sign
    assert np.allclose(quality.corner_scaled_jacobians(Z), -q, atol=1e-12)


def test_hadamard_and_sign_of_corner_coefficients():
    X = synth.perturbed_cubes(300, noise=0.6, seed=5)
    q = quality.corner_scaled_jacobians(X)
    assert np.all(np.abs(q) <= 1 + 1e-12)
    for e in range(X.shape[2]):
        _, b = oracle.coefficients(X[:, :, e])  # b[:8]: corner coefficients, node order
        assert np.all(np.sign(q[:, e]) == np.sign(b[:8])) or np.any(np.abs(b[:8]) < 1e-12)


def test_collapsed_edge_gives_zero_at_its_corners():
    X = REF.copy()
    X[1] = X[0]  # nodes 1 and 2 coincide
    q = quality.corner_scaled_jacobians(X[:, :, None])[:, 0]
    assert q[0] == 0.0 and q[1] == 0.0
    assert np.all(q[2:] > 0)


def test_nonfinite_is_nan():
    X = synth.perturbed_cubes(3, seed=6)
    X[4, 2, 1] = np.inf
    q = quality.min_scaled_jacobian(X)
    assert np.isnan(q[1]) and np.isfinite(q[0]) and np.isfinite(q[2])
