"""Pins of the oracle's barycentric interpolation against the paper (CPU only)."""
import itertools

import numpy as np

from oracle.band import build_band
from oracle.geometry import circle, sphere
from oracle.interp import interp_matrix, lagrange_1d, stencil_offsets, tensor_weights


def test_cubic_weights_closed_forms():
    """1-D cubic and linear weights from the proof of Theorem 3.3 (a = s dx)."""
    s = np.random.default_rng(0).uniform(0, 1, 1000)
    w3 = lagrange_1d(s, 3)
    w1 = lagrange_1d(s, 1)
    assert np.allclose(w3[:, 0], -s * (1 - s) * (2 - s) / 6, atol=1e-15)
    assert np.allclose(w3[:, 1], (1 + s) * (1 - s) * (2 - s) / 2, atol=1e-15)
    # remaining two by the mirror symmetry s -> 1 - s of the equispaced stencil
    assert np.allclose(w3[:, 2], (2 - (1 - s)) * (1 + (1 - s)) * s / 2, atol=1e-15)
    assert np.allclose(w3[:, 3], -(1 - s) * s * (1 + s) / 6, atol=1e-15)
    assert np.allclose(w1[:, 0], 1 - s, atol=1e-15)
    assert np.allclose(w1[:, 1], s, atol=1e-15)


def test_exact_node_is_kronecker():
    w = lagrange_1d(np.array([0.0]), 3)
    assert np.array_equal(w[0], [0.0, 1.0, 0.0, 0.0])


def test_bicubic_sign_pattern_fig32c():
    """Fig. 3.2(c): corners +, edge points -, centre points + for s in (0,1)^2."""
    rng = np.random.default_rng(1)
    expect = np.array([[+1, -1, -1, +1], [-1, +1, +1, -1], [-1, +1, +1, -1], [+1, -1, -1, +1]])
    for _ in range(200):
        fr = rng.uniform(0.01, 0.99, size=(1, 2))
        W = tensor_weights(fr, 3).reshape(4, 4)  # [y][x]
        assert np.array_equal(np.sign(W), expect)


def test_tricubic_corners_negative_remark():
    """Remark after Theorem 3.3: in 3-D the corner weights are negative."""
    fr = np.random.default_rng(2).uniform(0.01, 0.99, size=(100, 3))
    W = tensor_weights(fr, 3).reshape(-1, 4, 4, 4)
    for c in itertools.product((0, 3), repeat=3):
        assert np.all(W[(slice(None),) + c] < 0)


def test_partition_of_unity_and_polynomial_reproduction():
    """E reproduces every x^a y^b z^c with a, b, c <= 3 exactly (tensor cubic)."""
    band = build_band(sphere(), 1.0 / 8)
    rng = np.random.default_rng(3)
    y = rng.normal(size=(400, 3))
    y /= np.linalg.norm(y, axis=1)[:, None]
    E = interp_matrix(band, y, 3)
    X = band.points(band.keys)
    for a, b, c in itertools.product(range(4), repeat=3):
        vals = X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c
        exact = y[:, 0] ** a * y[:, 1] ** b * y[:, 2] ** c
        assert np.abs(E @ vals - exact).max() < 1e-12
    # degree 4 in one variable is not reproduced (the test can fail)
    vals = X[:, 0] ** 4
    assert np.abs(E @ vals - y[:, 0] ** 4).max() > 1e-6


def test_linear_transfer_reproduces_bilinear():
    band = build_band(circle(), 1.0 / 16)
    y = np.random.default_rng(4).uniform(-1, 1, size=(300, 2))
    y /= np.linalg.norm(y, axis=1)[:, None]
    E1 = interp_matrix(band, y, 1)
    X = band.points(band.keys)
    for a, b in itertools.product(range(2), repeat=2):
        assert np.abs(E1 @ (X[:, 0] ** a * X[:, 1] ** b) - y[:, 0] ** a * y[:, 1] ** b).max() < 1e-13


def test_stencil_offsets_order():
    offs = stencil_offsets(3, 3)
    assert offs.shape == (64, 3)
    assert list(offs[1]) == [1, 0, 0] and list(offs[4]) == [0, 1, 0] and list(offs[16]) == [0, 0, 1]
