"""Pins of the oracle's learned-smoother network (CPU only)."""
import numpy as np

from oracle.band import build_band
from oracle.geometry import sphere
from oracle.mlp import MLP, correction, features, loss_and_grad, neighbour27
from oracle.operators import Operators
import synth


def _setup(dx=1 / 8):
    band = build_band(sphere(), dx)
    op = Operators(band)
    return band, op, op.A_matrix(1.0), op.diag_M()


def test_gradient_matches_central_differences():
    band, op, A, dM = _setup()
    mlp = MLP.init(3, scale=1.5)
    mlp.b1 += 0.05
    mlp.b2 += 0.05
    r = synth.random_band_vector(band.nb, 4)
    nb27 = neighbour27(band)
    L, grads = loss_and_grad(mlp, band, A, r, dM, nb27)
    rng = np.random.default_rng(5)
    params = mlp.params()
    for p, g in zip(params[:5], grads[:5]):
        for _ in range(6):
            idx = tuple(rng.integers(0, n) for n in p.shape)
            h = 1e-6
            old = p[idx]
            p[idx] = old + h
            Lp, _ = loss_and_grad(mlp, band, A, r, dM, nb27)
            p[idx] = old - h
            Lm, _ = loss_and_grad(mlp, band, A, r, dM, nb27)
            p[idx] = old
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, g[idx])
    # b3 (a scalar)
    h = 1e-6
    mlp.b3 += h
    Lp, _ = loss_and_grad(mlp, band, A, r, dM, nb27)
    mlp.b3 -= 2 * h
    Lm, _ = loss_and_grad(mlp, band, A, r, dM, nb27)
    mlp.b3 += h
    assert abs((Lp - Lm) / (2 * h) - grads[5][0]) <= 1e-6 * max(1.0, abs(grads[5][0]))


def test_correction_is_positively_homogeneous_and_zero_at_zero():
    band, op, A, dM = _setup()
    mlp = MLP.init(1)
    r = synth.random_band_vector(band.nb, 2)
    du1, _ = correction(mlp, band, r, dM)
    du2, _ = correction(mlp, band, 3.5 * r, dM)
    assert np.abs(du2 - 3.5 * du1).max() <= 1e-13 * np.abs(du2).max()
    du0, _ = correction(mlp, band, np.zeros(band.nb), dM)
    assert np.abs(du0).max() < 1e-250


def test_features_definition():
    """27-neighbourhood (a fastest, 0 off the band), scaled by its max; offsets; dx^2 M_ii."""
    band, op, A, dM = _setup()
    r = synth.random_band_vector(band.nb, 6)
    X, s = features(band, r, dM)
    ijk = band.coords_of(band.keys)
    for i in np.random.default_rng(0).choice(band.nb, 20, replace=False):
        vals = []
        for c in (-1, 0, 1):
            for b in (-1, 0, 1):
                for a in (-1, 0, 1):
                    key = band.key_of((ijk[i] + np.array([a, b, c]))[None, :])
                    j = band.index_in_band(key)[0]
                    vals.append(r[j] if j >= 0 else 0.0)
        vals = np.asarray(vals)
        assert np.allclose(X[i, :27] * s[i], vals, rtol=1e-15, atol=0)
        assert abs(s[i] - np.abs(vals).max()) <= 1e-15 * s[i] + 1e-300
        assert X[i, 13] * s[i] == r[i]
    assert np.allclose(X[:, 30], band.dx ** 2 * op.M.diagonal())
