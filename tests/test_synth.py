"""Seeded input generators (CPU): determinism, ranges and closed forms."""
import numpy as np

import synth


def test_ellipsoid_batch_is_seeded_and_in_range():
    a = synth.ellipsoid_batch(seed=0, count=64)
    b = synth.ellipsoid_batch(seed=0, count=64)
    assert a == b and len(a) == 64
    axes = np.array([ax for ax, _ in a])
    assert axes.min() >= 0.6 and axes.max() <= 1.2
    assert {dx for _, dx in a} <= {1 / 64, 1 / 96, 1 / 128}
    assert len({dx for _, dx in a}) == 3  # uneven band sizes
    assert synth.ellipsoid_batch(seed=1, count=64) != a


def test_harmonic_fields_are_sphere_harmonics_on_the_sphere():
    """On the unit sphere harmonic_field is the u of sphere_harmonics (same
    coefficients), and the several-seed form equals the one-seed form."""
    rng = np.random.default_rng(3)
    y = rng.normal(size=(500, 3))
    y /= np.linalg.norm(y, axis=1, keepdims=True)
    for seed in (0, 5):
        u, _ = synth.sphere_harmonics(y, seed=seed)
        assert np.allclose(synth.harmonic_field(y, seed=seed), u, rtol=0, atol=1e-13)
    fs = synth.harmonic_fields(y, [0, 5])
    assert np.allclose(fs[1], synth.harmonic_field(y, seed=5), rtol=0, atol=1e-13)
    # radial invariance: the field depends on the direction only
    assert np.allclose(synth.harmonic_field(2.5 * y, seed=0), synth.harmonic_field(y, seed=0),
                       rtol=0, atol=1e-13)
