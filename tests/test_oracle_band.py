"""Pins of the oracle's band and stencils against the paper (CPU only)."""
import numpy as np
import pytest

from conftest import load_golden
from oracle.band import build_band, default_lambda2, stencil, table41_counts
from oracle.geometry import circle, closest_point, ellipsoid, sphere, torus


@pytest.mark.parametrize("row", load_golden("table41.txt")[:4])
def test_table41_exact(row):
    """Table 4.1: DOFs, nnz(L), nnz(E_3), nnz(M), bit-exact integers."""
    dx, dofs, nnzL, nnzE, nnzM = row
    band = build_band(sphere(), dx, ghost=False)
    got = table41_counts(band)
    assert got == {"dofs": int(dofs), "nnzL": int(nnzL), "nnzE": int(nnzE), "nnzM": int(nnzM)}


@pytest.mark.slow
def test_table41_row_00125():
    dx, dofs, nnzL, nnzE, nnzM = load_golden("table41.txt")[4]
    got = table41_counts(build_band(sphere(), dx, ghost=False))
    assert got == {"dofs": int(dofs), "nnzL": int(nnzL), "nnzE": int(nnzE), "nnzM": int(nnzM)}


def test_lambda_formula():
    """lambda^2 = (d-1)(p+1)^2/4 + (1+(p+1)/2)^2: 13 in 2-D, 17 in 3-D for cubic."""
    assert default_lambda2(2, 3) == 13.0
    assert default_lambda2(3, 3) == 17.0


def test_band_brute_force_circle():
    """Band of the circle at dx = 1/16 by an independent per-node loop (polar form)."""
    dx = 1.0 / 16
    band = build_band(circle(), dx)
    n = band.n
    keys = []
    for j in range(n):
        for i in range(n):
            x, y = -2 + i * dx, -2 + j * dx
            dist = abs(np.hypot(x, y) - 1.0)
            if dist * dist <= 13 * dx * dx * (1 + 1e-12):
                keys.append(i + n * j)
    assert np.array_equal(np.asarray(keys), band.keys)


def test_ghost_ring_and_stencils_sphere():
    band = build_band(sphere(), 1.0 / 16)
    assert band.nb == 26974
    # ghost nodes are outside the tube, neighbours of the band
    thr = 17 * (band.dx * band.dx)
    assert np.all(band.dist2[band.nb:] > thr)
    assert np.all(band.dist2[: band.nb] <= thr)
    nbk = band.neighbour_keys(band.keys)
    assert np.all(band.index_in_bplus(nbk.ravel()) >= 0)
    # every cubic stencil node of B+ lies in B (also checked in build_band)
    base, s = stencil(band.cp, band.lo, band.dx, 3)
    assert np.all((s >= 0) & (s < 1))
    for off in np.ndindex(4, 4, 4):
        assert np.all(band.index_in_band(band.key_of(base + np.asarray(off))) >= 0)


def test_closest_points_are_on_surface_and_normal():
    rng = np.random.default_rng(1)
    X = rng.uniform(-1.6, 1.6, size=(2000, 3))
    for surf, level in [
        (sphere(), lambda y: np.sqrt((y ** 2).sum(1)) - 1.0),
        (torus(1.0, 0.4), lambda y: np.hypot(np.hypot(y[:, 0], y[:, 1]) - 1.0, y[:, 2]) - 0.4),
        (ellipsoid(1.2, 0.8, 0.6), lambda y: ((y / np.array([1.2, 0.8, 0.6])) ** 2).sum(1) - 1.0),
    ]:
        cp, d2 = closest_point(surf, X)
        ok = np.isfinite(d2) & (d2 < surf.reach ** 2 * 0.8)
        assert ok.sum() > 50
        assert np.abs(level(cp[ok])).max() < 1e-12
        assert np.allclose(((X - cp) ** 2).sum(1)[ok], d2[ok], rtol=1e-12, atol=1e-14)
        # x - cp(x) is normal to S: brute force over nearby surface points
        for idx in np.nonzero(ok)[0][:20]:
            y = cp[idx]
            eps = 1e-4
            for _ in range(5):
                t = rng.normal(size=3)
                cand, _ = closest_point(surf, (y + eps * t)[None, :])
                assert ((X[idx] - cand[0]) ** 2).sum() >= d2[idx] - 1e-12


def test_ellipsoid_reduces_to_sphere():
    rng = np.random.default_rng(2)
    X = rng.uniform(-1.5, 1.5, size=(500, 3))
    cp_e, d_e = closest_point(ellipsoid(1.0, 1.0, 1.0), X)
    cp_s, d_s = closest_point(sphere(), X)
    assert np.allclose(cp_e, cp_s, atol=1e-13)
    assert np.allclose(d_e, d_s, atol=1e-13)


def test_circle_band_size():
    """Circle at dx = 1/64: 2912 band points (the circle workload)."""
    assert build_band(circle(), 1.0 / 64).nb == 2912


def test_ellipsoid_medial_disk_is_far():
    """Nodes on the ellipsoid's medial disk (smallest axis coordinate 0, inside)
    have no stationary point of the secular equation above -min a^2; they are
    at least the reach away from S (brute force over a dense surface sample)."""
    surf = ellipsoid(1.1, 0.8, 0.7)
    X = np.array([[0.25, 0.0, 0.0], [0.3, 0.05, 0.0]])
    _, d2 = closest_point(surf, X)
    assert np.all(np.isinf(d2))
    th, ph = np.meshgrid(np.linspace(0, 2 * np.pi, 721), np.linspace(0, np.pi, 361))
    Y = np.stack([1.1 * np.sin(ph) * np.cos(th), 0.8 * np.sin(ph) * np.sin(th), 0.7 * np.cos(ph)], -1).reshape(-1, 3)
    for x in X:
        assert np.sqrt(((Y - x) ** 2).sum(1)).min() >= surf.reach * 0.99


def _dziuk_surface_points(n=60, seed=0):
    rng = np.random.default_rng(seed)
    z = rng.uniform(-0.99, 0.99, n * n)
    t = rng.uniform(0, 2 * np.pi, n * n)
    rho = np.sqrt(1 - z * z)
    return np.stack([z * z + rho * np.cos(t), rho * np.sin(t), z], 1)


def _dziuk_normal(P):
    a = P[:, 0] - P[:, 2] ** 2
    g = np.stack([a, P[:, 1], P[:, 2] * (1 - 2 * a)], 1)
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def test_dziuk_closest_point_by_newton():
    """Sec. 4.5.5: points x = y + t n(y) off the Dziuk surface with |t| below the
    reach return cp(x) = y (the foot of the normal), on the surface, and dist2
    = t^2; the reach is the smallest radius of curvature (1 / 10.44)."""
    from oracle.geometry import DZIUK_REACH, _dziuk, dziuk_min_curvature_radius
    assert abs(dziuk_min_curvature_radius() - DZIUK_REACH) < 1e-3
    P = _dziuk_surface_points()
    nrm = _dziuk_normal(P)
    t = np.random.default_rng(1).uniform(-0.9, 0.9, len(P)) * DZIUK_REACH
    X = P + t[:, None] * nrm
    cp, d2 = _dziuk(X)
    assert np.abs(cp - P).max() < 1e-9
    assert np.abs(np.sqrt(d2) - np.abs(t)).max() < 1e-9


def test_dziuk_candidate_filter_keeps_the_tube():
    """The oracle's candidate filter (first-order distance with slack) keeps
    every point within 2 band half-widths of the surface at dx = 1/64."""
    from oracle.band import _candidate_filter
    from oracle.geometry import dziuk
    dx = 1 / 64
    margin = np.sqrt(17.0 * dx * dx) * 1.01 + 2 * dx
    P = _dziuk_surface_points(80, 2)
    nrm = _dziuk_normal(P)
    t = np.random.default_rng(3).uniform(-1.0, 1.0, len(P)) * 2 * margin
    assert _candidate_filter(dziuk(), P + t[:, None] * nrm, margin).all()
