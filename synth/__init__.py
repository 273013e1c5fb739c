"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds only input generation: random draws from seeded numpy
generators and closed-form surface fields evaluated at points the caller
passes in (each side passes its own closest points).  It contains none of the
method's arithmetic (no closest points, interpolation, Laplacian or solver).

Workloads (shapes of the paper's experiments, Sec. 3.4 and Sec. 4.5):

* ``circle_fourier``  u = sin(theta) + cos(3 theta) on the unit circle,
  f = -u'' + c u = (1+c) sin(theta) + (9+c) cos(3 theta).
* ``sphere_harmonics``  u = sum a_lm Y_lm over l in {2, 3, 5}, m = -l..l
  (23 real orthonormal harmonics, l ascending then m ascending), a_lm ~ N(0,1)
  from ``numpy.random.default_rng(seed)``; since -Lap_S Y_lm = l(l+1) Y_lm,
  f = sum (c + l(l+1)) a_lm Y_lm.
* ``torus_paper``  the torus example of Sec. 4.5.4: u = sin(3 theta) +
  cos(2 phi) with f from the paper's closed form (re-derived).
* ``u_rand``  a smooth field sum_{j=1..8} prod_{a} sin(k_{j,a} y_a + phi_{j,a}),
  k_j integer vectors, 0 < |k_j| <= 4 (rejection sampling), phi ~ U[0, 2 pi).
* ``random_band_vector``  uniform [-1, 1) values (operator parity tests).
* ``ellipsoid_batch``  the batched workload: semi-axes ~ U[0.6, 1.2]^3 and a
  spacing drawn from {1/64, 1/96, 1/128} per instance.
* ``harmonic_field``  sum a_lm Y_lm(y / |y|) over l in {2, 3, 5} (a
  spherical-harmonic-like right-hand side on any star-shaped surface).
"""
from __future__ import annotations

from math import factorial, pi, sqrt

import numpy as np

SPHERE_DEGREES = (2, 3, 5)


def sphere_coefficients(seed: int = 0, degrees=SPHERE_DEGREES) -> list[tuple[int, int, float]]:
    """[(l, m, a_lm)] with a_lm ~ N(0,1); 23 entries for l in {2,3,5}."""
    lm = [(l, m) for l in degrees for m in range(-l, l + 1)]
    a = np.random.default_rng(seed).standard_normal(len(lm))
    return [(l, m, float(v)) for (l, m), v in zip(lm, a)]


def _assoc_legendre(l: int, m: int, x: np.ndarray) -> np.ndarray:
    """P_l^m(x), m >= 0, without the Condon-Shortley phase (upward recurrence)."""
    pmm = np.ones_like(x)
    if m > 0:
        somx2 = np.sqrt(np.maximum(0.0, (1.0 - x) * (1.0 + x)))
        fact = 1.0
        for _ in range(m):
            pmm = pmm * fact * somx2
            fact += 2.0
    if l == m:
        return pmm
    pmmp1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pmmp1
    pll = pmmp1
    for ll in range(m + 2, l + 1):
        pll = ((2 * ll - 1) * x * pmmp1 - (ll + m - 1) * pmm) / (ll - m)
        pmm, pmmp1 = pmmp1, pll
    return pll


def real_sph_harm(l: int, m: int, y: np.ndarray) -> np.ndarray:
    """Orthonormal real Y_lm at unit vectors y (N, 3); theta azimuth, phi polar."""
    x, yy, z = y[:, 0], y[:, 1], y[:, 2]
    r = np.sqrt(x * x + yy * yy + z * z)
    ct = z / r
    theta = np.arctan2(yy, x)
    am = abs(m)
    norm = sqrt((2 * l + 1) / (4 * pi) * factorial(l - am) / factorial(l + am))
    P = _assoc_legendre(l, am, ct)
    if m == 0:
        return norm * P
    if m > 0:
        return sqrt(2.0) * norm * P * np.cos(am * theta)
    return sqrt(2.0) * norm * P * np.sin(am * theta)


def sphere_harmonics(y: np.ndarray, c=1.0, seed: int = 0, degrees=SPHERE_DEGREES):
    """(u, f) at points y on the unit sphere (u exact, f = (c - Lap_S) u)."""
    u = np.zeros(y.shape[0])
    f = np.zeros(y.shape[0])
    cc = np.broadcast_to(np.asarray(c, dtype=np.float64), (y.shape[0],))
    for l, m, a in sphere_coefficients(seed, degrees):
        Y = real_sph_harm(l, m, y)
        u += a * Y
        f += a * (l * (l + 1)) * Y
    return u, f + cc * u


def circle_fourier(y: np.ndarray, c=1.0):
    """(u, f) for u = sin(theta) + cos(3 theta) on the unit circle."""
    th = np.arctan2(y[:, 1], y[:, 0])
    u = np.sin(th) + np.cos(3 * th)
    f = np.sin(th) + 9.0 * np.cos(3 * th) + np.asarray(c) * u
    return u, f


def circle_mode(y: np.ndarray, k: int, c=1.0):
    """(u, f) for u = cos(k theta): -Lap_S u = k^2 u."""
    th = np.arctan2(y[:, 1], y[:, 0])
    u = np.cos(k * th)
    return u, (k * k + np.asarray(c)) * u


def torus_paper(y: np.ndarray, R: float = 1.2, r: float = 0.6, c=1.0):
    """(u, f) of Sec. 4.5.4: u = sin(3 theta) + cos(2 phi) on the torus (R, r)."""
    th = np.arctan2(y[:, 1], y[:, 0])
    rho = np.sqrt(y[:, 0] ** 2 + y[:, 1] ** 2)
    ph = np.arctan2(y[:, 2], rho - R)
    u = np.sin(3 * th) + np.cos(2 * ph)
    rc = R + r * np.cos(ph)
    f = (9 * np.sin(3 * th) / rc ** 2
         - 2 * np.sin(ph) * np.sin(2 * ph) / (r * rc)
         + 4 * np.cos(2 * ph) / r ** 2
         + np.asarray(c) * u)
    return u, f


def u_rand_params(seed: int = 0, terms: int = 8, kmax: float = 4.0):
    rng = np.random.default_rng(seed)
    ks, phs = [], []
    while len(ks) < terms:
        k = rng.integers(-4, 5, size=3)
        n2 = int((k * k).sum())
        if 0 < n2 <= kmax * kmax:
            ks.append(k)
            phs.append(rng.uniform(0.0, 2 * pi, size=3))
    return np.asarray(ks, dtype=np.float64), np.asarray(phs)


def u_rand(y: np.ndarray, seed: int = 0) -> np.ndarray:
    ks, phs = u_rand_params(seed)
    out = np.zeros(y.shape[0])
    for k, ph in zip(ks, phs):
        term = np.ones(y.shape[0])
        for a in range(3):
            term = term * np.sin(k[a] * y[:, a] + ph[a])
        out += term
    return out


def mixed_rhs(y: np.ndarray, seed: int = 0) -> np.ndarray:
    """f = (1 + 0.5 x y) u_rand(y) (mixed-precision workload)."""
    return (1.0 + 0.5 * y[:, 0] * y[:, 1]) * u_rand(y, seed)


def variable_c(y: np.ndarray) -> np.ndarray:
    """c(y) = 1 + 0.5 sin(2 pi z) (learned-smoother workload)."""
    return 1.0 + 0.5 * np.sin(2 * pi * y[:, 2])


def random_band_vector(n: int, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=n)


def ellipsoid_batch(seed: int = 0, count: int = 64, lo: float = 0.6, hi: float = 1.2,
                    spacings=(1 / 64, 1 / 96, 1 / 128)):
    """[(semi-axes (a, b, c), dx)] for ``count`` instances."""
    rng = np.random.default_rng(seed)
    axes = rng.uniform(lo, hi, size=(count, 3))
    pick = rng.integers(0, len(spacings), size=count)
    return [(tuple(float(v) for v in axes[i]), float(spacings[pick[i]])) for i in range(count)]


def harmonic_field(y: np.ndarray, seed: int = 0, degrees=SPHERE_DEGREES) -> np.ndarray:
    """sum a_lm Y_lm(y / |y|), a_lm ~ N(0, 1) from the seed."""
    return harmonic_fields(y, [seed], degrees)[0]


def harmonic_fields(y: np.ndarray, seeds, degrees=SPHERE_DEGREES) -> list[np.ndarray]:
    """``harmonic_field`` for several seeds (the harmonics evaluated once)."""
    d = y / np.linalg.norm(y, axis=1, keepdims=True)
    lm = [(l, m) for l in degrees for m in range(-l, l + 1)]
    Y = np.stack([real_sph_harm(l, m, d) for l, m in lm], axis=1)
    return [Y @ np.array([a for _, _, a in sphere_coefficients(s, degrees)]) for s in seeds]


def sphere_vardiff(y: np.ndarray, c=1.0):
    """Variable-diffusion example on the unit sphere (Sec. 4.5.6): with the polar
    angle phi (cos phi = z), u = cos phi, a = cos phi + 1.5 and
    f = 2 cos phi (cos phi + 1.5) - sin^2 phi + c u.  Returns (u, a, f) at y."""
    z = y[:, 2] / np.linalg.norm(y, axis=1)
    u = z
    a = z + 1.5
    f = 2.0 * z * (z + 1.5) - (1.0 - z * z) + c * u
    return u, a, f


def dziuk_rhs(y: np.ndarray, c=1.0):
    """Exact solution u = x1 x2 on the Dziuk surface (x1 - x3^2)^2 + x2^2 + x3^2 = 1
    and f = -Lap_S u + c u at points y of the surface (Sec. 4.5.5).  With
    n = g / |g|, g = (a, x2, x3 (1 - 2a)), a = x1 - x3^2 and p = grad u =
    (x2, x1, 0): Lap_S u = -2 n1 n2 - (p.n) div(n), where
    div(n) = div(g) / |g| - g.grad(|g|^2) / (2 |g|^3), div(g) = 3 - 2a + 4 x3^2.
    Returns (u, f)."""
    x1, x2, x3 = y[:, 0], y[:, 1], y[:, 2]
    a = x1 - x3 * x3
    g = np.stack([a, x2, x3 * (1.0 - 2.0 * a)], axis=1)
    s2 = (g * g).sum(axis=1)
    s = np.sqrt(s2)
    n = g / s[:, None]
    # gradient of |g|^2 = a^2 + x2^2 + x3^2 (1 - 2a)^2
    ds1 = 2.0 * a - 4.0 * x3 * x3 * (1.0 - 2.0 * a)
    ds2 = 2.0 * x2
    ds3 = -4.0 * a * x3 + 2.0 * x3 * (1.0 - 2.0 * a) ** 2 + 8.0 * x3 ** 3 * (1.0 - 2.0 * a)
    div_g = 3.0 - 2.0 * a + 4.0 * x3 * x3
    div_n = div_g / s - (g[:, 0] * ds1 + g[:, 1] * ds2 + g[:, 2] * ds3) / (2.0 * s2 * s)
    pn = x2 * n[:, 0] + x1 * n[:, 1]
    u = x1 * x2
    lap = -2.0 * n[:, 0] * n[:, 1] - pn * div_n
    return u, -lap + c * u

