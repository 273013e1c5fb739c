"""Closest-point functions cp(x) and squared distances (Sec. 2.1).

TEST INFRASTRUCTURE ONLY (see the package header): the product path never
imports this module.

cp(x) is the point of the surface S nearest to x in Euclidean distance, well
defined inside a tube B(S) around S (Sec. 2.1).  Every function here takes an
(N, d) float64 array of grid-node coordinates and returns ``(cp, dist2)``:
the closest points (N, d) and the squared distances |x - cp(x)|^2 (N,).

Floating-point evaluation order is fixed and written out operation by
operation (numpy never fuses a multiply and an add), because the band is the
set {x : dist2(x) <= lambda^2 dx^2} and band membership is compared bit for
bit with the CUDA path:

* circle / sphere (centre 0, radius R):
      r   = sqrt((x0*x0 + x1*x1) + x2*x2)
      d   = r - R ;  dist2 = d*d
      t   = R / r ;  cp_a = x_a * t
* torus about the z axis (major radius R, minor radius r):  Sec. 4.5.4 gives
  the parametrisation; the closest point is the nearest point of the tube
  circle of the nearest point of the centre circle:
      rho = sqrt(x*x + y*y) ; a = rho - R ; q = sqrt(a*a + z*z)
      d   = q - r ;  dist2 = d*d
      s   = r / q ;  m = R + a*s ;  k = m / rho
      cp  = (x*k, y*k, z*s)
* ellipsoid with semi-axes (a0, a1, a2): cp_i = a_i^2 x_i / (a_i^2 + t) where
  t is the root, t > -min(a_i^2), of  sum_i a_i^2 x_i^2 / (a_i^2 + t)^2 = 1
  (the Lagrange condition for minimising |y - x|^2 on the surface).  The
  oracle finds t by plain bisection to the last bit (slow, obviously
  convergent: the function is strictly decreasing on that interval), with
      ax_i = |x_i| * a_i ;  bracket [-min a_i^2, sqrt((ax0^2+ax1^2)+ax2^2)+1e-300]
      mid = 0.5*(lo+hi), stop when mid equals an end of the bracket
      g_i = ax_i / (a_i^2 + mid) ;  F = ((g0*g0 + g1*g1) + g2*g2) - 1
      F > 0 -> lo = mid, else hi = mid ;  t = 0.5*(lo+hi)
      if F was never positive the node lies on the medial disk (the stationary
      point is not the minimiser; the node is >= reach from S): dist2 = inf
      cp_i = (a_i^2 * x_i) / (a_i^2 + t) ;  dist2 = (d0*d0 + d1*d1) + d2*d2
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CIRCLE, SPHERE, TORUS, ELLIPSOID, DZIUK = "circle", "sphere", "torus", "ellipsoid", "dziuk"

# Smallest radius of curvature of the Dziuk surface (x1 - x3^2)^2 + x2^2 + x3^2 = 1,
# 1 / 10.44 near x3 = +-0.92, from the principal curvatures on a fine parameter
# grid of the surface (``dziuk_min_curvature_radius``, pinned by a test).
DZIUK_REACH = 0.0957


@dataclass(frozen=True)
class Surface:
    """A closed curve (d = 2) or surface (d = 3) with a closed-form cp."""

    kind: str
    params: tuple = field(default_factory=tuple)

    @property
    def dim(self) -> int:
        return 2 if self.kind == CIRCLE else 3

    @property
    def reach(self) -> float:
        """Smallest radius of curvature: the tube B(S) on which cp is unique."""
        if self.kind in (CIRCLE, SPHERE):
            return float(self.params[0])
        if self.kind == TORUS:
            R, r = self.params
            return float(min(r, R - r))
        if self.kind == ELLIPSOID:
            a = sorted(self.params)
            return float(a[0] ** 2 / a[-1])
        if self.kind == DZIUK:
            return DZIUK_REACH
        raise ValueError(self.kind)


def circle(R: float = 1.0) -> Surface:
    return Surface(CIRCLE, (float(R),))


def sphere(R: float = 1.0) -> Surface:
    return Surface(SPHERE, (float(R),))


def torus(R: float, r: float) -> Surface:
    return Surface(TORUS, (float(R), float(r)))


def ellipsoid(a0: float, a1: float, a2: float) -> Surface:
    return Surface(ELLIPSOID, (float(a0), float(a1), float(a2)))


def dziuk() -> Surface:
    """The level set (x1 - x3^2)^2 + x2^2 + x3^2 = 1 of Sec. 4.5.5."""
    return Surface(DZIUK, ())


def _round_sphere(X: np.ndarray, R: float):
    if X.shape[1] == 2:
        r = np.sqrt(X[:, 0] * X[:, 0] + X[:, 1] * X[:, 1])
    else:
        r = np.sqrt((X[:, 0] * X[:, 0] + X[:, 1] * X[:, 1]) + X[:, 2] * X[:, 2])
    d = r - R
    dist2 = d * d
    # the centre (r = 0) has no closest point: t = inf there and cp = 0 * inf = nan
    with np.errstate(divide="ignore", invalid="ignore"):
        t = R / r
        cp = X * t[:, None]
    return cp, dist2


def _torus(X: np.ndarray, R: float, r: float):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    rho = np.sqrt(x * x + y * y)
    a = rho - R
    q = np.sqrt(a * a + z * z)
    d = q - r
    dist2 = d * d
    # the axis (rho = 0) and the centre circle (q = 0) have no closest point (nan)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = r / q
        m = R + a * s
        k = m / rho
        cp = np.stack([x * k, y * k, z * s], axis=1)
    return cp, dist2


def _ellipsoid_t(X: np.ndarray, axes: np.ndarray, iters: int = 1100) -> np.ndarray:
    """Root t of F(t) = sum a_i^2 x_i^2/(a_i^2+t)^2 - 1 by bisection.

    F is strictly decreasing on (-min a_i^2, inf).  Bracket: lower end just
    above -min a_i^2 (F -> +inf there unless the matching x_i vanish), upper
    end max a_i |x| (F < 0 there).  Bisection runs until the bracket stops
    shrinking in float64.
    """
    a2 = axes * axes
    amin2 = a2.min()
    ax = np.abs(X) * axes[None, :]
    lo = np.full(X.shape[0], -amin2)
    hi = np.sqrt((ax[:, 0] * ax[:, 0] + ax[:, 1] * ax[:, 1]) + ax[:, 2] * ax[:, 2]) + 1e-300
    moved = np.zeros(X.shape[0], dtype=bool)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if np.all((mid == lo) | (mid == hi)):
            break
        # a collapsed bracket at -min a_i^2 with x_i = 0 gives 0/0 = nan there:
        # F > 0 is then false, so the node stays marked as never moved
        with np.errstate(divide="ignore", invalid="ignore"):
            g0 = ax[:, 0] / (a2[0] + mid)
            g1 = ax[:, 1] / (a2[1] + mid)
            g2 = ax[:, 2] / (a2[2] + mid)
            F = ((g0 * g0 + g1 * g1) + g2 * g2) - 1.0
        pos = F > 0
        moved |= pos
        lo = np.where(pos, mid, lo)
        hi = np.where(pos, hi, mid)
    t = 0.5 * (lo + hi)
    # F never positive: the root lies at or below -min a_i^2, x sits on the
    # medial disk and the stationary point found is not the nearest point
    # (such x are at least the reach away from S).
    return np.where(moved, t, np.nan)


def _ellipsoid(X: np.ndarray, axes):
    axes = np.asarray(axes, dtype=np.float64)
    t = _ellipsoid_t(X, axes)
    a2 = axes * axes
    cp = (a2[None, :] * X) / (a2[None, :] + t[:, None])
    diff = X - cp
    dist2 = (diff[:, 0] * diff[:, 0] + diff[:, 1] * diff[:, 1]) + diff[:, 2] * diff[:, 2]
    dist2 = np.where(np.isnan(t), np.inf, dist2)
    return cp, dist2


DZIUK_NEWTON_STEPS = 30


def _dziuk(X: np.ndarray):
    """Closest point on phi(y) = (y1 - y3^2)^2 + y2^2 + y3^2 - 1 = 0 by Newton's
    method on the Lagrange conditions (Sec. 4.5.5 minimises the squared
    distance with Newton's method):

        y - x + lam g(y) = 0,  phi(y) = 0,   g = grad(phi) / 2
                                              = (a, y2, y3 (1 - 2a)),  a = y1 - y3^2.

    Start y = x, lam = 0 (the first step is the gradient projection of x);
    each step solves [K, g; 2 g^T, 0] [dy; dl] = -[F1; F2] with
    K = I + lam dg/dy, whose only off-diagonal entry is K13 = K31 = -2 lam y3:
    dl = (F2 - 2 g.K^-1 F1) / (2 g.K^-1 g), dy = -K^-1 (F1 + g dl), K^-1 by
    the 2x2 block (y1, y3) and the scalar y2 block.  A fixed number of steps,
    every operation rounded separately in this order (the CUDA path repeats
    it bit for bit).  Nodes where a step is singular get nan (not in any band).
    """
    x1, x2, x3 = X[:, 0].copy(), X[:, 1].copy(), X[:, 2].copy()
    y1, y2, y3 = x1.copy(), x2.copy(), x3.copy()
    lam = np.zeros_like(x1)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        for _ in range(DZIUK_NEWTON_STEPS):
            y3s = y3 * y3
            a = y1 - y3s
            g1 = a
            g2 = y2
            g3 = y3 * (1.0 - 2.0 * a)
            F11 = (y1 - x1) + lam * g1
            F12 = (y2 - x2) + lam * g2
            F13 = (y3 - x3) + lam * g3
            F2 = ((a * a + y2 * y2) + y3s) - 1.0
            k11 = 1.0 + lam
            k22 = 1.0 + lam
            k13 = -2.0 * (lam * y3)
            k33 = 1.0 + lam * ((1.0 - 2.0 * y1) + 6.0 * y3s)
            det = k11 * k33 - k13 * k13
            # K^-1 F1 and K^-1 g
            p1 = (k33 * F11 - k13 * F13) / det
            p2 = F12 / k22
            p3 = (k11 * F13 - k13 * F11) / det
            q1 = (k33 * g1 - k13 * g3) / det
            q2 = g2 / k22
            q3 = (k11 * g3 - k13 * g1) / det
            gp = (g1 * p1 + g2 * p2) + g3 * p3
            gq = (g1 * q1 + g2 * q2) + g3 * q3
            dl = (F2 - 2.0 * gp) / (2.0 * gq)
            y1 = y1 - (p1 + q1 * dl)
            y2 = y2 - (p2 + q2 * dl)
            y3 = y3 - (p3 + q3 * dl)
            lam = lam + dl
        d1, d2, d3 = x1 - y1, x2 - y2, x3 - y3
        dist2 = (d1 * d1 + d2 * d2) + d3 * d3
    cp = np.stack([y1, y2, y3], axis=1)
    bad = ~np.isfinite(dist2)
    dist2[bad] = np.inf
    cp[bad] = np.nan
    return cp, dist2


def dziuk_min_curvature_radius(n: int = 400) -> float:
    """1 / max |kappa| over the Dziuk surface, from the shape operator
    (I - n n^T) Hess(phi) (I - n n^T) / |grad phi| at points of the surface
    x1 = x3^2 + rho cos(t), x2 = rho sin(t), rho = sqrt(1 - x3^2)."""
    z = np.linspace(-1.0, 1.0, n)[1:-1]
    t = np.linspace(0.0, 2 * np.pi, 2 * n, endpoint=False)
    Z, T = np.meshgrid(z, t, indexing="ij")
    rho = np.sqrt(1.0 - Z * Z)
    P = np.stack([Z * Z + rho * np.cos(T), rho * np.sin(T), Z], axis=-1).reshape(-1, 3)
    a = P[:, 0] - P[:, 2] ** 2
    G = 2.0 * np.stack([a, P[:, 1], P[:, 2] * (1.0 - 2.0 * a)], axis=1)
    H = np.zeros((len(P), 3, 3))
    H[:, 0, 0] = 2.0
    H[:, 1, 1] = 2.0
    H[:, 0, 2] = H[:, 2, 0] = -4.0 * P[:, 2]
    H[:, 2, 2] = 2.0 - 4.0 * a + 8.0 * P[:, 2] ** 2
    g = np.linalg.norm(G, axis=1)
    nrm = G / g[:, None]
    Pr = np.eye(3)[None] - nrm[:, :, None] * nrm[:, None, :]
    S = Pr @ H @ Pr / g[:, None, None]
    kmax = np.abs(np.linalg.eigvalsh(S)).max()
    return float(1.0 / kmax)


def closest_point(surface: Surface, X: np.ndarray):
    """(cp, dist2) of the grid nodes X, shape (N, d), float64."""
    X = np.asarray(X, dtype=np.float64)
    if surface.kind in (CIRCLE, SPHERE):
        return _round_sphere(X, surface.params[0])
    if surface.kind == TORUS:
        return _torus(X, *surface.params)
    if surface.kind == ELLIPSOID:
        return _ellipsoid(X, surface.params)
    if surface.kind == DZIUK:
        return _dziuk(X)
    raise ValueError(surface.kind)
