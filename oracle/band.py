"""Computational band on a uniform Cartesian grid (Sec. 3.1, Table 4.1).

TEST INFRASTRUCTURE ONLY (see the package header).

Grid.  Nodes x = lo + i*dx, i = 0..n-1 on every axis, with lo = -2 and
n = 4/dx + 1, so that the origin is a node (the convention under which the
band sizes and nnz counts of Table 4.1 come out exactly).  A node's key is
its lexicographic index  i0 + n*(i1 + n*i2)  (x fastest); the oracle keeps
every set sorted by key.

Band.  Sec. 3.1 asks for a set B containing B_interp (every node of an
interpolation stencil of some surface point) and B_edge (their difference-
stencil neighbours).  The tube  B = {x : |x - cp(x)|^2 <= lambda^2 dx^2}
with lambda^2 = (d-1)(p+1)^2/4 + (1+(p+1)/2)^2 (17 for the sphere with cubic
interpolation) reproduces every integer of Table 4.1, so the oracle uses that
tube.  The threshold is evaluated as  lambda2 * (dx*dx).

Ghost ring.  The Macdonald-Brandman-Ruuth form of M (Eq. 2.10 / Remark 3.2)
applies the Laplacian to E u, so Laplacian neighbours of band nodes that lie
outside B need (E u) too: the ghost ring G = N(B) minus B, B+ = B with G.
Unknowns live on B only.

Stencils.  For degree-p interpolation at y = cp(x) the stencil along each axis
is the p+1 nodes  floor((y-lo)/dx) - (p-1)/2 + j, j = 0..p  (p odd), and the
fractional position is  s = (y-lo)/dx - floor((y-lo)/dx)  in [0, 1).  The
division is the IEEE one (no reciprocal multiply).  Every stencil node of
every point of B+ must lie in B (checked).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .geometry import DZIUK, ELLIPSOID, Surface, closest_point


def default_lambda2(dim: int, p: int = 3) -> float:
    """lambda^2 = (d-1)(p+1)^2/4 + (1+(p+1)/2)^2: 13 for d=2, 17 for d=3 (p=3)."""
    return (dim - 1) * (p + 1) ** 2 / 4.0 + (1.0 + (p + 1) / 2.0) ** 2


def grid_size(dx: float, lo: float = -2.0, hi: float = 2.0) -> int:
    return int(round((hi - lo) / dx)) + 1


@dataclass
class Band:
    """Band B, ghost ring G and their closest points, sorted by grid key."""

    surface: Surface
    dx: float
    lo: float
    n: int
    lambda2: float
    keys: np.ndarray        # int64 keys of B (sorted)
    ghost_keys: np.ndarray  # int64 keys of G (sorted)
    cp: np.ndarray          # (|B|+|G|, d) closest points, B rows then G rows
    dist2: np.ndarray       # (|B|+|G|,) squared distances

    @property
    def dim(self) -> int:
        return self.surface.dim

    @property
    def nb(self) -> int:
        return int(self.keys.size)

    @property
    def ng(self) -> int:
        return int(self.ghost_keys.size)

    @property
    def all_keys(self) -> np.ndarray:
        return np.concatenate([self.keys, self.ghost_keys])

    def coords_of(self, keys: np.ndarray) -> np.ndarray:
        """Integer grid coordinates (N, d) of keys."""
        n = self.n
        out = [keys % n]
        rest = keys // n
        for _ in range(self.dim - 1):
            out.append(rest % n)
            rest = rest // n
        return np.stack(out, axis=1)

    def key_of(self, ijk: np.ndarray) -> np.ndarray:
        n = self.n
        key = ijk[:, -1].astype(np.int64)
        for a in range(self.dim - 2, -1, -1):
            key = key * n + ijk[:, a]
        return key

    def points(self, keys: np.ndarray) -> np.ndarray:
        return self.lo + self.coords_of(keys).astype(np.float64) * self.dx

    def index_in_band(self, keys: np.ndarray) -> np.ndarray:
        """Index into B of each key, -1 if the key is not in B."""
        pos = np.searchsorted(self.keys, keys)
        pos = np.minimum(pos, self.nb - 1)
        ok = self.keys[pos] == keys
        return np.where(ok, pos, -1)

    def index_in_bplus(self, keys: np.ndarray) -> np.ndarray:
        """Index into B+ (B rows then G rows) of each key, -1 if absent."""
        ib = self.index_in_band(keys)
        pos = np.searchsorted(self.ghost_keys, keys)
        pos = np.minimum(pos, max(self.ng - 1, 0))
        if self.ng:
            ok = self.ghost_keys[pos] == keys
            ig = np.where(ok, self.nb + pos, -1)
        else:
            ig = np.full(keys.shape, -1)
        return np.where(ib >= 0, ib, ig)

    def neighbour_keys(self, keys: np.ndarray) -> np.ndarray:
        """(N, 2d) keys of the 2d Laplacian neighbours, order -x,+x,-y,+y(,-z,+z)."""
        ijk = self.coords_of(keys)
        cols = []
        for a in range(self.dim):
            for sgn in (-1, 1):
                nb = ijk.copy()
                nb[:, a] += sgn
                cols.append(self.key_of(nb))
        return np.stack(cols, axis=1)


def stencil(cp: np.ndarray, lo: float, dx: float, p: int):
    """Stencil base node (N, d) int64 and fractions s (N, d) in [0, 1)."""
    t = (cp - lo) / dx
    fl = np.floor(t)
    s = t - fl
    base = fl.astype(np.int64) - (p - 1) // 2
    return base, s


def _candidate_filter(surface: Surface, X: np.ndarray, reach: float) -> np.ndarray:
    """Cheap superset filter: nodes that may lie within `reach` of S."""
    if surface.kind == ELLIPSOID:
        a = np.asarray(surface.params)
        rho = np.sqrt(((X / a[None, :]) ** 2).sum(axis=1))
        return a.min() * np.abs(rho - 1.0) <= reach
    if surface.kind == DZIUK:
        # first-order distance |phi| / |grad phi|, with a factor 4 of slack for
        # the curvature (at most about 10.4) over the band half-widths used
        x1, x2, x3 = X[:, 0], X[:, 1], X[:, 2]
        a = x1 - x3 * x3
        phi = a * a + x2 * x2 + x3 * x3 - 1.0
        g = 2.0 * np.sqrt(a * a + x2 * x2 + (x3 * (1.0 - 2.0 * a)) ** 2)
        with np.errstate(divide="ignore", invalid="ignore"):
            est = np.abs(phi) / g
        return ~(est > 4.0 * reach)
    return np.ones(X.shape[0], dtype=bool)


def build_band(surface: Surface, dx: float, lo: float = -2.0, hi: float = 2.0,
               lambda2: float | None = None, p: int = 3, ghost: bool = True) -> Band:
    """Build B = {x : dist2(x) <= lambda2*(dx*dx)} and (optionally) the ghost ring.

    ``ghost=False`` skips the ghost ring; Table 4.1 counts need only B (its
    coarsest rows, dx = 0.2, are too wide for a ghost ring around the unit
    sphere: the ring would reach the centre, where cp is undefined).
    """
    d = surface.dim
    if lambda2 is None:
        lambda2 = default_lambda2(d, p)
    if not dx > 0:
        raise ValueError("dx must be positive")
    n = grid_size(dx, lo, hi)
    thr = lambda2 * (dx * dx)
    coord = lo + np.arange(n, dtype=np.float64) * dx
    margin = np.sqrt(thr) * 1.01 + 2 * dx
    keys_l, cp_l, d2_l = [], [], []
    if d == 2:
        Y, Xg = np.meshgrid(coord, coord, indexing="ij")
        X = np.stack([Xg.ravel(), Y.ravel()], axis=1)
        cand = _candidate_filter(surface, X, margin)
        idx = np.nonzero(cand)[0]
        cp, d2 = closest_point(surface, X[idx])
        sel = d2 <= thr
        keys_l.append(idx[sel].astype(np.int64))
        cp_l.append(cp[sel])
        d2_l.append(d2[sel])
    else:
        Y, Xg = np.meshgrid(coord, coord, indexing="ij")
        xy = np.stack([Xg.ravel(), Y.ravel()], axis=1)
        for k in range(n):
            X = np.empty((n * n, 3))
            X[:, :2] = xy
            X[:, 2] = coord[k]
            cand = _candidate_filter(surface, X, margin)
            idx = np.nonzero(cand)[0]
            if idx.size == 0:
                continue
            cp, d2 = closest_point(surface, X[idx])
            sel = d2 <= thr
            if np.any(sel):
                keys_l.append(idx[sel].astype(np.int64) + np.int64(k) * n * n)
                cp_l.append(cp[sel])
                d2_l.append(d2[sel])
    keys = np.concatenate(keys_l) if keys_l else np.zeros(0, np.int64)
    cpB = np.concatenate(cp_l) if cp_l else np.zeros((0, d))
    d2B = np.concatenate(d2_l) if d2_l else np.zeros(0)
    order = np.argsort(keys, kind="stable")
    keys, cpB, d2B = keys[order], cpB[order], d2B[order]

    band = Band(surface, float(dx), float(lo), n, float(lambda2), keys,
                np.zeros(0, np.int64), cpB, d2B)
    ijk = band.coords_of(keys)
    if keys.size and (ijk.min() < 1 or ijk.max() > n - 2):
        raise ValueError("band touches the edge of the grid")
    if ghost:
        nbk = band.neighbour_keys(keys).ravel()
        gk = np.unique(nbk[band.index_in_band(nbk) < 0])
        cpG, d2G = closest_point(surface, band.points(gk))
        if not np.all(np.isfinite(cpG)):
            raise ValueError("the ghost ring reaches a point where cp is undefined")
        band.ghost_keys = gk
        band.cp = np.concatenate([cpB, cpG])
        band.dist2 = np.concatenate([d2B, d2G])
    check_stencils(band, p)
    return band


def check_stencils(band: Band, p: int) -> None:
    """Every degree-p stencil node of every point of B+ must lie in B."""
    base, _ = stencil(band.cp, band.lo, band.dx, p)
    for off in np.ndindex(*([p + 1] * band.dim)):
        node = base + np.asarray(off)[None, :]
        if np.any(band.index_in_band(band.key_of(node)) < 0):
            raise ValueError("an interpolation stencil leaves the band (reach violated)")


def table41_counts(band: Band, p: int = 3) -> dict:
    """|B|, nnz(L), nnz(E_p), nnz(M) as counted in Table 4.1.

    L is the 2d+1-point Laplacian restricted to B (out-of-band neighbours
    dropped, the convention that leaves E_1 L unchanged, Sec. 3.1).  E_p has
    (p+1)^d structural entries per row.  M = E_1 L - gamma (I - E_3) has the
    union of the patterns of E_1 L (inside the cubic stencil) and E_3, plus
    the diagonal wherever the node is not in its own cubic stencil.
    """
    nb = band.nb
    nbk = band.neighbour_keys(band.keys)
    nnzL = nb + int((band.index_in_band(nbk.ravel()) >= 0).sum())
    nnzE = nb * (p + 1) ** band.dim
    base, _ = stencil(band.cp[:nb], band.lo, band.dx, p)
    own = band.coords_of(band.keys)
    inside = np.all((own >= base) & (own <= base + p), axis=1)
    nnzM = nnzE + int((~inside).sum())
    return {"dofs": nb, "nnzL": nnzL, "nnzE": nnzE, "nnzM": nnzM}
