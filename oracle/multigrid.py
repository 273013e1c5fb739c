"""Closest Point Method V-cycle (Sec. 4, Algorithm 4.1) and the outer loop.

TEST INFRASTRUCTURE ONLY (see the package header).

Levels.  Level 0 is the finest grid (dx), level l has spacing dx * 2^l and a
band of its own built with the same lambda (Sec. 4.3: "bandwidths shrinking
proportional to the grid sizes"); the coarsest level K is solved directly.
The grids are nested because every spacing divides 2 (lo = -2).

Transfers (Sec. 4.3).  Restriction E_h^{2h}: each coarse band point takes the
value at its closest point, interpolated (degree ``transfer_p``, linear by
default as in Sec. 4.5) from the fine band.  Prolongation E_{2h}^h: each fine
band point takes the value at its closest point interpolated from the coarse
band.  No full-weighting factor.  Coarse operators are rediscretised:
A^{2h} = c I - M^{2h}.

Smoothers.
* ``rm``       Ruuth-Merriman Jacobi (Eq. 4.2): u += omega diag(At)^-1 (f - At u)
               with At = cI - L (band-restricted L), then u := E u.  The residual
               restricted in step 2 of Algorithm 4.1 is f - At u.
* ``jacobi``   standard Jacobi on A (Eq. 4.1): u += omega diag(A)^-1 (f - A u);
               the residual restricted in step 2 is f - A (E u) (Sec. 4.4,
               ``residual="extended"``) or f - A u (``residual="plain"``).
The paper uses omega = 1 with nu1 = nu2 = 3 (Sec. 4.5); the defaults here are
omega = 2/3 and nu1 = nu2 = 2.

V-cycle (Algorithm 4.1): nu1 smoothing steps, residual, restriction, either
the direct coarsest solve or a recursive V-cycle from zero, prolongation and
correction, nu2 smoothing steps.

Coarsest level.  Direct LU solve (Algorithm 4.1 step 2); when that level is
too large for a dense factorisation (``coarse_sweeps > 0``) a fixed number of
weighted Jacobi sweeps on A from zero stands in for it.

Outer loop.  Defect correction in float64:  r = f - A u  (A in the form of
``operators``), stop when ||r||_inf <= tol ||f||_inf, else u += V(0, r).
(The paper stops on the relative change of u, 1e-6; the relative residual is
the criterion used throughout this project.)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .band import Band, build_band
from .geometry import Surface
from .interp import interp_matrix
from .operators import Operators, PaperOperators, VarDiffOperators


@dataclass
class Level:
    band: Band
    ops: Operators
    c: np.ndarray                     # per-point c on this level
    R: object = None                  # restriction from this level to the next coarser
    P: object = None                  # prolongation from the next coarser to this level
    diagA: np.ndarray | None = None   # c - diag(M)


@dataclass
class MGOptions:
    nu1: int = 2
    nu2: int = 2
    omega: float = 2.0 / 3.0
    smoother: str = "rm"              # "rm" | "jacobi" | "rbgs" (red-black Gauss-Seidel on A)
    transfer_p: int = 1
    p: int = 3
    residual: str = "extended"        # "extended": f - A(E u) (Sec. 4.4); "plain": f - A u
    coarse_sweeps: int = 0            # > 0: coarsest level by Jacobi sweeps instead of LU
    coarse_gmres: int = 0             # > 0: coarsest level by that many restarts of GMRES(30)
    operator: str = "mbr"             # "mbr": diag(L) + (L - diag L) E (Eq. 2.10);
                                      # "paper": E_1 L_band - gamma (I - E_3) (Eq. 3.3)
    cycle: int = 1                    # coarse-grid corrections per level: 1 V-cycle, 2 W-cycle
    # operator "vardiff": E_3 L~ - gamma (I - E_3) with L~ the variable-diffusion
    # Laplacian of Sec. 4.5.6; a_fn(cp) gives the coefficient on the finest band


@dataclass
class Hierarchy:
    levels: list
    opts: MGOptions
    lu: tuple = field(default=None)

    @property
    def fine(self) -> Level:
        return self.levels[0]


def coarsest_spacing_ok(surface: Surface, dx: float, lambda2: float) -> bool:
    """Coarsening rule: (lambda + 1) dx < reach, so cp is unique on B+."""
    return (np.sqrt(lambda2) + 1.0) * dx < surface.reach


def build_hierarchy(surface: Surface, dx: float, coarsest_dx: float, c=1.0,
                    opts: MGOptions | None = None, c_fn=None, a_fn=None) -> Hierarchy:
    """Levels dx, 2dx, .., coarsest_dx.  ``c_fn(cp) -> c`` gives a variable c.

    A variable c is c_fn(cp(x)) on the finest band; coarser levels carry the
    restriction of the finer level's c (linear interpolation at their closest
    points), the reading that needs c only on the finest band.  The diffusion
    coefficient a of the "vardiff" operator (a_fn) is carried the same way.
    """
    opts = opts or MGOptions()
    levels = []
    h = dx
    while True:
        band = build_band(surface, h, p=opts.p)
        ops = (PaperOperators(band, opts.p) if opts.operator == "paper"
               else None if opts.operator == "vardiff" else Operators(band, opts.p))
        levels.append(Level(band, ops, np.full(band.nb, float(c))))
        if h >= coarsest_dx * (1 - 1e-12):
            break
        h *= 2.0
    for l in range(len(levels) - 1):
        fine, coarse = levels[l], levels[l + 1]
        fine.R = interp_matrix(fine.band, coarse.band.cp[: coarse.band.nb], opts.transfer_p)
        fine.P = interp_matrix(coarse.band, fine.band.cp[: fine.band.nb], opts.transfer_p)
    if opts.operator == "vardiff":
        a = np.asarray(a_fn(levels[0].band.cp[: levels[0].band.nb]), dtype=np.float64)
        for l, lev in enumerate(levels):
            if l > 0:
                a = levels[l - 1].R @ a
            lev.ops = VarDiffOperators(lev.band, a, opts.p)
    if c_fn is not None:
        # c is a surface function (footnote to Sec. 2.1) known on the finest band
        # as c(cp(x)); each coarser level takes it at its own closest points by
        # the restriction of Sec. 4.3 (interpolation at cp from the finer band).
        levels[0].c = np.asarray(c_fn(levels[0].band.cp[: levels[0].band.nb]), dtype=np.float64)
        for l in range(len(levels) - 1):
            levels[l + 1].c = levels[l].R @ levels[l].c
    for lev in levels:
        lev.diagA = lev.c - lev.ops.diag_M()
    hier = Hierarchy(levels, opts)
    last = levels[-1]
    if opts.coarse_sweeps == 0 and opts.coarse_gmres == 0:
        hier.lu = sla.lu_factor(last.ops.A_matrix(last.c).toarray())
    return hier


def colour(band) -> np.ndarray:
    """Red (0) / black (1) colour of the band nodes: parity of i + j (+ k)."""
    return band.coords_of(band.keys).sum(axis=1) % 2


def smooth(hier: Hierarchy, l: int, u: np.ndarray, f: np.ndarray) -> np.ndarray:
    lev, o = hier.levels[l], hier.opts
    if o.smoother == "rbgs":
        # Gauss-Seidel in red-black order (Sec. 4.4 names Gauss-Seidel as an
        # alternative to Jacobi): the red nodes take the weighted Jacobi update
        # of the current iterate, then the black nodes that of the updated one.
        col = colour(lev.band)
        for c in (0, 1):
            r = f - lev.ops.apply_A(u, lev.c)
            u = u + np.where(col == c, o.omega * r / lev.diagA, 0.0)
        return u
    if o.smoother == "rm":
        u = u + o.omega * (f - lev.ops.apply_Atilde(u, lev.c)) / lev.ops.diag_Atilde(lev.c)
        return lev.ops.extend(u)[: lev.ops.nb]
    if o.smoother == "jacobi":
        return u + o.omega * (f - lev.ops.apply_A(u, lev.c)) / lev.diagA
    raise ValueError(o.smoother)


def transfer_residual(hier: Hierarchy, l: int, u: np.ndarray, f: np.ndarray) -> np.ndarray:
    lev, o = hier.levels[l], hier.opts
    if o.smoother == "rm":
        return f - lev.ops.apply_Atilde(u, lev.c)
    if o.residual == "plain":
        return f - lev.ops.apply_A(u, lev.c)
    wb = lev.ops.extend(u)[: lev.ops.nb]
    return f - lev.ops.apply_A(wb, lev.c)


GMRES_M = 30


def gmres(A, b: np.ndarray, P: np.ndarray, m: int, restarts: int) -> np.ndarray:
    """Restarted GMRES(m) for A x = b from x = 0, right-preconditioned by
    diag(P): each cycle builds an orthonormal basis of the Krylov space of
    A diag(P) from r = b - A x (classical Gram-Schmidt applied twice), reduces
    the Hessenberg matrix with Givens rotations and adds diag(P) V y, y the
    least-squares minimiser of ||beta e_1 - H y|| (Saad and Schultz's
    algorithm; a fixed number of steps, no early exit)."""
    n = b.size
    x = np.zeros(n)
    for _ in range(restarts):
        r = b - A @ x
        beta = np.linalg.norm(r)
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        if beta == 0.0:
            break
        V[0] = r / beta
        g = np.zeros(m + 1)
        g[0] = beta
        cs, sn = np.zeros(m), np.zeros(m)
        for j in range(m):
            w = A @ (P * V[j])
            for _ in range(2):
                h = V[: j + 1] @ w
                w = w - V[: j + 1].T @ h
                H[: j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            V[j + 1] = w / H[j + 1, j] if H[j + 1, j] > 1e-300 else 0.0
            for i in range(j):
                a, bb = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * bb
                H[i + 1, j] = -sn[i] * a + cs[i] * bb
            a, bb = H[j, j], H[j + 1, j]
            rr = np.hypot(a, bb)
            cs[j], sn[j] = (a / rr, bb / rr) if rr > 0 else (1.0, 0.0)
            H[j, j], H[j + 1, j] = rr, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
        y = np.linalg.solve(np.triu(H[:m, :m]), g[:m])
        x = x + P * (V[:m].T @ y)
    return x


def coarse_solve(hier: Hierarchy, f: np.ndarray) -> np.ndarray:
    o = hier.opts
    if o.coarse_gmres > 0:
        last = hier.levels[-1]
        A = last.ops.A_matrix(last.c)
        return gmres(A, f, o.omega / last.diagA, GMRES_M, o.coarse_gmres)
    if o.coarse_sweeps > 0:
        last = hier.levels[-1]
        u = np.zeros_like(f)
        for _ in range(o.coarse_sweeps):
            u = u + o.omega * (f - last.ops.apply_A(u, last.c)) / last.diagA
        return u
    return sla.lu_solve(hier.lu, f)


def vcycle(hier: Hierarchy, u: np.ndarray, f: np.ndarray, l: int = 0) -> np.ndarray:
    """One V-cycle V^h(u, f) of Algorithm 4.1 on level l."""
    o = hier.opts
    if l == len(hier.levels) - 1:
        return coarse_solve(hier, f)
    for _ in range(o.nu1):
        u = smooth(hier, l, u, f)
    r = transfer_residual(hier, l, u, f)
    lev = hier.levels[l]
    fc = lev.R @ r
    if l + 1 == len(hier.levels) - 1:
        uc = coarse_solve(hier, fc)
    else:
        # V-cycle (cycle = 1) or W-cycle (cycle = 2): that many cycles of the
        # next level, the first from zero (remark at Algorithm 4.1)
        uc = np.zeros_like(fc)
        for _ in range(o.cycle):
            uc = vcycle(hier, uc, fc, l + 1)
    u = u + lev.P @ uc
    for _ in range(o.nu2):
        u = smooth(hier, l, u, f)
    return u


def fmg(hier: Hierarchy, f: np.ndarray) -> np.ndarray:
    """Full multigrid from zero: f restricted to every level, the coarsest
    level solved, then on each finer level the prolonged coarse solution is the
    start of one cycle of that level (remark at Algorithm 4.1)."""
    fs = [f]
    for l in range(len(hier.levels) - 1):
        fs.append(hier.levels[l].R @ fs[-1])
    u = coarse_solve(hier, fs[-1])
    for l in range(len(hier.levels) - 2, -1, -1):
        u = vcycle(hier, hier.levels[l].P @ u, fs[l], l)
    return u


@dataclass
class SolveReport:
    iters: int
    history: list
    converged: bool


def solve(hier: Hierarchy, f: np.ndarray, tol: float = 1e-10, max_iter: int = 100,
          u0: np.ndarray | None = None, first_fmg: bool = False) -> tuple[np.ndarray, SolveReport]:
    """Outer defect correction: u += V(0, f - A u) until ||r||/||f|| <= tol
    (first_fmg: the first correction is the full-multigrid solution of f - A u)."""
    fine = hier.fine
    u = np.zeros_like(f) if u0 is None else u0.copy()
    fn = np.abs(f).max()
    hist = []
    for it in range(max_iter + 1):
        r = fine.ops.residual(u, f, fine.c)
        rel = np.abs(r).max() / fn
        hist.append(rel)
        if rel <= tol:
            return u, SolveReport(it, hist, True)
        if it == max_iter:
            break
        u = u + (fmg(hier, r) if first_fmg and it == 0 else vcycle(hier, np.zeros_like(r), r))
    return u, SolveReport(max_iter, hist, False)
