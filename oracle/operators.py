"""Discrete operators of the embedding equation (Sec. 3.1-3.2, Sec. 4.2).

TEST INFRASTRUCTURE ONLY (see the package header).

Notation (d = dimension, gamma = 2d/dx^2, Sec. 3.1):

* L        the 2d+1-point Laplacian (1/dx^2){-2d, 1, .., 1}.  Two versions:
           ``lap_plus``  rows B, columns B+ (all neighbours kept, via the
                         ghost ring);
           ``lap_band``  rows B, columns B, neighbours outside B dropped
                         (the band-restricted L of Sec. 3.1 / Table 4.1).
* E        cubic closest-point extension, rows B+, columns B.
* M        the operator of the Macdonald-Brandman-Ruuth embedding (Eq. 2.10),
           discretised to second order with cubic E in both terms
           (Remark 3.2):
               M = diag(L) + (L - diag L) E  =  L E - gamma (I - E),
           with L = ``lap_plus`` (so diag L = -gamma on every row).
* A        = diag(c) - M  (c a positive constant or a per-point surface
           function c(cp(x)), footnote of Sec. 2.1).
* M_paper  = E_1 L - gamma (I - E_3)  (Eq. 3.3, p = 1, q = 3, L = lap_band):
           the paper's own scheme, used for Theorem 3.3 and Table 3.1.
* A_tilde  = cI - L  (L = lap_band): the shifted Cartesian Laplacian of the
           Ruuth-Merriman smoother (Sec. 4.2).

``apply_M`` evaluates M u in the difference form
    (M u)_i = sum_{k in N(i)} (w_k - w_i)/dx^2 + gamma (w_i - u_i),  w = E u,
which is the same linear map as the assembled matrix but cancels the large
gamma-sized terms before rounding (the assembled product loses about
eps * gamma * |u|).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .band import Band
from .interp import extension_matrix, interp_matrix


def gamma(band: Band) -> float:
    return 2.0 * band.dim / (band.dx * band.dx)


def neighbours_plus(band: Band) -> np.ndarray:
    """(|B|, 2d) indices into B+ of the Laplacian neighbours of B."""
    nbk = band.neighbour_keys(band.keys)
    idx = band.index_in_bplus(nbk.ravel()).reshape(nbk.shape)
    if np.any(idx < 0):
        raise ValueError("a Laplacian neighbour is outside B+")
    return idx


def lap_plus(band: Band) -> sp.csr_matrix:
    nb, d = band.nb, band.dim
    h2 = band.dx * band.dx
    nbr = neighbours_plus(band)
    rows = np.concatenate([np.arange(nb), np.repeat(np.arange(nb), 2 * d)])
    cols = np.concatenate([np.arange(nb), nbr.ravel()])
    vals = np.concatenate([np.full(nb, -2.0 * d / h2), np.full(nb * 2 * d, 1.0 / h2)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nb, nb + band.ng))


def lap_band(band: Band) -> sp.csr_matrix:
    nb, d = band.nb, band.dim
    h2 = band.dx * band.dx
    nbk = band.neighbour_keys(band.keys)
    idx = band.index_in_band(nbk.ravel()).reshape(nbk.shape)
    r, c = np.nonzero(idx >= 0)
    rows = np.concatenate([np.arange(nb), r])
    cols = np.concatenate([np.arange(nb), idx[r, c]])
    vals = np.concatenate([np.full(nb, -2.0 * d / h2), np.full(r.size, 1.0 / h2)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nb, nb))


class Operators:
    """Assembled E, L and M of one level, plus matrix-free applications."""

    def __init__(self, band: Band, p: int = 3):
        self.band = band
        self.p = p
        self.nb = band.nb
        self.gamma = gamma(band)
        self.h2 = band.dx * band.dx
        self.E = extension_matrix(band, p)          # (|B+|, |B|)
        self.nbr = neighbours_plus(band)            # (|B|, 2d)
        self.Lp = lap_plus(band)                    # (|B|, |B+|)
        self.Lb = lap_band(band)                    # (|B|, |B|)
        self._M = None

    # --- M in the form diag(L) + (L - diag L) E -----------------------------
    @property
    def M(self) -> sp.csr_matrix:
        if self._M is None:
            nb = self.nb
            off = self.Lp - sp.csr_matrix(
                (np.full(nb, -self.gamma), (np.arange(nb), np.arange(nb))),
                shape=self.Lp.shape)
            self._M = (off @ self.E - self.gamma * sp.identity(nb, format="csr")).tocsr()
        return self._M

    def extend(self, u: np.ndarray) -> np.ndarray:
        """w = E u on B+."""
        return self.E @ u

    def apply_M(self, u: np.ndarray) -> np.ndarray:
        """M u in the difference form (see the module header)."""
        w = self.E @ u
        wb = w[: self.nb]
        lap = (w[self.nbr] - wb[:, None]).sum(axis=1) / self.h2
        return lap + self.gamma * (wb - u)

    def apply_A(self, u: np.ndarray, c) -> np.ndarray:
        return c * u - self.apply_M(u)

    def residual(self, u: np.ndarray, f: np.ndarray, c) -> np.ndarray:
        """r = f - A u."""
        return f - self.apply_A(u, c)

    def diag_M(self) -> np.ndarray:
        """M_ii = -gamma + (1/dx^2) sum_{k in N(i)} E_{k,i}."""
        nb, ncol = self.nb, self.E.shape[0]
        rows = np.repeat(np.arange(nb), self.nbr.shape[1])
        N = sp.csr_matrix((np.ones(rows.size), (rows, self.nbr.ravel())), shape=(nb, ncol))
        s = np.asarray(N.multiply(self.E.T.tocsr()).sum(axis=1)).ravel()
        return -self.gamma + s / self.h2

    def A_matrix(self, c) -> sp.csr_matrix:
        cvec = np.broadcast_to(np.asarray(c, dtype=np.float64), (self.nb,))
        return (sp.diags(cvec) - self.M).tocsr()

    # --- Ruuth-Merriman pieces (Sec. 4.2) ----------------------------------
    def apply_Atilde(self, u: np.ndarray, c) -> np.ndarray:
        """(cI - L) u with the band-restricted L."""
        return c * u - self.Lb @ u

    def diag_Atilde(self, c) -> np.ndarray:
        return np.broadcast_to(np.asarray(c, dtype=np.float64) + self.gamma, (self.nb,)).copy()


def paper_M(band: Band) -> sp.csr_matrix:
    """M = E_1 L - gamma (I - E_3), Eq. 3.3 with L band-restricted (Sec. 3.1)."""
    nb = band.nb
    cpB = band.cp[:nb]
    E1 = interp_matrix(band, cpB, 1)
    E3 = interp_matrix(band, cpB, 3)
    L = lap_band(band)
    g = gamma(band)
    return (E1 @ L - g * (sp.identity(nb, format="csr") - E3)).tocsr()


class PaperOperators(Operators):
    """The paper's scheme (Eq. 3.3) behind the interface of ``Operators``:
    M = E_1 L_band - gamma (I - E_3) on B, assembled by ``paper_M`` and applied
    as a sparse product.  E (cubic, rows B+) is kept for the re-extended
    residual of Sec. 4.4; everything else follows from M."""

    def __init__(self, band: Band, p: int = 3):
        super().__init__(band, p)
        self._M = paper_M(band)

    @property
    def M(self) -> sp.csr_matrix:
        return self._M

    def apply_M(self, u: np.ndarray) -> np.ndarray:
        return self._M @ u

    def diag_M(self) -> np.ndarray:
        return self._M.diagonal().copy()


def lap_vardiff(band: Band, a: np.ndarray) -> sp.csr_matrix:
    """L~ = sum over axes of D^b diag(A^f a) D^f (Sec. 4.5.6) restricted to B:
    for a band node i and each neighbour k = i +- e_axis in B, the face
    coefficient (a_i + a_k) / 2 multiplies (u_k - u_i) / dx^2; neighbours
    outside B are dropped, as in the band-restricted L."""
    nb = band.nb
    h2 = band.dx * band.dx
    nbk = band.neighbour_keys(band.keys)
    idx = band.index_in_band(nbk.ravel()).reshape(nbk.shape)
    r, q = np.nonzero(idx >= 0)
    k = idx[r, q]
    face = 0.5 * (a[r] + a[k]) / h2
    rows = np.concatenate([r, r])
    cols = np.concatenate([k, r])
    vals = np.concatenate([face, -face])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nb, nb))


class VarDiffOperators(Operators):
    """Variable diffusion (Sec. 4.5.6): M = E_1 L~ - diag(gamma a) (I - E_3) on B
    with L~ from ``lap_vardiff`` and a the diffusion coefficient at the closest
    points of B.  The section writes one E for both terms and one gamma; as in
    Eq. 3.3 the differential term takes linear (E_1) and the side condition
    cubic (E_3) interpolation, and the side condition of node i is weighted by
    gamma a_i, gamma = 2d/dx^2, so that it balances the local diffusion as
    gamma balances a unit coefficient (with E_3 in both terms, or one gamma,
    Jacobi-smoothed V-cycles diverge on the sphere at dx = 1/32).  With a = 1
    this is the paper-form M of Eq. 3.3 exactly."""

    def __init__(self, band: Band, a: np.ndarray, p: int = 3):
        super().__init__(band, p)
        nb = band.nb
        self.a = np.asarray(a, dtype=np.float64)
        E1 = interp_matrix(band, band.cp[:nb], 1)
        E3 = interp_matrix(band, band.cp[:nb], p)
        self.Lt = lap_vardiff(band, self.a)
        G = sp.diags(self.gamma * self.a)
        self._M = (E1 @ self.Lt - G @ (sp.identity(nb, format="csr") - E3)).tocsr()

    @property
    def M(self) -> sp.csr_matrix:
        return self._M

    def apply_M(self, u: np.ndarray) -> np.ndarray:
        return self._M @ u

    def diag_M(self) -> np.ndarray:
        return self._M.diagonal().copy()

