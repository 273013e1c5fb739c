"""Tensor-product barycentric Lagrange interpolation E_p (Sec. 3.1, Eq. 3.1-3.2).

TEST INFRASTRUCTURE ONLY (see the package header).

Along one axis the p+1 stencil nodes sit at positions -(p-1)/2 .. (p+1)/2
(in units of dx, relative to floor((y-lo)/dx)), and the target sits at the
fraction s in [0, 1).  The oracle evaluates the 1-D Lagrange basis with the
second-kind ("true") barycentric formula of Berrut & Trefethen, cited in
Sec. 3.1:

    l_j(s) = (b_j / (s - s_j)) / sum_k (b_k / (s - s_k)),
    b_j    = 1 / prod_{k != j} (s_j - s_k),

with l_j(s) = delta_{jk} when s equals the node s_k exactly.  For equispaced
nodes b_j is proportional to (-1)^j binom(p, j).  The d-dimensional weight
of stencil node (j_0, .., j_{d-1}) is the product of the 1-D weights
(dimension-by-dimension interpolation, Sec. 3.3, proof of Theorem 3.3).

E_p is assembled as a scipy CSR matrix whose row r holds the (p+1)^d weights
of target r at the band indices of its stencil nodes (explicit zeros kept:
the row pattern is the full stencil, as counted in Table 4.1).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .band import Band, stencil


def nodes_1d(p: int) -> np.ndarray:
    """Stencil node positions relative to floor(t): -(p-1)/2 .. (p+1)/2."""
    return np.arange(p + 1, dtype=np.float64) - (p - 1) // 2


def bary_weights_1d(p: int) -> np.ndarray:
    """b_j = 1 / prod_{k != j} (s_j - s_k)."""
    s = nodes_1d(p)
    b = np.empty(p + 1)
    for j in range(p + 1):
        b[j] = 1.0 / np.prod([s[j] - s[k] for k in range(p + 1) if k != j])
    return b


def lagrange_1d(s: np.ndarray, p: int) -> np.ndarray:
    """(N, p+1) 1-D Lagrange weights at fractions s (N,), second-kind formula."""
    s = np.asarray(s, dtype=np.float64)
    nodes = nodes_1d(p)
    b = bary_weights_1d(p)
    diff = s[:, None] - nodes[None, :]
    exact = diff == 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        terms = b[None, :] / diff
        w = terms / terms.sum(axis=1, keepdims=True)
    hit = exact.any(axis=1)
    w[hit] = exact[hit].astype(np.float64)
    return w


def tensor_weights(frac: np.ndarray, p: int) -> np.ndarray:
    """(N, (p+1)^d) tensor-product weights; node order: last axis slowest."""
    N, d = frac.shape
    w1 = [lagrange_1d(frac[:, a], p) for a in range(d)]
    out = np.ones((N, 1))
    for a in range(d - 1, -1, -1):
        # node order: axis 0 fastest, axis d-1 slowest
        out = (out[:, :, None] * w1[a][:, None, :]).reshape(N, -1)
    return out


def stencil_offsets(d: int, p: int) -> np.ndarray:
    """((p+1)^d, d) offsets, axis 0 fastest (matches tensor_weights)."""
    offs = [o[::-1] for o in itertools.product(range(p + 1), repeat=d)]
    return np.asarray(offs, dtype=np.int64)


def interp_matrix(src: Band, targets_cp: np.ndarray, p: int) -> sp.csr_matrix:
    """Matrix interpolating values on src's band B at the points targets_cp.

    Row r: weights of degree-p interpolation at targets_cp[r] from the
    stencil nodes (all in B of src, checked).
    """
    N, d = targets_cp.shape
    base, frac = stencil(targets_cp, src.lo, src.dx, p)
    W = tensor_weights(frac, p)
    offs = stencil_offsets(d, p)
    nodes = base[:, None, :] + offs[None, :, :]
    cols = src.index_in_band(src.key_of(nodes.reshape(-1, d)))
    if np.any(cols < 0):
        raise ValueError("interpolation stencil outside the source band")
    rows = np.repeat(np.arange(N), offs.shape[0])
    return sp.csr_matrix((W.ravel(), (rows, cols)), shape=(N, src.nb))


def extension_matrix(band: Band, p: int = 3) -> sp.csr_matrix:
    """E_p on B+ (rows: B then ghost ring) from B (columns)."""
    return interp_matrix(band, band.cp, p)
