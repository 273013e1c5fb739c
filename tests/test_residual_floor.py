"""Rounding floor of the FP64 residual in difference form, and the relative
form the GPU's outer residual uses (CPU, oracle operators).

Evaluated directly (w = E u, then (w_k - w_i)/dx^2 and gamma (w_i - u_i)), the
FP64 result carries errors of about eps |u| 2d/dx^2: the relative residual of a
solve cannot go below that.  In the relative form every point j has a
reference value ref_j = u at one node of its stencil, delta_j = sum_m E_jm
(u_m - ref_j) is formed from differences, and the stencil combines
(ref_k - ref_i) + (delta_k - delta_i) and (ref_i - u_i) + delta_i.  Both are
compared with the formula evaluated in extended precision with the FP64
weights of each row divided by their sum: the exact cubic weights sum to 1
(partition of unity), the rounded ones miss by ~eps, which alone shifts the
direct form by ~eps |u| 2d/dx^2; the relative form never multiplies |u| by a
weight, so it keeps the exact partition of unity.
"""
import numpy as np
import pytest

from oracle import geometry
from oracle.band import build_band
from oracle.operators import Operators


def _apply_M_extended(op, u):
    ld = np.longdouble
    E = op.E.tocsr()
    wsum = np.add.reduceat(E.data.astype(ld), E.indptr[:-1])
    w = np.add.reduceat(E.data.astype(ld) * u.astype(ld)[E.indices], E.indptr[:-1]) / wsum
    wb = w[: op.nb]
    lap = (w[op.nbr] - wb[:, None]).sum(axis=1) / ld(op.h2)
    return lap + ld(op.gamma) * (wb - u.astype(ld))


def _apply_M_relative(op, u):
    E = op.E.tocsr()
    ref = u[E.indices[E.indptr[:-1]]]          # u at the first node of each stencil
    rows = np.repeat(np.arange(E.shape[0]), np.diff(E.indptr))
    delta = np.add.reduceat(E.data * (u[E.indices] - ref[rows]), E.indptr[:-1])
    rb, db = ref[: op.nb], delta[: op.nb]
    lap = ((ref[op.nbr] - rb[:, None]) + (delta[op.nbr] - db[:, None])).sum(axis=1) / op.h2
    return lap + op.gamma * ((rb - u) + db)


def test_relative_form_lowers_the_residual_floor():
    if np.finfo(np.longdouble).eps >= np.finfo(np.float64).eps:
        pytest.skip("no extended precision on this platform")
    band = build_band(geometry.circle(1.0), 1 / 2048)
    op = Operators(band)
    th = np.arctan2(band.cp[: band.nb, 1], band.cp[: band.nb, 0])
    u = 2.0 + np.cos(3.0 * th)
    exact = _apply_M_extended(op, u)
    scale = float(np.abs(exact).max())
    err_direct = float(np.abs(op.apply_M(u) - exact).max()) / scale
    err_relative = float(np.abs(_apply_M_relative(op, u) - exact).max()) / scale
    # the direct form is at its floor (eps |u| 2d/dx^2 ~ 1e-8 absolute here) ...
    assert err_direct > 1e-11, err_direct
    # ... and the relative form of the same arithmetic is far below it
    assert err_relative < err_direct / 30, (err_relative, err_direct)
    assert err_relative < 1e-11, err_relative
