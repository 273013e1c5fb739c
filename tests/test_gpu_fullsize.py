"""Parity at the benchmark size (unit sphere, dx = 1/256) on sampled outputs.

The oracle cannot assemble the 6.8M-point operator in a test's time budget, so
it evaluates the definition of M (Eq. 2.10 with cubic E, Remark 3.2) point by
point at sampled band points, with its own closest points, from the GPU's
vector values looked up by grid coordinates.
"""
import numpy as np
import pytest

from conftest import load_golden
from helpers import gpu_keys, require_cuda
from oracle.geometry import closest_point, sphere
from oracle.interp import lagrange_1d

pytestmark = pytest.mark.gpu

DX = 1.0 / 256


def _golden_size():
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "band_sizes.txt")
    for line in open(here):
        p = line.split()
        if p and not line.startswith("#") and p[0] == "sphere" and p[2] == "256":
            return int(p[3]), int(p[4])
    raise KeyError


def _Mu_at(i_keys, keys_sorted, order, u, ijk, n):
    """(M u)_i by the definition, for the band points with grid coordinates ijk[i]."""
    h2 = DX * DX
    out = []
    surf = sphere()
    for own in i_keys:
        acc = -6.0 / h2 * u[order[np.searchsorted(keys_sorted, gpu_keys(own[None, :], n))[0]]]
        for a in range(3):
            for sgn in (-1, 1):
                nb = own.copy()
                nb[a] += sgn
                X = -2.0 + nb.astype(np.float64) * DX
                cp, _ = closest_point(surf, X[None, :])
                t = (cp[0] + 2.0) / DX
                fl = np.floor(t)
                w = [lagrange_1d(np.array([t[ax] - fl[ax]]), 3)[0] for ax in range(3)]
                base = fl.astype(np.int64) - 1
                for c in range(4):
                    for b in range(4):
                        for aa in range(4):
                            node = base + np.array([aa, b, c])
                            k = gpu_keys(node[None, :], n)[0]
                            j = np.searchsorted(keys_sorted, k)
                            assert keys_sorted[j] == k
                            acc += w[0][aa] * w[1][b] * w[2][c] * u[order[j]] / h2
        out.append(acc)
    return np.asarray(out)


def test_fullsize_band_and_apply_sampled():
    torch, pkg = require_cuda()
    g = pkg.Band("sphere", (), DX)
    assert (g.nb, g.ng) == _golden_size()
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8)
    ijk, _, _ = g.export()
    n = int(round(4 / DX)) + 1
    keys = gpu_keys(ijk[: g.nb], n)
    order = np.argsort(keys)
    ks = keys[order]
    rng = np.random.default_rng(0)
    u = rng.uniform(-1, 1, g.nb)
    Mu = H.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    sample = rng.choice(g.nb, 60, replace=False)
    ref = _Mu_at(ijk[sample], ks, order, u, ijk, n)
    scale = np.abs(Mu).max()
    assert np.abs(Mu[sample] - ref).max() <= 1e-13 * scale


def test_fullsize_mixed_solve_residual_sampled():
    """Solve at full size; the oracle's pointwise residual at sampled points
    confirms the GPU's reported relative residual."""
    torch, pkg = require_cuda()
    import synth
    g = pkg.Band("sphere", (), DX)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8, residual="plain")
    ijk, cp, _ = g.export()
    _, f = synth.sphere_harmonics(cp[: g.nb])
    u, rep = H.solve(torch.from_numpy(f).cuda(), tol=1e-10, mode="mixed", inner_cycles=2)
    assert rep["converged"] and rep["rel_residual"] <= 1e-10
    u = u.cpu().numpy()
    n = int(round(4 / DX)) + 1
    keys = gpu_keys(ijk[: g.nb], n)
    order = np.argsort(keys)
    sample = np.random.default_rng(1).choice(g.nb, 40, replace=False)
    Mu = _Mu_at(ijk[sample], keys[order], order, u, ijk, n)
    r = f[sample] - 1.0 * u[sample] + Mu
    assert np.abs(r).max() <= 3e-10 * np.abs(f).max()
