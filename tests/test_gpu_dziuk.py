"""A level-set surface on the GPU (Sec. 4.5.5): the Dziuk surface
(x1 - x3^2)^2 + x2^2 + x3^2 = 1 with closest points by Newton's method.

* the band, ghost ring and closest points built by the CUDA library equal the
  oracle's bit for bit (same Newton steps, rounded in the same order);
* cpm_apply equals the oracle's M u;
* a GPU solve of -Lap_S u + u = f with u = x1 x2 (f in closed form) at
  dx = 1/128 approaches u to the discretisation error.
"""
import numpy as np
import pytest

from helpers import gpu_keys, perm_gpu_to_oracle, require_cuda
from oracle.band import build_band
from oracle.geometry import dziuk
from oracle.operators import Operators
import synth

pytestmark = pytest.mark.gpu


def test_dziuk_band_bit_exact():
    torch, pkg = require_cuda()
    dx = 1 / 64
    g = pkg.Band("dziuk", (), dx)
    ob = build_band(dziuk(), dx)
    assert (g.nb, g.ng) == (ob.nb, ob.ng)
    ijk, cp, base = g.export()
    keys = gpu_keys(ijk, ob.n)
    assert np.array_equal(np.sort(keys[: g.nb]), ob.keys)
    assert np.array_equal(np.sort(keys[g.nb:]), ob.ghost_keys)
    idx = ob.index_in_bplus(keys)
    assert np.array_equal(cp, ob.cp[idx])  # bit-identical Newton closest points


def test_dziuk_apply_parity():
    torch, pkg = require_cuda()
    dx = 1 / 64
    g = pkg.Band("dziuk", (), dx)
    H = pkg.Hierarchy(g, coarsest_dx=dx, coarse_sweeps=1)
    ob = build_band(dziuk(), dx)
    perm = perm_gpu_to_oracle(g, ob)
    u_o = synth.random_band_vector(ob.nb, 71)
    ref = Operators(ob).apply_M(u_o)[perm]
    got = H.apply(torch.from_numpy(u_o[perm]).cuda()).cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-13


def test_dziuk_solve_converges_to_the_closed_form():
    """dx = 1/128 with V-cycles down to dx = 1/64, the coarsest spacing the reach
    0.0957 allows; that level (about 460 k points, too large for a dense solve)
    is solved by restarted GMRES(30) on the device.  The residual falls to
    1e-8 and the solution approaches u = x1 x2 to the discretisation error at
    this spacing."""
    torch, pkg = require_cuda()
    dx = 1 / 128
    g = pkg.Band("dziuk", (), dx)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 64, residual="plain", coarse_gmres=4)
    assert H.n_levels == 2
    _, cp, _ = g.export()
    uex, f = synth.dziuk_rhs(cp[: g.nb])
    u, rep = H.solve(torch.from_numpy(f).cuda(), tol=1e-8, max_iter=60, mode="mixed",
                     inner_cycles=2)
    assert rep["converged"], rep["history"]
    err = np.abs(u.cpu().numpy() - uex).max() / np.abs(uex).max()
    assert err < 3e-4, err
