"""The outer residual in FP32-pair arithmetic on the GPU (cpm_residual with
outer_f64 = 0, the default for the operator of Eq. 2.10) against the oracle's
residual f - (c - M) u and against the GPU's FP64 evaluation of the same
relative form, on small bands and at full size (unit sphere dx = 1/256 and
1/512) for converged solutions, where r is a small difference of large terms."""
import numpy as np
import pytest

from helpers import oracle_surface, perm_gpu_to_oracle, require_cuda
from oracle.band import build_band
from oracle.operators import Operators
import synth

pytestmark = pytest.mark.gpu

CASES = [("circle", (), 1 / 256), ("sphere", (), 1 / 64), ("torus", (1.0, 0.4), 1 / 32),
         ("ellipsoid", (1.0, 0.9, 0.7), 1 / 32)]


def _smooth(kind, cp):
    if kind == "circle":
        return synth.circle_fourier(cp)[0]
    if kind == "sphere":
        return synth.sphere_harmonics(cp)[0]
    return np.sin(2 * cp[:, 0]) * np.cos(3 * cp[:, 1]) + cp[:, 2] ** 2


def pair_floor(dx):
    """Bound on max |r_pair - r| / max |f| for smooth data: the pair floor grows
    like 1/dx (CPU pin: test_pair_residual_floor.py); measured about 2.7e-14 / dx
    on the circle and 1.4e-14 / dx on the sphere at dx = 1/256."""
    return 4e-14 / dx


@pytest.mark.parametrize("kind,params,dx", CASES)
def test_pair_residual_against_oracle_and_f64(kind, params, dx):
    """Random u: r is large, pairs and FP64 agree to ~1e-14 of max |r|.
    Smooth u with f = A u + 1e-9 noise: r is ~1e-9 of f, a difference of
    terms 1e9 times larger; the pair residual equals the oracle's and the FP64
    form's within the pair floor."""
    torch, pkg = require_cuda()
    g = pkg.Band(kind, params, dx)
    Hp = pkg.Hierarchy(g, coarsest_dx=dx)
    H64 = pkg.Hierarchy(g, coarsest_dx=dx, outer_f64=True)
    ob = build_band(oracle_surface(kind, params), dx)
    op = Operators(ob)
    perm = perm_gpu_to_oracle(g, ob)
    rng = np.random.default_rng(5)
    u_r = rng.uniform(-1, 1, ob.nb)
    f_r = rng.uniform(-1, 1, ob.nb)
    u_s = _smooth(kind, ob.cp[: ob.nb])
    f_s = op.apply_A(u_s, 1.0) + 1e-9 * rng.standard_normal(ob.nb)
    d = ob.dim
    for u_o, f_o, tol in ((u_r, f_r, 1e-13), (u_s, f_s, pair_floor(dx))):
        ref = op.residual(u_o, f_o, 1.0)[perm]
        u = torch.from_numpy(u_o[perm]).cuda()
        f = torch.from_numpy(f_o[perm]).cuda()
        rp = Hp.residual(f, u).cpu().numpy()
        r64 = H64.residual(f, u).cpu().numpy()
        scale = np.abs(f_o).max() if tol > 1e-13 else np.abs(ref).max()
        # the oracle evaluates the direct form (w = E u, then the stencil), whose
        # own rounding is about eps |u| 2d / dx^2 per term
        oracle_floor = 8 * np.finfo(float).eps * np.abs(u_o).max() * 2 * d / dx ** 2
        assert np.abs(rp - ref).max() <= tol * scale + oracle_floor, (np.abs(rp - ref).max() / scale)
        assert np.abs(rp - r64).max() <= tol * scale, (np.abs(rp - r64).max() / scale)
        inf_p, l2_p = Hp.residual_norms(f, u)
        inf_64, _ = H64.residual_norms(f, u)
        assert abs(inf_p - inf_64) <= 1e-3 * inf_64 + tol


@pytest.mark.parametrize("dx", [1 / 256, 1 / 512])
def test_pair_residual_fullsize_solve(dx):
    """Unit sphere at full size: the default (pair) outer residual drives the
    mixed solve to 1e-10 and the solve's FP64 check confirms it; the FP64 form
    evaluated separately agrees, and the two evaluations of r differ by at most
    the pair floor (about 5.5e-12 of max |f| at dx = 1/256, 1.1e-11 at 1/512)."""
    torch, pkg = require_cuda()
    g = pkg.Band("sphere", (), dx)
    Hp = pkg.Hierarchy(g, coarsest_dx=1 / 8, residual="plain", nu1=4, nu2=4)
    _, cp, _ = g.export()
    _, f_h = synth.sphere_harmonics(cp[: g.nb])
    f = torch.from_numpy(f_h).cuda()
    u, rep = Hp.solve(f, tol=1e-10, mode="mixed", inner_cycles=3)
    assert rep["converged"], rep
    Hp.close()
    H64 = pkg.Hierarchy(g, coarsest_dx=1 / 8, residual="plain", nu1=4, nu2=4, outer_f64=True)
    r64 = H64.residual(f, u)
    fmax = float(f.abs().max())
    rel64 = float(r64.abs().max()) / fmax  # the solve's test: max |r| / max |f|
    # the reported residual is the FP64 one after a check, else the pair one,
    # which is within the solve's estimate of the FP64 one
    assert rel64 <= 1e-10, (rel64, rep)
    assert abs(rel64 - rep["rel_residual"]) <= max(rep["pair_floor"], 1e-3 * rel64), (rel64, rep)
    H64.close()
    Hp = pkg.Hierarchy(g, coarsest_dx=1 / 8, residual="plain", nu1=4, nu2=4)
    rp = Hp.residual(f, u)
    diff = float((rp - r64).abs().max()) / fmax
    assert diff <= pair_floor(dx), diff
    # the solve's own estimate of the pair rounding error bounds it (and is not
    # vacuous), and at most one FP64 check was needed
    assert diff <= rep["pair_floor"] <= 100 * max(diff, 1e-13), (diff, rep["pair_floor"])
    assert rep["f64_checks"] <= 1, rep


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_tolerance_below_the_pair_floor(mode):
    """Circle dx = 1/64, tol = 1e-12: below the pair floor (about 1.3e-12 here)
    but above what FP64 reaches (the sparse direct solution's residual is about
    2e-12 in extended precision, the iteration gets below 1e-12).  The solve
    notices that the pair residual cannot decide, checks in FP64, finishes with
    FP64 residuals, and the result meets the tolerance in FP64."""
    torch, pkg = require_cuda()
    g = pkg.Band("circle", (), 1 / 64)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8)
    H64 = pkg.Hierarchy(g, coarsest_dx=1 / 8, outer_f64=True)
    _, cp, _ = g.export()
    _, f_h = synth.circle_fourier(cp[: g.nb])
    f = torch.from_numpy(f_h).cuda()
    u, rep = H.solve(f, tol=1e-12, max_iter=80, mode=mode)
    assert rep["converged"] and rep["f64_checks"] >= 1, rep
    r64 = H64.residual(f, u)
    assert float(r64.abs().max()) / float(f.abs().max()) <= 1e-12
