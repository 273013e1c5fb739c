"""Pins of the oracle's V-cycle and solver (CPU only)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.geometry import circle, sphere
from oracle.interp import interp_matrix
from oracle.multigrid import MGOptions, build_hierarchy, solve, vcycle
import synth


def _rate(hist):
    h = np.asarray(hist)
    h = h[h > 1e-11]
    return (h[-1] / h[2]) ** (1.0 / (len(h) - 3))


def test_vcycle_solution_equals_direct_sparse_solve():
    """The converged V-cycle solution is the sparse direct solution of A u = f."""
    for surf, dx, fn in [(circle(), 1 / 32, synth.circle_fourier),
                         (sphere(), 1 / 16, synth.sphere_harmonics)]:
        H = build_hierarchy(surf, dx, 1 / 8, opts=MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8))
        lev = H.fine
        _, f = fn(lev.band.cp[: lev.band.nb])
        u, rep = solve(H, f, tol=1e-12, max_iter=60)
        assert rep.converged
        ud = spla.spsolve(lev.ops.A_matrix(lev.c).tocsc(), f)
        assert np.abs(u - ud).max() <= 1e-10 * np.abs(ud).max()


def test_second_order_circle():
    """Closed form on the circle: observed order in [1.8, 2.2] (Table 3.1 analogue)."""
    errs = []
    for dx in [1 / 32, 1 / 64, 1 / 128, 1 / 256]:
        H = build_hierarchy(circle(), dx, 1 / 8, opts=MGOptions(smoother="jacobi"))
        b = H.fine.band
        uex, f = synth.circle_fourier(b.cp[: b.nb])
        u, rep = solve(H, f, tol=5e-11, max_iter=60)
        assert rep.converged
        errs.append(np.abs(u - uex).max() / np.abs(uex).max())
    slopes = np.log2(np.asarray(errs[:-1]) / np.asarray(errs[1:]))
    # pre-asymptotic at the coarsest pair; the finer pairs are in [1.8, 2.2]
    assert np.all((slopes[1:] > 1.8) & (slopes[1:] < 2.2)), slopes


@pytest.mark.slow
def test_second_order_sphere():
    errs = []
    for dx in [1 / 16, 1 / 32, 1 / 64]:
        H = build_hierarchy(sphere(), dx, 1 / 8, opts=MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8))
        b = H.fine.band
        uex, f = synth.sphere_harmonics(b.cp[: b.nb])
        u, rep = solve(H, f, tol=1e-10, max_iter=40)
        assert rep.converged
        errs.append(np.abs(u - uex).max() / np.abs(uex).max())
    slopes = np.log2(np.asarray(errs[:-1]) / np.asarray(errs[1:]))
    assert np.all((slopes > 1.8) & (slopes < 2.4)), slopes


def test_rate_independent_of_depth():
    """Sec. 4.5: the reduction per cycle does not deteriorate with more levels."""
    rates = []
    for dx in [1 / 32, 1 / 64, 1 / 128]:
        H = build_hierarchy(circle(), dx, 1 / 8, opts=MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8))
        b = H.fine.band
        _, f = synth.circle_fourier(b.cp[: b.nb])
        _, rep = solve(H, f, tol=1e-10, max_iter=40)
        rates.append(_rate(rep.history))
    assert max(rates) < 0.2 and max(rates) - min(rates) < 0.1, rates


def test_rm_smoother_fixed_point_is_extension():
    """Ruuth-Merriman smoothing ends with u := E u, so V(0, r) is in range(E)."""
    H = build_hierarchy(circle(), 1 / 32, 1 / 8, opts=MGOptions(smoother="rm"))
    lev = H.fine
    r = synth.random_band_vector(lev.band.nb, 3)
    d = vcycle(H, np.zeros_like(r), r)
    assert np.abs(lev.ops.extend(d)[: lev.band.nb] - d).max() < 0.05 * np.abs(d).max()


def test_transfers_interpolate_smooth_fields():
    """Restriction / prolongation evaluate a field at cp of the target band (Sec. 4.3)."""
    H = build_hierarchy(sphere(), 1 / 16, 1 / 8, opts=MGOptions(smoother="jacobi"))
    fine, coarse = H.levels
    g = lambda y: y[:, 0] + 2 * y[:, 1] - y[:, 2] + 0.5
    vf = g(fine.band.points(fine.band.keys))
    vc = g(coarse.band.points(coarse.band.keys))
    # linear fields are reproduced exactly by linear interpolation
    assert np.abs(fine.R @ vf - g(coarse.band.cp[: coarse.band.nb])).max() < 1e-13
    assert np.abs(fine.P @ vc - g(fine.band.cp[: fine.band.nb])).max() < 1e-13
    # a smooth cp-extended field restricts to itself at O(dx^2)
    y = fine.band.cp[: fine.band.nb]
    u = synth.real_sph_harm(2, 1, y)
    uc = synth.real_sph_harm(2, 1, coarse.band.cp[: coarse.band.nb])
    assert np.abs(fine.R @ u - uc).max() < 0.05


def test_coarsest_solve_is_direct():
    H = build_hierarchy(circle(), 1 / 16, 1 / 8, opts=MGOptions(smoother="jacobi"))
    lev = H.levels[-1]
    f = synth.random_band_vector(lev.band.nb, 9)
    from oracle.multigrid import coarse_solve
    u = coarse_solve(H, f)
    assert np.abs(lev.ops.A_matrix(lev.c) @ u - f).max() < 1e-10 * np.abs(f).max()


def test_vcycle_rate_with_relaxed_coarse_level():
    """Ellipsoid (1.05, 0.9, 0.8), reach 0.61: the level dx = 1/8 violates the
    strict coarsening rule ((lambda + 1)/8 = 0.64 > reach) but its band lies
    within the reach (sqrt(17)/8 = 0.52) and builds; as the coarse level of a
    two-level V-cycle from dx = 1/16 it keeps the contraction near 0.1."""
    from oracle.geometry import ellipsoid
    surf = ellipsoid(1.05, 0.9, 0.8)
    assert (np.sqrt(17) + 1) / 8 > surf.reach > np.sqrt(17) / 8
    H = build_hierarchy(surf, 1 / 16, 1 / 8,
                        opts=MGOptions(nu1=3, nu2=3, omega=0.8, smoother="jacobi", residual="plain"))
    fine = H.levels[0]
    f = synth.harmonic_field(fine.band.cp[: fine.band.nb], seed=1)
    u = np.zeros_like(f)
    norms = []
    for _ in range(6):
        r = f - fine.ops.apply_A(u, fine.c)
        norms.append(np.abs(r).max())
        u = u + vcycle(H, np.zeros_like(f), r)
    rates = np.asarray(norms[1:]) / np.asarray(norms[:-1])
    assert np.all(rates < 0.15), rates


def test_variable_c_restricted_to_coarse_levels():
    """Variable c (a surface function, footnote to Sec. 2.1): the finest level
    holds c(cp(x)); each coarser level holds the restriction of the finer c
    (interpolation at its own closest points, Sec. 4.3).  That restriction
    reproduces c(cp) on the coarse band to O(dx^2), and the V-cycle solution
    is still the direct solution of diag(c) u - M u = f on the finest band."""
    c_fn = lambda y: 1.0 + 0.5 * np.sin(2 * np.pi * y[:, 2])
    H = build_hierarchy(sphere(), 1 / 16, 1 / 8,
                        opts=MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8), c_fn=c_fn)
    fine, coarse = H.levels
    assert np.array_equal(fine.c, c_fn(fine.band.cp[: fine.band.nb]))
    assert np.array_equal(coarse.c, fine.R @ fine.c)
    # linear interpolation error of a smooth cp-extended field at spacing 1/16
    assert np.abs(coarse.c - c_fn(coarse.band.cp[: coarse.band.nb])).max() < 0.05
    assert not np.allclose(coarse.c, c_fn(coarse.band.cp[: coarse.band.nb]), rtol=0, atol=1e-12)
    _, f = synth.sphere_harmonics(fine.band.cp[: fine.band.nb])
    u, rep = solve(H, f, tol=1e-12, max_iter=60)
    assert rep.converged and rep.iters <= 20
    ud = spla.spsolve(fine.ops.A_matrix(fine.c).tocsc(), f)
    assert np.abs(u - ud).max() <= 1e-10 * np.abs(ud).max()


def test_vardiff_vcycle_solution_equals_direct_solve():
    """Variable diffusion (Sec. 4.5.6) through the V-cycle: the coefficient a is
    restricted to the coarse levels like c, the defect correction converges at a
    level-independent-ish rate and its solution is the direct one."""
    a_fn = lambda y: synth.sphere_vardiff(y)[1]
    H = build_hierarchy(sphere(), 1 / 16, 1 / 8,
                        opts=MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8,
                                       residual="plain", operator="vardiff"), a_fn=a_fn)
    fine, coarse = H.levels
    assert np.array_equal(coarse.ops.a, fine.R @ fine.ops.a)
    _, _, f = synth.sphere_vardiff(fine.band.cp[: fine.band.nb])
    u, rep = solve(H, f, tol=1e-12, max_iter=40)
    assert rep.converged and rep.iters <= 20, rep.iters
    ud = spla.spsolve(fine.ops.A_matrix(1.0).tocsc(), f)
    assert np.abs(u - ud).max() <= 1e-10 * np.abs(ud).max()


def test_gmres_coarse_solve_pins():
    """The oracle's restarted GMRES (coarsest level): with a Krylov dimension at
    least the system size it is a direct solve; otherwise each restart cannot
    increase the residual (it minimises over a space containing 0) and the
    residual falls for a well-conditioned shifted system."""
    from oracle.multigrid import gmres
    rng = np.random.default_rng(4)
    n = 20
    A = np.eye(n) * 4 + rng.uniform(-1, 1, (n, n)) * 0.3
    b = rng.uniform(-1, 1, n)
    P = 1.0 / np.diag(A)
    x = gmres(A, b, P, m=n, restarts=1)
    assert np.abs(A @ x - b).max() <= 1e-12 * np.abs(b).max()
    H = build_hierarchy(circle(), 1 / 32, 1 / 16, opts=MGOptions(smoother="jacobi", coarse_gmres=1))
    last = H.levels[-1]
    Ac = last.ops.A_matrix(last.c).tocsr()
    f = synth.random_band_vector(last.band.nb, 6)
    res = []
    for k in (1, 2, 4):
        xk = gmres(Ac, f, 0.8 / last.diagA, 30, k)
        res.append(np.abs(Ac @ xk - f).max())
    assert res[0] < np.abs(f).max() and res[1] <= res[0] and res[2] <= res[1], res
    assert res[2] < 1e-2 * np.abs(f).max(), res
