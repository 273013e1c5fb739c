"""Pins of the oracle's smoothers and V-cycle against their matrix forms (CPU).

The V-cycle of Algorithm 4.1 started from u = 0 is a linear map T of the
right-hand side.  Written with matrices assembled independently of the
oracle's step-by-step code (A from the assembled operator, its diagonal taken
from the matrix, transfers from the interpolation matrices), one cycle is

    smoothing   u <- S u + W f,   Jacobi on A (Eq. 4.1): S = I - omega D^-1 A,
                                  W = omega D^-1, D = diag(A);
                                  Ruuth-Merriman (Eq. 4.2): S = E_B (I - omega Dt^-1 At),
                                  W = E_B omega Dt^-1, At = cI - L_band;
    correction  u <- u + P T_c R (f - A_r u),  A_r = A (plain residual),
                A E_B (the re-extended residual of Sec. 4.4) or At (RM),
                T_c = A_c^-1 on the coarsest level, else the coarse V-cycle map;

nu1 smoothing steps, the correction, nu2 smoothing steps.  The tests apply
the oracle's V-cycle to unit vectors (brute force on the circle, random probes
on the sphere) and compare with that formula, so a wrong weight, diagonal,
sweep count, residual or transfer fails.  The outer defect correction
u += V(0, f - A u) contracts errors by I - T A; its spectral radius is
compared with the contraction the oracle's solve loop shows.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.geometry import circle, sphere
from oracle.interp import interp_matrix
from oracle.multigrid import MGOptions, build_hierarchy, coarse_solve, smooth, solve, vcycle
import synth


def _level_mats(lev, opts):
    """(S, W, A, A_r) of one level as dense or sparse matrices."""
    ops, nb = lev.ops, lev.band.nb
    A = ops.A_matrix(lev.c).toarray()
    E_B = ops.E[:nb].toarray()
    if opts.smoother == "rbgs":
        # red half-step (colour 0 = even i + j), then black half-step
        Dinv = 1.0 / np.diag(A)
        red = (lev.band.coords_of(lev.band.keys).sum(axis=1) % 2 == 0).astype(float)
        S_parts, W_parts = [], []
        for m in (red, 1.0 - red):
            S_parts.append(np.eye(nb) - opts.omega * (m * Dinv)[:, None] * A)
            W_parts.append(np.diag(opts.omega * m * Dinv))
        S = S_parts[1] @ S_parts[0]
        W = S_parts[1] @ W_parts[0] + W_parts[1]
        A_r = A if opts.residual == "plain" else A @ E_B
        return S, W, A, A_r
    if opts.smoother == "jacobi":
        Dinv = 1.0 / np.diag(A)
        S = np.eye(nb) - opts.omega * Dinv[:, None] * A
        W = np.diag(opts.omega * Dinv)
        A_r = A if opts.residual == "plain" else A @ E_B
    else:
        At = (sp.diags(np.broadcast_to(lev.c, (nb,))) - ops.Lb).toarray()
        Dtinv = 1.0 / np.diag(At)
        S = E_B @ (np.eye(nb) - opts.omega * Dtinv[:, None] * At)
        W = E_B @ np.diag(opts.omega * Dtinv)
        A_r = At
    return S, W, A, A_r


def _formula_T(H, l=0):
    """Dense matrix of V(0, .) on level l from the formula in the module header."""
    o = H.opts
    lev = H.levels[l]
    _, _, A, _ = _level_mats(lev, o)
    if l == len(H.levels) - 1:
        return np.linalg.inv(A)
    S, W, _, A_r = _level_mats(lev, o)
    nb = lev.band.nb
    coarse = H.levels[l + 1]
    R = interp_matrix(lev.band, coarse.band.cp[: coarse.band.nb], o.transfer_p).toarray()
    P = interp_matrix(coarse.band, lev.band.cp[:nb], o.transfer_p).toarray()
    Tc = _formula_T(H, l + 1)
    if o.cycle == 2 and l + 1 < len(H.levels) - 1:
        # W-cycle: a second coarse cycle from the first's result,
        # V(V(0, g), g) = (I - Tc Ac) Tc g + Tc g for the consistent coarse cycle
        Ac = _level_mats(H.levels[l + 1], o)[2]
        Tc = 2 * Tc - Tc @ Ac @ Tc
    N = np.zeros((nb, nb))
    for _ in range(o.nu1):
        N = S @ N + W
    N = N + P @ Tc @ R @ (np.eye(nb) - A_r @ N)
    for _ in range(o.nu2):
        N = S @ N + W
    return N


def _brute_T(H):
    n = H.fine.band.nb
    return np.stack([vcycle(H, np.zeros(n), e) for e in np.eye(n)], axis=1)


CASES_EXTRA = [MGOptions(smoother="rbgs", nu1=2, nu2=2, omega=1.0, residual="plain"),
               MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8, residual="plain", transfer_p=3)]
CASES = [MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8, residual="plain"),
         MGOptions(smoother="jacobi", nu1=2, nu2=2, omega=2 / 3, residual="extended"),
         MGOptions(smoother="jacobi", nu1=1, nu2=2, omega=0.8, residual="plain"),
         MGOptions(smoother="rm", nu1=3, nu2=3, omega=1.0),
         MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8, residual="extended",
                   operator="paper")]


@pytest.mark.parametrize("opts", CASES + CASES_EXTRA,
                         ids=lambda o: f"{o.smoother}-{o.nu1}{o.nu2}-{o.omega:.2f}-{o.residual}-{o.operator}"
                                       f"-p{o.transfer_p}")
def test_two_level_vcycle_matrix_equals_formula(opts):
    """Circle dx = 1/16 -> 1/8 (712 and 360 points): brute-force V-cycle matrix."""
    H = build_hierarchy(circle(), 1 / 16, 1 / 8, opts=opts)
    T = _brute_T(H)
    F = _formula_T(H)
    assert np.abs(T - F).max() <= 1e-12 * np.abs(F).max()


def test_three_level_vcycle_matrix_equals_recursive_formula():
    """Circle dx = 1/32 -> 1/16 -> 1/8: the coarse correction is the recursive
    V-cycle map of the next level (Algorithm 4.1 with u = 0 on coarse levels)."""
    opts = CASES[1]
    H = build_hierarchy(circle(), 1 / 32, 1 / 8, opts=opts)
    assert len(H.levels) == 3
    T = _brute_T(H)
    F = _formula_T(H)
    assert np.abs(T - F).max() <= 1e-11 * np.abs(F).max()
    # dropping the recursion (a direct solve one level down) is a different map
    Hd = build_hierarchy(circle(), 1 / 32, 1 / 16, opts=opts)
    assert np.abs(_brute_T(Hd) - T).max() > 1e-3 * np.abs(T).max()


def test_sphere_vcycle_probes_equal_formula():
    """Unit sphere dx = 1/16 -> 1/8 (26974 and 7190 points): the V-cycle map on
    three random probes equals the formula evaluated with sparse matrices."""
    opts = MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8, residual="extended")
    H = build_hierarchy(sphere(), 1 / 16, 1 / 8, opts=opts)
    fine, coarse = H.levels
    nb = fine.band.nb
    A = fine.ops.A_matrix(fine.c).tocsr()
    d = A.diagonal()
    A_r = (A @ fine.ops.E[:nb]).tocsr()
    Ac = coarse.ops.A_matrix(coarse.c).toarray()
    lu = sla.lu_factor(Ac)
    R = interp_matrix(fine.band, coarse.band.cp[: coarse.band.nb], 1)
    P = interp_matrix(coarse.band, fine.band.cp[:nb], 1)
    for seed in range(3):
        f = synth.random_band_vector(nb, 40 + seed)
        u = np.zeros(nb)
        for _ in range(opts.nu1):
            u = u + opts.omega * (f - A @ u) / d
        u = u + P @ sla.lu_solve(lu, R @ (f - A_r @ u))
        for _ in range(opts.nu2):
            u = u + opts.omega * (f - A @ u) / d
        got = vcycle(H, np.zeros(nb), f)
        assert np.abs(got - u).max() <= 1e-12 * np.abs(u).max()


@pytest.mark.parametrize("opts", [CASES[0], CASES[1]], ids=["nu3-omega0.8-plain", "nu2-omega0.67-ext"])
def test_spectral_radius_matches_observed_contraction(opts):
    """rho(I - T A) of the brute-force map is the asymptotic contraction per
    outer iteration of the oracle's solve loop (circle dx = 1/16 -> 1/8)."""
    H = build_hierarchy(circle(), 1 / 16, 1 / 8, opts=opts)
    lev = H.fine
    A = lev.ops.A_matrix(lev.c).toarray()
    G = np.eye(A.shape[0]) - _brute_T(H) @ A
    rho = np.abs(np.linalg.eigvals(G)).max()
    assert 0.02 < rho < 0.2, rho
    f = synth.random_band_vector(lev.band.nb, 5)
    _, rep = solve(H, f, tol=1e-14, max_iter=12)
    h = np.asarray(rep.history)
    h = h[h > 1e-13]
    observed = (h[-1] / h[-4]) ** (1.0 / 3.0)
    assert abs(observed - rho) <= 0.15 * rho, (observed, rho)


def test_rm_vcycle_is_not_consistent_with_A():
    """Ruuth-Merriman smoothing and its residual use cI - L_band (Eq. 4.2), so
    the cycle is not a splitting of A: its own iteration V(u, 0) contracts fast,
    but the defect correction u += V(0, f - A u) has rho(I - T A) >= 1 and
    does not converge to A^-1 f.  This is the stagnation the reading of the
    smoother (Jacobi on A as the default) rests on."""
    opts = CASES[3]
    assert opts.smoother == "rm"
    H = build_hierarchy(circle(), 1 / 16, 1 / 8, opts=opts)
    lev = H.fine
    n = lev.band.nb
    A = lev.ops.A_matrix(lev.c).toarray()
    T = _brute_T(H)
    V0 = np.stack([vcycle(H, e, np.zeros(n)) for e in np.eye(n)], axis=1)
    assert np.abs(np.linalg.eigvals(V0)).max() < 0.2
    assert np.abs(V0 - (np.eye(n) - T @ A)).max() > 1e-2
    assert np.abs(np.linalg.eigvals(np.eye(n) - T @ A)).max() >= 1.0


def test_coarse_sweeps_are_the_jacobi_neumann_series():
    """coarse_sweeps = k replaces the direct coarsest solve by k weighted Jacobi
    sweeps on A from zero: u = sum_{j<k} S^j omega D^-1 f = (I - S^k) A^-1 f."""
    k = 7
    opts = MGOptions(smoother="jacobi", nu1=2, nu2=2, omega=0.8, coarse_sweeps=k)
    H = build_hierarchy(circle(), 1 / 16, 1 / 8, opts=opts)
    last = H.levels[-1]
    A = last.ops.A_matrix(last.c).toarray()
    S = np.eye(len(A)) - 0.8 * A / np.diag(A)[:, None]
    f = synth.random_band_vector(len(A), 8)
    ref = (np.eye(len(A)) - np.linalg.matrix_power(S, k)) @ np.linalg.solve(A, f)
    got = coarse_solve(H, f)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # and the smoothing step of the finest level is one such sweep
    u0 = synth.random_band_vector(H.fine.band.nb, 9)
    fl = synth.random_band_vector(H.fine.band.nb, 10)
    Af = H.fine.ops.A_matrix(H.fine.c).toarray()
    ref1 = u0 + 0.8 * (fl - Af @ u0) / np.diag(Af)
    assert np.abs(smooth(H, 0, u0, fl) - ref1).max() <= 1e-12 * np.abs(ref1).max()


def test_paper_form_operator_is_eq_3_3():
    """The paper-form operator of the oracle's V-cycle is M = E_1 L_band -
    gamma (I - E_3), assembled independently here from the interpolation and
    Laplacian matrices; its V-cycle defect correction converges to the direct
    solution."""
    from oracle.operators import PaperOperators, gamma, lap_band
    opts = CASES[4]
    H = build_hierarchy(circle(), 1 / 32, 1 / 8, opts=opts)
    lev = H.fine
    b = lev.band
    cpB = b.cp[: b.nb]
    M = (interp_matrix(b, cpB, 1) @ lap_band(b)
         - gamma(b) * (sp.identity(b.nb) - interp_matrix(b, cpB, 3))).toarray()
    assert isinstance(lev.ops, PaperOperators)
    assert np.abs(lev.ops.M.toarray() - M).max() <= 1e-12 * gamma(b)
    f = synth.random_band_vector(b.nb, 12)
    u, rep = solve(H, f, tol=1e-12, max_iter=60)
    assert rep.converged and rep.iters <= 20
    ud = np.linalg.solve(np.diag(lev.c) - M, f)
    assert np.abs(u - ud).max() <= 1e-10 * np.abs(ud).max()


def test_w_cycle_matrix_equals_recursive_formula():
    """cycle = 2 (the W-cycle of the remark at Algorithm 4.1) on circle
    dx = 1/32 -> 1/16 -> 1/8: the middle level takes two coarse cycles, the
    second from the first's result; it differs from the V-cycle."""
    opts = MGOptions(smoother="jacobi", nu1=2, nu2=2, omega=0.8, residual="plain", cycle=2)
    H = build_hierarchy(circle(), 1 / 32, 1 / 8, opts=opts)
    T = _brute_T(H)
    F = _formula_T(H)
    assert np.abs(T - F).max() <= 1e-11 * np.abs(F).max()
    Hv = build_hierarchy(circle(), 1 / 32, 1 / 8,
                         opts=MGOptions(smoother="jacobi", nu1=2, nu2=2, omega=0.8, residual="plain"))
    assert np.abs(_brute_T(Hv) - T).max() > 1e-3 * np.abs(T).max()


def test_fmg_is_prolonged_coarse_solution_then_one_cycle():
    """Full multigrid on two levels (circle dx = 1/16 -> 1/8): the coarsest
    solution of the restricted right-hand side, prolonged, starts one cycle:
    fmg(f) = G P A_c^-1 R f + T f with G = V(., 0) and T = V(0, .)."""
    from oracle.multigrid import fmg
    opts = MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8, residual="extended")
    H = build_hierarchy(circle(), 1 / 16, 1 / 8, opts=opts)
    fine, coarse = H.levels
    n = fine.band.nb
    T = _brute_T(H)
    G = np.stack([vcycle(H, e, np.zeros(n)) for e in np.eye(n)], axis=1)
    Ac = coarse.ops.A_matrix(coarse.c).toarray()
    R = interp_matrix(fine.band, coarse.band.cp[: coarse.band.nb], 1).toarray()
    P = interp_matrix(coarse.band, fine.band.cp[:n], 1).toarray()
    f = synth.random_band_vector(n, 13)
    ref = G @ (P @ np.linalg.solve(Ac, R @ f)) + T @ f
    got = fmg(H, f)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    # the defect correction that starts with it converges to the direct solution
    A = fine.ops.A_matrix(fine.c).toarray()
    u, rep = solve(H, f, tol=1e-12, max_iter=40, first_fmg=True)
    assert rep.converged
    assert np.abs(u - np.linalg.solve(A, f)).max() <= 1e-10 * np.abs(u).max()


def test_cubic_transfers_speed_up_the_cycle():
    """Cubic (degree 3) restriction and prolongation: on circle dx = 1/32 ->
    1/8 the defect correction contracts faster than with linear transfers
    (rho(I - T A) from the brute-force map)."""
    rhos = []
    for p in (1, 3):
        H = build_hierarchy(circle(), 1 / 32, 1 / 8,
                            opts=MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8,
                                           residual="plain", transfer_p=p))
        A = H.fine.ops.A_matrix(H.fine.c).toarray()
        rhos.append(np.abs(np.linalg.eigvals(np.eye(len(A)) - _brute_T(H) @ A)).max())
    assert rhos[1] < 0.5 * rhos[0], rhos


def test_red_black_gauss_seidel_degrades_with_resolution():
    """Red-black Gauss-Seidel on A (the alternative smoother Sec. 4.4 names):
    the interpolation stencils couple nodes of one colour, and the contraction
    rho(I - T A) of the defect correction it smooths grows as dx shrinks; with
    the MBR form it exceeds 1 at dx = 1/32 (circle), so it is implemented but
    is not a usable smoother here."""
    rho = {}
    for op in ("mbr", "paper"):
        for dx in (1 / 16, 1 / 32):
            H = build_hierarchy(circle(), dx, 1 / 8,
                                opts=MGOptions(smoother="rbgs", nu1=3, nu2=3, omega=1.0,
                                               residual="plain", operator=op))
            A = H.fine.ops.A_matrix(H.fine.c).toarray()
            rho[op, dx] = np.abs(np.linalg.eigvals(np.eye(len(A)) - _brute_T(H) @ A)).max()
        assert rho[op, 1 / 32] > 1.5 * rho[op, 1 / 16], rho
    assert rho["mbr", 1 / 32] > 1.0 and rho["paper", 1 / 32] > 0.6, rho
