"""GPU parity for the stated workload configurations (CUDA path vs the oracle).

* variable c = 1 + 0.5 sin(2 pi z) at cp (footnote to Sec. 2.1): residual,
  one V-cycle and the converged solve, with c restricted to coarse levels by
  the closest-point restriction of Sec. 4.3 on both sides;
* the circle schedule of the 2-D workload: nu1 = nu2 = 2, omega = 2/3,
  levels dx = 1/64 .. 1/8, against the sparse direct solution and the exact
  solution sin(theta) + cos(3 theta);
* a batch of uneven systems solved by cpm_solve_batch against the oracle's
  sparse direct solutions.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from helpers import oracle_surface, perm_gpu_to_oracle, require_cuda
from oracle.band import build_band
from oracle.multigrid import MGOptions, build_hierarchy, vcycle
from oracle.operators import Operators
import synth

pytestmark = pytest.mark.gpu


def c_fn(y):
    return 1.0 + 0.5 * np.sin(2 * np.pi * y[:, 2])


def _variable_c_pair():
    torch, pkg = require_cuda()
    g = pkg.Band("sphere", (), 1 / 16)
    ijk, cp, _ = g.export()
    c_dev = torch.from_numpy(c_fn(cp[: g.nb])).cuda()
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8, nu1=3, nu2=3, omega=0.8, residual="extended",
                      c_device=c_dev)
    OH = build_hierarchy(oracle_surface("sphere", ()), 1 / 16, 1 / 8,
                         opts=MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8), c_fn=c_fn)
    perm = perm_gpu_to_oracle(g, OH.fine.band)
    return torch, pkg, g, H, OH, perm


def test_variable_c_residual_vcycle_and_solve():
    torch, pkg, g, H, OH, perm = _variable_c_pair()
    fine = OH.fine
    nb = fine.band.nb
    # residual r = f - (diag(c) - M) u, FP64, random inputs (no cancellation)
    f_o = synth.random_band_vector(nb, 31)
    u_o = synth.random_band_vector(nb, 32)
    ref = fine.ops.residual(u_o, f_o, fine.c)[perm]
    got = H.residual(torch.from_numpy(f_o[perm]).cuda(), torch.from_numpy(u_o[perm]).cuda())
    err = np.abs(got.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 1e-13, err
    # one FP64 V-cycle from zero (coarse c = restriction of the fine c)
    ref = vcycle(OH, np.zeros(nb), f_o)[perm]
    u = torch.zeros(nb, dtype=torch.float64, device="cuda")
    H.vcycle(torch.from_numpy(f_o[perm]).cuda(), u)
    err = np.abs(u.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 1e-10, err
    # converged solution = sparse direct solution, both solver forms
    _, f_s = synth.sphere_harmonics(fine.band.cp[:nb])
    ud = spla.spsolve(fine.ops.A_matrix(fine.c).tocsc(), f_s)
    for mode in ("f64", "mixed"):
        us, rep = H.solve(torch.from_numpy(f_s[perm]).cuda(), tol=1e-12, max_iter=80, mode=mode)
        assert rep["converged"], (mode, rep)
        err = np.abs(us.cpu().numpy() - ud[perm]).max() / np.abs(ud).max()
        assert err <= 1e-9, (mode, err)


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_circle_schedule_nu2_omega_two_thirds(mode):
    """Unit circle, dx = 1/64 (2912 points), (1 - Lap_S) u = f with
    u = sin(theta) + cos(3 theta), weighted Jacobi omega = 2/3 with 2 pre- and 2
    post-sweeps, levels down to dx = 1/8, solved to 1e-10 and to 1e-12."""
    torch, pkg = require_cuda()
    dx = 1 / 64
    g = pkg.Band("circle", (), dx)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8, nu1=2, nu2=2, omega=2 / 3)
    assert H.n_levels == 4 and g.nb == 2912
    ob = build_band(oracle_surface("circle", ()), dx)
    perm = perm_gpu_to_oracle(g, ob)
    uex_o, f_o = synth.circle_fourier(ob.cp[: ob.nb])
    ud = spla.spsolve(Operators(ob).A_matrix(1.0).tocsc(), f_o)
    ft = torch.from_numpy(f_o[perm]).cuda()
    u10, rep10 = H.solve(ft, tol=1e-10, max_iter=100, mode=mode)
    assert rep10["converged"] and rep10["rel_residual"] <= 1e-10, rep10
    # the discretisation error dominates the 1e-10 algebraic error (second order)
    e_exact = np.abs(u10.cpu().numpy() - uex_o[perm]).max() / np.abs(uex_o).max()
    assert 1e-5 < e_exact < 1e-3, e_exact
    u12, rep12 = H.solve(ft, tol=1e-12, max_iter=100, mode=mode)
    assert rep12["converged"], rep12
    err = np.abs(u12.cpu().numpy() - ud[perm]).max() / np.abs(ud).max()
    assert err <= 1e-9, err


def test_batch_matches_oracle_direct_solutions():
    """An uneven batch (circle 1/64, sphere 1/16, ellipsoid (1.05, 0.9, 0.8) 1/16;
    2 right-hand sides each) solved by one cpm_solve_batch call: every system's
    solution equals the oracle's sparse direct solution within 1e-9."""
    torch, pkg = require_cuda()
    cases = [("circle", (), 1 / 64), ("sphere", (), 1 / 16), ("ellipsoid", (1.05, 0.9, 0.8), 1 / 16)]
    n_rhs = 2
    hs, fs, refs = [], [], []
    for i, (kind, params, dx) in enumerate(cases):
        g = pkg.Band(kind, params, dx)
        H = pkg.Hierarchy(g, coarsest_dx=1 / 8)
        ob = build_band(oracle_surface(kind, params), dx)
        perm = perm_gpu_to_oracle(g, ob)
        A = Operators(ob).A_matrix(1.0).tocsc()
        lu = spla.splu(A)
        for k in range(n_rhs):
            f_o = synth.random_band_vector(ob.nb, 100 * i + k)
            refs.append(lu.solve(f_o)[perm])
            fs.append(torch.from_numpy(f_o[perm]).cuda())
        hs.append(H)
    sizes = [h.nb for h in hs]
    assert len(set(sizes)) == len(sizes)
    B = pkg.Batch(hs, n_rhs)
    for mode in ("mixed", "f64"):
        us, reps = B.solve(fs, tol=1e-12, max_iter=100, mode=mode, inner_cycles=2, zero_init=True)
        for s, (u, ref, rep) in enumerate(zip(us, refs, reps)):
            assert rep["converged"], (mode, s, rep)
            err = np.abs(u.cpu().numpy() - ref).max() / np.abs(ref).max()
            assert err <= 1e-9, (mode, s, err)
    B.close()
