"""Smoother and cycle variants on the GPU against the oracle (remark at
Algorithm 4.1, Sec. 4.4): cubic restriction / prolongation, the W-cycle, full
multigrid and red-black Gauss-Seidel smoothing."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from helpers import oracle_surface, perm_gpu_to_oracle, require_cuda
from oracle.multigrid import MGOptions, build_hierarchy, fmg, vcycle
import synth

pytestmark = pytest.mark.gpu


def _pair(kind, params, dx, coarsest=1 / 8, **kw):
    torch, pkg = require_cuda()
    o = dict(smoother="jacobi", nu1=3, nu2=3, omega=0.8, residual="extended")
    o.update(kw)
    g = pkg.Band(kind, params, dx)
    H = pkg.Hierarchy(g, coarsest_dx=coarsest, nu1=o["nu1"], nu2=o["nu2"], omega=o["omega"],
                      smoother=o["smoother"], residual=o["residual"],
                      transfer_deg=o.get("transfer_p", 1), cycle=o.get("cycle", 1))
    OH = build_hierarchy(oracle_surface(kind, params), dx, coarsest, opts=MGOptions(**o))
    perm = perm_gpu_to_oracle(g, OH.fine.band)
    return torch, pkg, g, H, OH, perm


VARIANTS = [dict(transfer_p=3), dict(cycle=2), dict(smoother="rbgs", omega=1.0, residual="plain")]


@pytest.mark.parametrize("kw", VARIANTS, ids=["cubic-transfers", "w-cycle", "red-black-gs"])
@pytest.mark.parametrize("kind,params,dx", [("circle", (), 1 / 64), ("sphere", (), 1 / 32)])
def test_cycle_variant_parity(kind, params, dx, kw):
    """One FP64 cycle from zero equals the oracle's (FP32 within single precision)."""
    torch, pkg, g, H, OH, perm = _pair(kind, params, dx, **kw)
    nb = OH.fine.band.nb
    f_o = synth.random_band_vector(nb, 51)
    ref = vcycle(OH, np.zeros(nb), f_o)[perm]
    u = torch.zeros(nb, dtype=torch.float64, device="cuda")
    H.vcycle(torch.from_numpy(f_o[perm]).cuda(), u)
    err = np.abs(u.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 1e-10, err
    u32 = torch.zeros(nb, dtype=torch.float32, device="cuda")
    H.vcycle(torch.from_numpy(f_o[perm]).float().cuda(), u32)
    assert np.abs(u32.double().cpu().numpy() - ref).max() <= 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("kw", VARIANTS[:2], ids=["cubic-transfers", "w-cycle"])
def test_cycle_variant_solves(kw):
    """Circle dx = 1/64: the converged solution equals the sparse direct solution."""
    torch, pkg, g, H, OH, perm = _pair("circle", (), 1 / 64, **kw)
    fine = OH.fine
    _, f_o = synth.circle_fourier(fine.band.cp[: fine.band.nb])
    ud = spla.spsolve(fine.ops.A_matrix(1.0).tocsc(), f_o)
    for mode in ("f64", "mixed"):
        u, rep = H.solve(torch.from_numpy(f_o[perm]).cuda(), tol=1e-12, max_iter=60, mode=mode)
        assert rep["converged"], (mode, rep)
        assert np.abs(u.cpu().numpy() - ud[perm]).max() <= 1e-9 * np.abs(ud).max()


@pytest.mark.parametrize("kind,params,dx", [("circle", (), 1 / 64), ("sphere", (), 1 / 32)])
def test_full_multigrid_first_iteration(kind, params, dx):
    """cpm_solve with fmg: after one outer iteration from u = 0 the iterate is the
    oracle's full-multigrid solution of f (FP64); the solve then converges."""
    torch, pkg, g, H, OH, perm = _pair(kind, params, dx, transfer_p=3)
    nb = OH.fine.band.nb
    f_o = synth.random_band_vector(nb, 52)
    ref = fmg(OH, f_o)[perm]
    ft = torch.from_numpy(f_o[perm]).cuda()
    u1, rep1 = H.solve(ft, tol=1e-30, max_iter=1, mode="f64", fmg=True, raise_on_fail=False)
    assert rep1["iters"] == 1
    err = np.abs(u1.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 1e-10, err
    for mode in ("f64", "mixed"):
        u, rep = H.solve(ft, tol=1e-10, max_iter=60, mode=mode, fmg=True)
        assert rep["converged"], (mode, rep)


@pytest.mark.parametrize("kind,params,dx", [("circle", (), 1 / 64), ("sphere", (), 1 / 32)])
def test_relative_form_vcycle_parity(kind, params, dx):
    """relative = 1: the V-cycle's residuals and Jacobi updates in the relative
    form (the same operator, other rounding) equal the oracle's cycle in FP64,
    and the FP32 cycles of both forms stay within single precision of it on
    smooth data."""
    torch, pkg = require_cuda()
    g = pkg.Band(kind, params, dx)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8, nu1=3, nu2=3, omega=0.8, residual="plain", relative=True)
    H0 = pkg.Hierarchy(g, coarsest_dx=1 / 8, nu1=3, nu2=3, omega=0.8, residual="plain")
    OH = build_hierarchy(oracle_surface(kind, params), dx, 1 / 8,
                         opts=MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8, residual="plain"))
    perm = perm_gpu_to_oracle(g, OH.fine.band)
    nb = OH.fine.band.nb
    f_o = synth.random_band_vector(nb, 53)
    ref = vcycle(OH, np.zeros(nb), f_o)[perm]
    u = torch.zeros(nb, dtype=torch.float64, device="cuda")
    H.vcycle(torch.from_numpy(f_o[perm]).cuda(), u)
    assert np.abs(u.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    fn = synth.circle_fourier if kind == "circle" else synth.sphere_harmonics
    _, fs = fn(OH.fine.band.cp[:nb])
    ref = vcycle(OH, np.zeros(nb), fs)[perm]
    errs = []
    for h in (H, H0):
        u32 = torch.zeros(nb, dtype=torch.float32, device="cuda")
        h.vcycle(torch.from_numpy(fs[perm]).float().cuda(), u32)
        errs.append(np.abs(u32.double().cpu().numpy() - ref).max() / np.abs(ref).max())
    assert errs[0] <= 1e-4 and errs[1] <= 1e-4, errs


def test_gmres_coarsest_solve_parity():
    """A coarsest level above the dense limit is solved by restarted GMRES(30)
    on the device (3 restarts, right-preconditioned by omega / diag(A)): one
    V-cycle sphere dx = 1/32 -> 1/16 (26,974 coarse points) equals the oracle's
    cycle with the same GMRES coarsest solve, and the solve converges."""
    torch, pkg = require_cuda()
    g = pkg.Band("sphere", (), 1 / 32)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 16, nu1=3, nu2=3, omega=0.8, residual="plain",
                      coarse_dense_max=1000, coarse_f64_max=1000)
    OH = build_hierarchy(oracle_surface("sphere", ()), 1 / 32, 1 / 16,
                         opts=MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8, residual="plain",
                                        coarse_gmres=3))
    perm = perm_gpu_to_oracle(g, OH.fine.band)
    nb = OH.fine.band.nb
    f_o = synth.random_band_vector(nb, 54)
    ref = vcycle(OH, np.zeros(nb), f_o)[perm]
    u = torch.zeros(nb, dtype=torch.float64, device="cuda")
    H.vcycle(torch.from_numpy(f_o[perm]).cuda(), u)
    err = np.abs(u.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 1e-9, err
    for mode in ("f64", "mixed"):
        _, rep = H.solve(torch.from_numpy(f_o[perm]).cuda(), tol=1e-10, max_iter=60, mode=mode)
        assert rep["converged"], (mode, rep)
