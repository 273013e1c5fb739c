"""GPU solves vs the oracle and the closed forms (FP64 and mixed precision)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from helpers import oracle_surface, perm_gpu_to_oracle, require_cuda
from oracle.band import build_band
from oracle.operators import Operators
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["f64", "mixed"])
@pytest.mark.parametrize("kind,params,dx,fn", [
    ("circle", (), 1 / 64, synth.circle_fourier),
    ("sphere", (), 1 / 16, synth.sphere_harmonics),
    ("sphere", (), 1 / 32, synth.sphere_harmonics)])
def test_solve_matches_direct(kind, params, dx, fn, mode):
    """Converged GPU solution equals the sparse direct solution within 1e-9."""
    torch, pkg = require_cuda()
    g = pkg.Band(kind, params, dx)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8)
    ob = build_band(oracle_surface(kind, params), dx)
    op = Operators(ob)
    perm = perm_gpu_to_oracle(g, ob)
    _, f_o = fn(ob.cp[: ob.nb])
    ud = spla.spsolve(op.A_matrix(1.0).tocsc(), f_o)
    u, rep = H.solve(torch.from_numpy(f_o[perm]).cuda(), tol=1e-12, max_iter=80, mode=mode)
    assert rep["converged"], rep
    err = np.abs(u.cpu().numpy() - ud[perm]).max() / np.abs(ud).max()
    assert err <= 1e-9, err


def test_solve_second_order_sphere():
    torch, pkg = require_cuda()
    errs = []
    for dx in [1 / 16, 1 / 32, 1 / 64]:
        g = pkg.Band("sphere", (), dx)
        H = pkg.Hierarchy(g, coarsest_dx=1 / 8)
        _, cp, _ = g.export()
        uex, f = synth.sphere_harmonics(cp[: g.nb])
        u, rep = H.solve(torch.from_numpy(f).cuda(), tol=1e-10, mode="mixed")
        assert rep["converged"]
        errs.append(np.abs(u.cpu().numpy() - uex).max() / np.abs(uex).max())
    slopes = np.log2(np.asarray(errs[:-1]) / np.asarray(errs[1:]))
    assert np.all((slopes > 1.8) & (slopes < 2.4)), slopes


def test_solve_reports_non_convergence():
    torch, pkg = require_cuda()
    g = pkg.Band("sphere", (), 1 / 16)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8)
    _, cp, _ = g.export()
    _, f = synth.sphere_harmonics(cp[: g.nb])
    u, rep = H.solve(torch.from_numpy(f).cuda(), tol=1e-10, max_iter=1, raise_on_fail=False)
    assert rep["status"] == pkg.capi.CPM_ERR_NOT_CONVERGED and not rep["converged"]


def test_graph_and_plain_launches_agree():
    torch, pkg = require_cuda()
    g = pkg.Band("sphere", (), 1 / 32)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8)
    _, cp, _ = g.export()
    _, f = synth.sphere_harmonics(cp[: g.nb])
    ft = torch.from_numpy(f).cuda()
    for mode in ["f64", "mixed"]:
        u1, r1 = H.solve(ft, tol=1e-10, mode=mode, use_graph=True)
        u2, r2 = H.solve(ft, tol=1e-10, mode=mode, use_graph=False)
        assert r1["iters"] == r2["iters"]
        assert torch.equal(u1, u2)


def test_solve_edge_cases_zero_and_non_finite_rhs():
    """f = 0: the solution u = 0 is returned at iteration 0 with a zero residual.
    A NaN or an infinity in f is rejected with CPM_ERR_ARG (the maximum of |f|
    skips NaN, so the sum of squares is checked as well), not run to divergence."""
    torch, pkg = require_cuda()
    g = pkg.Band("circle", (), 1 / 32)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8)
    f0 = torch.zeros(g.nb, dtype=torch.float64, device="cuda")
    for mode in ("f64", "mixed"):
        u, rep = H.solve(f0, tol=1e-10, mode=mode)
        assert rep["converged"] and rep["iters"] == 0 and rep["rel_residual"] == 0.0, rep
        assert float(u.abs().max()) == 0.0
    for bad in (float("nan"), float("inf")):
        f = torch.ones(g.nb, dtype=torch.float64, device="cuda")
        f[g.nb // 2] = bad
        with pytest.raises(pkg.capi.CpmError) as e:
            H.solve(f, tol=1e-10, mode="mixed")
        assert e.value.status == pkg.capi.CPM_ERR_ARG
