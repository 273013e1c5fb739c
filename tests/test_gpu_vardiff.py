"""Variable diffusion on the GPU (Sec. 4.5.6): -div_S(a grad_S u) + c u = f with
M = E_1 L~ - diag(gamma a)(I - E_3), L~ = sum over axes of D^b diag(A^f a) D^f,
against the oracle's assembled operator, V-cycle and direct solution, and the
closed-form sphere example of the section (u = cos phi, a = cos phi + 1.5)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from helpers import oracle_surface, perm_gpu_to_oracle, require_cuda
from oracle.band import build_band
from oracle.multigrid import MGOptions, build_hierarchy, vcycle
from oracle.operators import VarDiffOperators
import synth

pytestmark = pytest.mark.gpu


def a_sphere(y):
    return synth.sphere_vardiff(y)[1]


def a_wavy(y):
    return 1.5 + 0.5 * np.sin(2 * np.pi * y[:, 2]) * np.cos(np.pi * y[:, 0])


def _hier(pkg, torch, g, a_fn, **kw):
    _, cp, _ = g.export()
    a = torch.from_numpy(a_fn(cp[: g.nb])).cuda()
    return pkg.Hierarchy(g, op_form="vardiff", a_device=a, **kw)


@pytest.mark.parametrize("kind,params,dx,a_fn", [("sphere", (), 1 / 16, a_sphere),
                                                 ("torus", (1.0, 0.4), 1 / 32, a_wavy)])
def test_vardiff_apply_parity(kind, params, dx, a_fn):
    torch, pkg = require_cuda()
    g = pkg.Band(kind, params, dx)
    H = _hier(pkg, torch, g, a_fn, coarsest_dx=dx)
    ob = build_band(oracle_surface(kind, params), dx)
    op = VarDiffOperators(ob, a_fn(ob.cp[: ob.nb]))
    perm = perm_gpu_to_oracle(g, ob)
    u_o = synth.random_band_vector(ob.nb, 61)
    ref = (op.M @ u_o)[perm]
    u = torch.from_numpy(u_o[perm]).cuda()
    got = H.apply(u).cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-13
    got32 = H.apply(u.float()).double().cpu().numpy()
    assert np.abs(got32 - ref).max() / np.abs(ref).max() <= 2e-6


def test_vardiff_vcycle_and_solve():
    torch, pkg = require_cuda()
    dx = 1 / 16
    g = pkg.Band("sphere", (), dx)
    H = _hier(pkg, torch, g, a_sphere, coarsest_dx=1 / 8, nu1=3, nu2=3, omega=0.8, residual="plain")
    OH = build_hierarchy(oracle_surface("sphere", ()), dx, 1 / 8,
                         opts=MGOptions(smoother="jacobi", nu1=3, nu2=3, omega=0.8, residual="plain",
                                        operator="vardiff"), a_fn=a_sphere)
    perm = perm_gpu_to_oracle(g, OH.fine.band)
    nb = OH.fine.band.nb
    f_o = synth.random_band_vector(nb, 62)
    ref = vcycle(OH, np.zeros(nb), f_o)[perm]
    u = torch.zeros(nb, dtype=torch.float64, device="cuda")
    H.vcycle(torch.from_numpy(f_o[perm]).cuda(), u)
    assert np.abs(u.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    _, _, f_s = synth.sphere_vardiff(OH.fine.band.cp[:nb])
    ud = spla.spsolve(OH.fine.ops.A_matrix(1.0).tocsc(), f_s)
    for mode in ("f64", "mixed"):
        us, rep = H.solve(torch.from_numpy(f_s[perm]).cuda(), tol=1e-12, max_iter=80, mode=mode)
        assert rep["converged"], (mode, rep)
        assert np.abs(us.cpu().numpy() - ud[perm]).max() <= 1e-9 * np.abs(ud).max()


def test_vardiff_sphere_second_order():
    """The closed form of Sec. 4.5.6, solved on the GPU to 1e-10 at dx = 1/16,
    1/32, 1/64: relative max error falls at second order."""
    torch, pkg = require_cuda()
    errs = []
    for dx in (1 / 16, 1 / 32, 1 / 64):
        g = pkg.Band("sphere", (), dx)
        H = _hier(pkg, torch, g, a_sphere, coarsest_dx=1 / 8, nu1=3, nu2=3, omega=0.8, residual="plain")
        _, cp, _ = g.export()
        uex, _, f = synth.sphere_vardiff(cp[: g.nb])
        u, rep = H.solve(torch.from_numpy(f).cuda(), tol=1e-10, max_iter=100, mode="mixed",
                         inner_cycles=2)
        assert rep["converged"], (dx, rep)
        errs.append(np.abs(u.cpu().numpy() - uex).max() / np.abs(uex).max())
    order = np.log2(np.asarray(errs[:-1]) / np.asarray(errs[1:]))
    assert np.all((order > 1.8) & (order < 2.3)), (errs, order)
