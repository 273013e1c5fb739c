"""GPU operators vs the oracle: cpm_apply, smoothing, V-cycle (FP64 and FP32)."""
import numpy as np
import pytest

from helpers import oracle_surface, perm_gpu_to_oracle, require_cuda
from oracle.band import build_band
from oracle.multigrid import MGOptions, build_hierarchy, smooth, vcycle
from oracle.operators import Operators
import synth

pytestmark = pytest.mark.gpu

APPLY_CASES = [("circle", (), 1 / 64), ("sphere", (), 1 / 16), ("sphere", (), 1 / 32),
               ("torus", (1.0, 0.4), 1 / 32), ("ellipsoid", (1.1, 0.8, 0.7), 1 / 32)]


@pytest.mark.parametrize("kind,params,dx", APPLY_CASES)
def test_apply_f64_parity(kind, params, dx):
    """cpm_apply FP64 within 1e-13 of the oracle's M u (relative max-norm)."""
    torch, pkg = require_cuda()
    g = pkg.Band(kind, params, dx)
    H = pkg.Hierarchy(g)
    ob = build_band(oracle_surface(kind, params), dx)
    op = Operators(ob)
    perm = perm_gpu_to_oracle(g, ob)
    u_o = synth.random_band_vector(ob.nb, 11)
    ref = op.apply_M(u_o)[perm]
    u = torch.from_numpy(u_o[perm]).cuda()
    got = H.apply(u).cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= 1e-13, err
    # FP32 apply: same operator within single-precision rounding
    got32 = H.apply(u.float()).double().cpu().numpy()
    err32 = np.abs(got32 - ref).max() / np.abs(ref).max()
    assert err32 <= 2e-6, err32


def test_apply_smooth_field_relative_to_operator_norm():
    """Smooth u (cancellation): compare against ||M||_inf ||u||_inf."""
    torch, pkg = require_cuda()
    g = pkg.Band("sphere", (), 1 / 32)
    H = pkg.Hierarchy(g)
    ob = build_band(oracle_surface("sphere", ()), 1 / 32)
    op = Operators(ob)
    perm = perm_gpu_to_oracle(g, ob)
    u_o, _ = synth.sphere_harmonics(ob.cp[: ob.nb])
    ref = op.apply_M(u_o)[perm]
    got = H.apply(torch.from_numpy(u_o[perm]).cuda()).cpu().numpy()
    normM = np.abs(op.M).sum(axis=1).max()
    assert np.abs(got - ref).max() <= 1e-14 * normM * np.abs(u_o).max()


def _hier_pair(kind, params, dx, smoother="jacobi", nu=3, omega=0.8, residual="extended",
               coarsest=1 / 8, coarse_sweeps=0):
    torch, pkg = require_cuda()
    g = pkg.Band(kind, params, dx)
    H = pkg.Hierarchy(g, coarsest_dx=coarsest, nu1=nu, nu2=nu, omega=omega, smoother=smoother,
                      residual=residual, coarse_sweeps=coarse_sweeps)
    OH = build_hierarchy(oracle_surface(kind, params), dx, coarsest,
                         opts=MGOptions(smoother=smoother, nu1=nu, nu2=nu, omega=omega,
                                        residual=residual, coarse_sweeps=coarse_sweeps))
    perm = perm_gpu_to_oracle(g, OH.fine.band)
    return torch, pkg, g, H, OH, perm


@pytest.mark.parametrize("smoother", ["jacobi", "rm"])
def test_smooth_parity(smoother):
    torch, pkg, g, H, OH, perm = _hier_pair("sphere", (), 1 / 32, smoother)
    nb = OH.fine.band.nb
    f_o = synth.random_band_vector(nb, 1)
    u_o = synth.random_band_vector(nb, 2)
    ref = u_o.copy()
    for _ in range(2):
        ref = smooth(OH, 0, ref, f_o)
    u = torch.from_numpy(u_o[perm]).cuda()
    H.smooth(torch.from_numpy(f_o[perm]).cuda(), u, sweeps=2)
    err = np.abs(u.cpu().numpy() - ref[perm]).max() / np.abs(ref).max()
    assert err <= 1e-12, err


@pytest.mark.parametrize("residual", ["extended", "plain"])
@pytest.mark.parametrize("kind,params,dx", [("circle", (), 1 / 64), ("sphere", (), 1 / 32)])
def test_vcycle_parity(kind, params, dx, residual):
    """One FP64 V-cycle (Algorithm 4.1) from zero equals the oracle's."""
    torch, pkg, g, H, OH, perm = _hier_pair(kind, params, dx, residual=residual)
    assert H.n_levels == len(OH.levels)
    nb = OH.fine.band.nb
    f_o = synth.random_band_vector(nb, 3)
    ref = vcycle(OH, np.zeros(nb), f_o)[perm]
    u = torch.zeros(nb, dtype=torch.float64, device="cuda")
    H.vcycle(torch.from_numpy(f_o[perm]).cuda(), u)
    err = np.abs(u.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 1e-10, err
    # FP32 V-cycle: same cycle in single precision
    u32 = torch.zeros(nb, dtype=torch.float32, device="cuda")
    H.vcycle(torch.from_numpy(f_o[perm]).float().cuda(), u32)
    err32 = np.abs(u32.double().cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err32 <= 1e-3, err32


def test_vcycle_parity_rm_and_coarse_sweeps():
    """Ruuth-Merriman V-cycle, and a coarsest level solved by Jacobi sweeps."""
    torch, pkg, g, H, OH, perm = _hier_pair("sphere", (), 1 / 32, smoother="rm", omega=1.0)
    nb = OH.fine.band.nb
    f_o = synth.random_band_vector(nb, 4)
    ref = vcycle(OH, np.zeros(nb), f_o)[perm]
    u = torch.zeros(nb, dtype=torch.float64, device="cuda")
    H.vcycle(torch.from_numpy(f_o[perm]).cuda(), u)
    assert np.abs(u.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    torch, pkg, g, H, OH, perm = _hier_pair("torus", (1.0, 0.4), 1 / 32, coarsest=1 / 16,
                                            coarse_sweeps=20)
    nb = OH.fine.band.nb
    ref = vcycle(OH, np.zeros(nb), synth.random_band_vector(nb, 5))[perm]
    u = torch.zeros(nb, dtype=torch.float64, device="cuda")
    H.vcycle(torch.from_numpy(synth.random_band_vector(nb, 5)[perm]).cuda(), u)
    assert np.abs(u.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()


def test_vcycle_parity_large_coarsest_level():
    """Torus: the coarsest level (dx = 1/16, ~33k points) is solved with the FP32
    explicit inverse and two FP64 refinement steps; the V-cycle still matches the
    oracle's (sparse LU coarsest solve)."""
    torch, pkg, g, H, OH, perm = _hier_pair("torus", (1.0, 0.4), 1 / 32, coarsest=1 / 16)
    nb = OH.fine.band.nb
    assert OH.levels[-1].band.nb > 16384
    f_o = synth.random_band_vector(nb, 12)
    ref = vcycle(OH, np.zeros(nb), f_o)[perm]
    u = torch.zeros(nb, dtype=torch.float64, device="cuda")
    H.vcycle(torch.from_numpy(f_o[perm]).cuda(), u)
    assert np.abs(u.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()


def test_vcycle_parity_relaxed_coarse_level():
    """Ellipsoid (1.05, 0.9, 0.8), reach 0.61: the level dx = 1/8 has a band
    within the reach (sqrt(17)/8 = 0.52) but not its ghost ring margin
    ((sqrt(17)+1)/8 = 0.64).  It builds (cp is defined on all of B+), the GPU
    V-cycle matches the oracle's on it, and auto coarsening takes it only when
    the coarsest strict level is too large for the dense solve."""
    torch, pkg, g, H, OH, perm = _hier_pair("ellipsoid", (1.05, 0.9, 0.8), 1 / 16, coarsest=1 / 8)
    nb = OH.fine.band.nb
    assert H.n_levels == 2 and H.level_size(1) == OH.levels[1].band.nb
    f_o = synth.random_band_vector(nb, 21)
    ref = vcycle(OH, np.zeros(nb), f_o)[perm]
    u = torch.zeros(nb, dtype=torch.float64, device="cuda")
    H.vcycle(torch.from_numpy(f_o[perm]).cuda(), u)
    assert np.abs(u.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    _, rep = H.solve(torch.from_numpy(f_o[perm]).cuda(), tol=1e-10, mode="mixed")
    assert rep["converged"] and rep["iters"] <= 12, rep
    # auto: the strict rule stops at dx = 1/16; with a dense limit below |B(1/16)|
    # the relaxed level dx = 1/8 is added
    Ha = pkg.Hierarchy(g, coarse_dense_max=8192)
    assert Ha.n_levels == 2 and Ha.level_size(1) == H.level_size(1)
    Hs = pkg.Hierarchy(g)
    assert Hs.n_levels == 1
    # an explicit spacing whose band leaves the reach is refused
    with pytest.raises(pkg.capi.CpmError) as e:
        pkg.Hierarchy(g, coarsest_dx=1 / 4)
    assert e.value.status == pkg.capi.CPM_ERR_REACH


def test_extension_variants_agree_bit_for_bit():
    """The three FP32 extension decompositions (one thread per point; persistent
    pipelined tiles; chunks of points with one base) evaluate the same
    contraction in the same order: identical w = E u over B and B+, identical
    V-cycles; the per-level choice made by timing is one of them."""
    torch, pkg = require_cuda()
    g = pkg.Band("sphere", (), 1 / 32)
    Hs = [pkg.Hierarchy(g, coarsest_dx=1 / 8, ext_variant=v) for v in range(3)]
    Ha = pkg.Hierarchy(g, coarsest_dx=1 / 8)
    for l in range(Ha.n_levels):
        v, ms = Ha.ext_tuning(l)
        assert v in (0, 1, 2) and all(m > 0 for m in ms), (l, v, ms)
    u = torch.from_numpy(synth.random_band_vector(g.nb, 81)).float().cuda()
    outs = [[H.extend(u, with_ghost=gh) for H in Hs] for gh in (False, True)]
    for o in outs:
        assert torch.equal(o[0], o[1]) and torch.equal(o[0], o[2])
    f = torch.from_numpy(synth.random_band_vector(g.nb, 82)).float().cuda()
    us = []
    for H in Hs:
        x = torch.zeros_like(f)
        H.vcycle(f, x)
        us.append(x)
    assert torch.equal(us[0], us[1]) and torch.equal(us[0], us[2])
