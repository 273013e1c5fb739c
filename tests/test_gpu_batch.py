"""Batched solves (cpm_build_batch / cpm_solve_batch) against single solves."""
import os

import numpy as np
import pytest

from helpers import require_cuda
import synth

pytestmark = pytest.mark.gpu

# uneven bands: a sphere, an ellipsoid and a torus, each with its own coarsest
# solve (FP64 inverse, FP64 inverse, FP32 inverse with refinement)
SURFACES = [("sphere", (), 1 / 32, 1 / 8), ("ellipsoid", (1.0, 0.9, 0.8), 1 / 24, 1 / 12),
            ("torus", (1.0, 0.4), 1 / 32, 1 / 16)]


def _setup(pkg, n_rhs):
    import torch
    hs, fs = [], []
    for i, (kind, params, dx, cdx) in enumerate(SURFACES):
        g = pkg.Band(kind, params, dx)
        H = pkg.Hierarchy(g, coarsest_dx=cdx)
        _, cp, _ = g.export()
        for k in range(n_rhs):
            fs.append(torch.from_numpy(synth.harmonic_field(cp[: g.nb], seed=10 * i + k)).cuda())
        hs.append(H)
    return hs, fs


@pytest.mark.parametrize("mode", ["mixed", "f64"])
def test_batch_equals_single_solves(mode, tmp_path):
    """Every system's result is bit-identical to cpm_solve's on the same input."""
    torch, pkg = require_cuda()
    n_rhs = 2
    hs, fs = _setup(pkg, n_rhs)
    B = pkg.Batch(hs, n_rhs, tune_cache=str(tmp_path / "tune.txt"))
    us, reps = B.solve(fs, tol=1e-10, mode=mode, inner_cycles=2 if mode == "mixed" else 1)
    assert len(us) == len(fs) == len(SURFACES) * n_rhs
    for s, (u, f, rep) in enumerate(zip(us, fs, reps)):
        H = hs[s // n_rhs]
        u1, r1 = H.solve(f, tol=1e-10, mode=mode, inner_cycles=2 if mode == "mixed" else 1)
        assert rep["converged"] and r1["converged"]
        assert rep["iters"] == r1["iters"], (s, rep["iters"], r1["iters"])
        assert np.allclose(rep["history"], r1["history"], rtol=0, atol=0)
        assert torch.equal(u, u1), s
        rel, _ = H.residual_norms(f, u)
        assert rel <= 1e-10
    K, ms = B.info()
    assert K in (1, 2)
    assert sum(1 for v in ms if v > 0) == 2  # K = 1, 2 (three lockstep groups)
    B.close()


def test_batch_group_larger_than_one_coarse_pass():
    """Five right-hand sides of one hierarchy: one lockstep group whose coarse
    solve takes two passes over the inverse (4 + 1 vectors); every result is
    still bit-identical to its own cpm_solve."""
    torch, pkg = require_cuda()
    g = pkg.Band("sphere", (), 1 / 32)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8)
    _, cp, _ = g.export()
    fs = [torch.from_numpy(f).cuda() for f in synth.harmonic_fields(cp[: g.nb], range(5))]
    B = pkg.Batch([H], 5)
    for mode in ("mixed", "f64"):
        us, reps = B.solve(fs, tol=1e-10, mode=mode)
        for u, f, rep in zip(us, fs, reps):
            u1, r1 = H.solve(f, tol=1e-10, mode=mode)
            assert rep["converged"] and rep["iters"] == r1["iters"]
            assert torch.equal(u, u1)
    assert B.info()[0] == 1
    B.close()


def test_tune_cache_is_reused(tmp_path):
    torch, pkg = require_cuda()
    hs, fs = _setup(pkg, 1)
    cache = str(tmp_path / "tune.txt")
    B1 = pkg.Batch(hs, 1, tune_cache=cache)
    u1, _ = B1.solve(fs, mode="mixed")
    K1, _ = B1.info()
    assert os.path.exists(cache)
    B2 = pkg.Batch(hs, 1, tune_cache=cache)
    u2, _ = B2.solve(fs, mode="mixed")
    K2, ms2 = B2.info()
    assert K2 == K1 and all(v == 0 for v in ms2)  # no tuning iterations
    for a, b in zip(u1, u2):
        assert torch.equal(a, b)  # the concurrency does not change the arithmetic
    B1.close()
    B2.close()


def test_batch_reports_non_convergence_and_rejects_bad_input():
    torch, pkg = require_cuda()
    hs, fs = _setup(pkg, 1)
    B = pkg.Batch(hs, 1)
    us, reps = B.solve(fs, max_iter=1, raise_on_fail=False)
    assert all(r["status"] == pkg.capi.CPM_ERR_NOT_CONVERGED for r in reps)
    assert all(r["iters"] == 1 and not r["converged"] for r in reps)
    with pytest.raises(ValueError):
        B.solve(fs[:-1])
    o = pkg.capi.cpm_solve_opts()
    o.tol, o.max_iter, o.mode, o.learned = 1e-10, 10, pkg.capi.CPM_SOLVE_MIXED, 1
    ptrs = [f.data_ptr() for f in fs]
    with pytest.raises(pkg.capi.CpmError) as e:
        pkg.capi.cpm_solve_batch(B.handle, ptrs, ptrs, o, 0, raise_on_fail=False)
    assert e.value.status == pkg.capi.CPM_ERR_ARG
    B.close()
