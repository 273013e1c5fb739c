"""Learned smoother on the GPU vs the FP64 oracle network, training and judge."""
import numpy as np
import pytest

from helpers import oracle_surface, perm_gpu_to_oracle, require_cuda
from oracle.band import build_band
from oracle.mlp import MLP, correction, loss_and_grad, neighbour27
from oracle.operators import Operators
import synth

pytestmark = pytest.mark.gpu


def oracle_mlp(p):
    p = np.asarray(p, dtype=np.float64)
    return MLP(p[0:31 * 64].reshape(31, 64), p[2048:2112], p[2112:6208].reshape(64, 64),
               p[6208:6272], p[6272:6336], float(p[6336]))


def _pair(kind="sphere", params=(), dx=1 / 16, seed=3):
    torch, pkg = require_cuda()
    g = pkg.Band(kind, params, dx)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8 if kind == "sphere" else dx * 2, coarse_sweeps=0 if kind == "sphere" else 10)
    sm = pkg.Smoother(seed)
    params_ = sm.get_params()
    params_[2048:2112] += 0.1  # positive biases: more active units
    params_[6208:6272] += 0.1
    sm.set_params(params_)
    H.set_smoother(sm)
    ob = build_band(oracle_surface(kind, params), dx)
    op = Operators(ob)
    perm = perm_gpu_to_oracle(g, ob)
    return torch, pkg, g, H, sm, ob, op, perm, oracle_mlp(params_)


def test_correction_matches_oracle():
    torch, pkg, g, H, sm, ob, op, perm, om = _pair()
    r = synth.random_band_vector(ob.nb, 8).astype(np.float32).astype(np.float64)
    ref, _ = correction(om, ob, r, op.diag_M())
    got = H.smoother_correction(torch.from_numpy(r[perm]).float().cuda()).double().cpu().numpy()
    err = np.abs(got - ref[perm]).max() / np.abs(ref).max()
    assert err < 3e-2, err  # BF16 features and weights, FP32 accumulation


def test_loss_and_gradient_match_oracle():
    torch, pkg, g, H, sm, ob, op, perm, om = _pair()
    r = synth.random_band_vector(ob.nb, 9).astype(np.float32).astype(np.float64)
    L_ref, grads = loss_and_grad(om, ob, op.A_matrix(1.0), r, op.diag_M(), neighbour27(ob))
    L, gp = H.smoother_loss_grad(torch.from_numpy(r[perm]).float().cuda())
    assert abs(L - L_ref) <= 2e-2 * L_ref, (L, L_ref)
    ref = np.zeros(6337)
    ref[0:31 * 64] = grads[0].ravel()
    ref[2048:2112] = grads[1]
    ref[2112:6208] = grads[2].ravel()
    ref[6208:6272] = grads[3]
    ref[6272:6336] = grads[4]
    ref[6336] = grads[5][0]
    assert np.all(gp[31 * 64:2048] == 0)
    for a, b in [(0, 31 * 64), (2048, 2112), (2112, 6208), (6208, 6272), (6272, 6336)]:
        rel = np.linalg.norm(gp[a:b] - ref[a:b]) / np.linalg.norm(ref[a:b])
        assert rel < 6e-2, (a, b, rel)


def test_training_reduces_loss_and_solve_is_judged():
    """Training through the C ABI only (cpm_mlp_train: scaling, schedule and Adam
    inside the library); the loss falls and a learned solve is judged."""
    torch, pkg = require_cuda()
    from paper_1307_4354_gb300 import train as tr
    sets = [tr.residual_fields("ellipsoid", (1.1, 0.9, 0.8), 1 / 32, seed=1),
            tr.residual_fields("torus", (1.0, 0.4), 1 / 32, seed=2)]
    sm = pkg.Smoother(0)
    rep = tr.train(sm, sets, steps=300, lr=2e-3)
    assert rep["steps"] == 300 and rep["fields"] == 8
    assert rep["loss_last"] < 0.8 * rep["loss_first"], rep
    # a learned solve converges to the tolerance, judged against Jacobi
    H, _ = tr.residual_fields("torus", (1.0, 0.35), 1 / 32, seed=5,
                              c_fn=lambda y: 1.0 + 0.5 * np.sin(2 * np.pi * y[:, 2]))
    H.set_smoother(sm)
    u, rep = H.solve(H._f, tol=1e-10, mode="mixed", learned=True, max_iter=80)
    assert rep["converged"], rep
    assert rep["learned_iters"] >= 1 and rep["jacobi_factor"] > 0
    if rep["fallback"]:
        assert rep["learned_worst"] > 1.25 * rep["jacobi_factor"]
    else:
        assert rep["learned_worst"] <= 1.25 * rep["jacobi_factor"]
    u2, rep2 = H.solve(H._f, tol=1e-10, mode="mixed", learned=False, max_iter=80)
    assert rep2["converged"]
    assert torch.abs(u - u2).max().item() <= 1e-8 * torch.abs(u2).max().item()


def test_train_scales_fields_and_matches_train_steps():
    """cpm_mlp_train equals the same schedule of cpm_mlp_train_step calls on
    fields scaled by 1 / max|r| (the scaling and the schedule live in the library)."""
    torch, pkg = require_cuda()
    from paper_1307_4354_gb300 import train as tr
    H, fields = tr.residual_fields("ellipsoid", (1.0, 0.9, 0.7), 1 / 24, seed=3, iters=(0, 1))
    a, b = pkg.Smoother(4), pkg.Smoother(4)
    a.train([(H, r) for r in fields], steps=6, lr=1e-3, lr_final=1e-3)
    H.set_smoother(b)
    for k in range(6):  # 6 steps over 2 fields: 3 consecutive steps per field
        r = fields[k // 3]
        H.smoother_train_step((r / r.abs().max()).float().contiguous(), 1e-3, want_loss=False)
    pa, pb = a.get_params(), b.get_params()
    # The loss gradient's transposed extension accumulates with atomics, so the
    # two runs agree to FP32 rounding only, and Adam's normalised step m/sqrt(v)
    # magnifies that where a gradient component is near zero; a wrong scaling
    # or schedule moves parameters by a whole step (lr = 1e-3).
    assert np.abs(pa - pb).max() <= 1e-5 * np.abs(pb).max()
    with pytest.raises(pkg.capi.CpmError):
        a.train([(H, torch.zeros_like(fields[0]))], steps=1)


def test_save_and_load_round_trip(tmp_path):
    torch, pkg = require_cuda()
    from paper_1307_4354_gb300 import train as tr
    H, fields = tr.residual_fields("torus", (1.0, 0.4), 1 / 32, seed=4, iters=(0, 1))
    sm = pkg.Smoother(2)
    sm.train([(H, r) for r in fields], steps=20)
    path = str(tmp_path / "net.cpmmlp")
    sm.save(path)
    back = pkg.Smoother.load(path)
    assert np.array_equal(back.get_params(), sm.get_params())
    r32 = (fields[1] / fields[1].abs().max()).float().contiguous()
    d1 = H.smoother_correction(r32)
    H.set_smoother(back)
    d2 = H.smoother_correction(r32)
    assert torch.equal(d1, d2)
    # training continues from the saved Adam state: the same next step on both
    # (to rounding: the transposed extension of the gradient sums with atomics)
    p0 = sm.get_params()
    sm.train([(H, fields[0])], steps=1)
    back.train([(H, fields[0])], steps=1)
    p1, p2 = sm.get_params(), back.get_params()
    assert np.abs(p1 - p2).max() <= 1e-3 * np.abs(p1 - p0).max()
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a network")
    with pytest.raises(pkg.capi.CpmError):
        pkg.Smoother.load(str(bad))


def test_trained_network_gains_over_jacobi_on_a_held_out_surface():
    """The network trained on residuals of seeded ellipsoids and tori (dx = 1/64)
    through cpm_mlp_train cuts the residual per outer iteration of the mixed
    solve more than the plain Jacobi V-cycles on a surface it never saw: the
    unit sphere at dx = 1/256 (6.8 M points).  The judge keeps it, and its mean
    and worst reduction factors are below Jacobi's reference factor."""
    torch, pkg = require_cuda()
    from paper_1307_4354_gb300 import train as tr
    sets = tr.training_set(seed=0, spacings=(1 / 64,))
    sm = pkg.Smoother(0)
    rep_t = tr.train(sm, sets, steps=400, lr=2e-3, lr_final=2e-4)
    assert rep_t["loss_last"] < 0.05 * rep_t["loss_first"], rep_t
    del sets
    g = pkg.Band("sphere", (), 1 / 256)
    H = pkg.Hierarchy(g, coarsest_dx=1 / 8, residual="plain")
    _, cp, _ = g.export()
    _, f = synth.sphere_harmonics(cp[: g.nb])
    H.set_smoother(sm)
    _, rep = H.solve(torch.from_numpy(f).cuda(), tol=1e-10, mode="mixed", learned=True,
                     inner_cycles=3, max_iter=60)
    assert rep["converged"] and not rep["fallback"], rep
    assert rep["learned_worst"] < rep["jacobi_factor"], (rep["learned_worst"], rep["jacobi_factor"])
