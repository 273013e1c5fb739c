"""Training of the learned smoother on residuals of the method's own V-cycles.

Residual fields come from mixed-precision solves on seeded surfaces: for a
right-hand side f, the outer residuals r_k = f - A u_k of the first few outer
iterations (the inputs the smoother sees at the start of a V-cycle) are
computed with the library (cpm_solve with a capped iteration count, then
cpm_residual) and cast to FP32.  Each training step is one Adam step of the
library's own forward/backward kernels on one field (cpm_mlp_train_step).
"""
from __future__ import annotations

import math

import numpy as np
import torch

import synth

from .solver import Band, Hierarchy, Smoother


def training_surfaces(seed: int = 0, n_ellipsoids: int = 3, n_tori: int = 2):
    """Seeded ellipsoids (semi-axes U[0.6, 1.2]^3) and tori (R = 1, r U[0.3, 0.45])."""
    rng = np.random.default_rng(seed)
    out = [("ellipsoid", tuple(float(a) for a in rng.uniform(0.6, 1.2, 3))) for _ in range(n_ellipsoids)]
    out += [("torus", (1.0, float(rng.uniform(0.3, 0.45)))) for _ in range(n_tori)]
    return out


def _coarsest(kind, params, dx):
    reach = min(params) ** 2 / max(params) if kind == "ellipsoid" else min(params[1], params[0] - params[1])
    h = dx
    while (math.sqrt(17.0) + 1.0) * 2 * h < reach:
        h *= 2
    return h


def residual_fields(kind, params, dx, seed, iters=(0, 1, 2, 3), c_fn=None):
    """(hierarchy, [FP32 residual fields]) for one surface and one random f."""
    band = Band(kind, params, dx)
    _, cp, _ = band.export()
    cpb = cp[: band.nb]
    c_dev = None
    if c_fn is not None:
        c_dev = torch.from_numpy(c_fn(cpb)).cuda()
    H = Hierarchy(band, coarsest_dx=_coarsest(kind, params, dx), c_device=c_dev)
    y = cpb / np.linalg.norm(cpb, axis=1, keepdims=True)
    _, f = synth.sphere_harmonics(y, seed=seed)
    ft = torch.from_numpy(f).cuda()
    fields = []
    for k in iters:
        if k == 0:
            r = ft.clone()
        else:
            u, _ = H.solve(ft, tol=1e-14, max_iter=k, mode="mixed", inner_cycles=1,
                           raise_on_fail=False)
            r = H.residual(ft, u)
        fields.append((r / r.abs().max()).float().contiguous())
    H._f = ft
    return H, fields


def train(smoother: Smoother, sets, steps: int = 400, lr: float = 2e-3, log_every: int = 0):
    """Adam steps cycling over the (hierarchy, fields) sets; returns the loss history."""
    hist = []
    for H, _ in sets:
        H.set_smoother(smoother)
    per = max(1, steps // max(1, sum(len(f) for _, f in sets)))
    step = 0
    while step < steps:
        for H, fields in sets:
            for r in fields:
                for _ in range(per):
                    if step >= steps:
                        break
                    want = log_every and step % log_every == 0
                    loss = H.smoother_train_step(r, lr, want_loss=bool(want))
                    if want:
                        hist.append((step, loss))
                    step += 1
    return hist


def mean_loss(sets) -> float:
    vals = [H.smoother_loss_grad(r)[0] for H, fields in sets for r in fields]
    return float(np.mean(vals))
