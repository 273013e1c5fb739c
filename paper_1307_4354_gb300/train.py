"""Training data for the learned smoother: residuals of the method's own V-cycles.

For a right-hand side f on a seeded surface, the outer residuals
r_k = f - A u_k of the first few outer iterations of a mixed-precision solve
(the inputs the smoother sees at the start of a V-cycle) are produced with the
library (cpm_solve with a capped iteration count, then cpm_residual).  The
fields stay FP64 on the device; ``Smoother.train`` (cpm_mlp_train) scales and
casts them and runs the Adam schedule inside the library.  Nothing here
computes: it only chooses surfaces and calls the C ABI.
"""
from __future__ import annotations

import math

import numpy as np
import torch

import synth

from .solver import Band, Hierarchy


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
    """(hierarchy, [FP64 residual fields on the device]) for one surface and one random f."""
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
        fields.append(r)
    H._f = ft
    return H, fields


def training_set(seed: int = 0, spacings=(1 / 64, 1 / 96, 1 / 128), n_ellipsoids: int = 3,
                 n_tori: int = 2, iters=(0, 1, 2, 3)):
    """Residual fields of seeded ellipsoids and tori, each at a spacing drawn in turn
    from `spacings` (the training spacings of the learned-smoother workload)."""
    sets = []
    for i, (kind, prm) in enumerate(training_surfaces(seed, n_ellipsoids, n_tori)):
        sets.append(residual_fields(kind, prm, spacings[i % len(spacings)], seed=seed + i, iters=iters))
    return sets


def train(smoother, sets, steps: int = 400, lr: float = 2e-3, lr_final: float = 0.0) -> dict:
    """cpm_mlp_train over every field of every (hierarchy, fields) set."""
    pairs = [(H, r) for H, fields in sets for r in fields]
    return smoother.train(pairs, steps=steps, lr=lr, lr_final=lr_final)
