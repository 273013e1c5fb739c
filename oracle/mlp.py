"""Learned smoother in FP64: features, the per-point network, loss and gradients.

TEST INFRASTRUCTURE ONLY (see the package header).  The paper has no learned
component; this module is the FP64 reference for the project's learned
smoother, which replaces the first pre-smoothing Jacobi sweep (Eq. 4.1) of the
finest level.

Features of band point i (31 values):
  * r at the 27 nodes x_i + (a, b, c) dx, a, b, c in {-1, 0, 1} (a fastest),
    0 where the node is not in B, divided by s_i = max of their |r| (+1e-300);
  * (x_i - cp(x_i)) / dx (3 values);
  * dx^2 M_ii (1 value).
Network: h1 = relu(W1^T x + b1) (64), h2 = relu(W2^T h1 + b2) (64),
y = w3^T h2 + b3.  Correction: du_i = s_i dx^2 y_i, so du is positively
1-homogeneous in r (du(alpha r) = alpha du(r), alpha > 0).
Loss of one residual field r: L = ||r - A du||^2 / ||r||^2 (the residual left
after the smoothing step), with A = diag(c) - M assembled by ``operators``.
Gradients are the analytic backward pass of that composition.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .band import Band

NFEAT = 31
HIDDEN = 64


def neighbour27(band: Band) -> np.ndarray:
    """(|B|, 27) band indices of the 3^d neighbourhood (a fastest), -1 off the band."""
    ijk = band.coords_of(band.keys)
    cols = []
    for c in (-1, 0, 1):
        for b in (-1, 0, 1):
            for a in (-1, 0, 1):
                nb = ijk.copy()
                nb[:, 0] += a
                nb[:, 1] += b
                nb[:, 2] += c
                cols.append(band.index_in_band(band.key_of(nb)))
    return np.stack(cols, axis=1)


def features(band: Band, r: np.ndarray, diagM: np.ndarray, nbr27: np.ndarray | None = None):
    """(X (|B|, 31), s (|B|,)) of the residual field r on B."""
    if nbr27 is None:
        nbr27 = neighbour27(band)
    R = np.where(nbr27 >= 0, r[np.maximum(nbr27, 0)], 0.0)
    s = np.abs(R).max(axis=1) + 1e-300
    nb = band.nb
    X = np.empty((nb, NFEAT))
    X[:, :27] = R / s[:, None]
    X[:, 27:30] = (band.points(band.keys) - band.cp[:nb]) / band.dx
    X[:, 30] = band.dx * band.dx * diagM
    return X, s


@dataclass
class MLP:
    W1: np.ndarray  # (31, 64)
    b1: np.ndarray  # (64,)
    W2: np.ndarray  # (64, 64)
    b2: np.ndarray  # (64,)
    w3: np.ndarray  # (64,)
    b3: float

    @staticmethod
    def init(seed: int = 0, scale: float = 1.0) -> "MLP":
        rng = np.random.default_rng(seed)
        return MLP(rng.normal(0, scale / np.sqrt(NFEAT), (NFEAT, HIDDEN)), np.zeros(HIDDEN),
                   rng.normal(0, scale / np.sqrt(HIDDEN), (HIDDEN, HIDDEN)), np.zeros(HIDDEN),
                   rng.normal(0, scale / np.sqrt(HIDDEN), HIDDEN), 0.0)

    def params(self):
        return [self.W1, self.b1, self.W2, self.b2, self.w3, np.array([self.b3])]

    def forward(self, X: np.ndarray):
        z1 = X @ self.W1 + self.b1
        h1 = np.maximum(z1, 0.0)
        z2 = h1 @ self.W2 + self.b2
        h2 = np.maximum(z2, 0.0)
        y = h2 @ self.w3 + self.b3
        return y, (X, z1, h1, z2, h2)

    def backward(self, cache, dy: np.ndarray):
        """Gradients of sum_i dy_i y_i with respect to the parameters."""
        X, z1, h1, z2, h2 = cache
        dw3 = h2.T @ dy
        db3 = dy.sum()
        dz2 = np.outer(dy, self.w3) * (z2 > 0)
        dW2 = h1.T @ dz2
        db2 = dz2.sum(axis=0)
        dz1 = (dz2 @ self.W2.T) * (z1 > 0)
        dW1 = X.T @ dz1
        db1 = dz1.sum(axis=0)
        return [dW1, db1, dW2, db2, dw3, np.array([db3])]


def correction(mlp: MLP, band: Band, r: np.ndarray, diagM: np.ndarray, nbr27=None):
    """du = s dx^2 y(X) for the residual field r."""
    X, s = features(band, r, diagM, nbr27)
    y, cache = mlp.forward(X)
    return s * band.dx * band.dx * y, (X, s, y, cache)


def loss_and_grad(mlp: MLP, band: Band, A, r: np.ndarray, diagM: np.ndarray, nbr27=None):
    """L = ||r - A du||^2 / ||r||^2 and its parameter gradients."""
    du, (X, s, y, cache) = correction(mlp, band, r, diagM, nbr27)
    z = r - A @ du
    nr2 = float(r @ r)
    L = float(z @ z) / nr2
    g_du = -2.0 * (A.T @ z) / nr2
    dy = g_du * s * band.dx * band.dx
    return L, mlp.backward(cache, dy)
