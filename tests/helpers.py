"""Shared test helpers: run the CUDA path and map its band order to the oracle's."""
import numpy as np
import pytest

from oracle.geometry import circle, dziuk, ellipsoid, sphere, torus


def oracle_surface(kind, params):
    return {"circle": lambda: circle(*params) if params else circle(),
            "sphere": lambda: sphere(*params) if params else sphere(),
            "torus": lambda: torus(*params),
            "ellipsoid": lambda: ellipsoid(*params),
            "dziuk": dziuk}[kind]()


def gpu_keys(ijk, n):
    """Lexicographic grid keys (x fastest) of GPU-exported coordinates."""
    key = ijk[:, -1].astype(np.int64)
    for a in range(ijk.shape[1] - 2, -1, -1):
        key = key * n + ijk[:, a]
    return key


def perm_gpu_to_oracle(gband, oband):
    """idx such that oracle_vector[idx] is in GPU band order (B only)."""
    ijk, _, _ = gband.export()
    keys = gpu_keys(ijk[: gband.nb], oband.n)
    idx = oband.index_in_band(keys)
    assert np.all(idx >= 0)
    return idx


def require_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1307_4354_gb300 as pkg
    pkg.build()
    return torch, pkg
