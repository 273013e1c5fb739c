"""GPU band build vs the oracle: bit-exact sets, closest points and stencil bases."""
import numpy as np
import pytest

from conftest import load_golden
from helpers import gpu_keys, oracle_surface, require_cuda
from oracle.band import build_band

pytestmark = pytest.mark.gpu

CASES = [("circle", (), 1 / 64), ("circle", (), 1 / 8), ("sphere", (), 1 / 16), ("sphere", (), 1 / 32),
         ("torus", (1.0, 0.4), 1 / 32), ("torus", (1.2, 0.6), 1 / 32),
         ("ellipsoid", (1.1, 0.8, 0.7), 1 / 32), ("ellipsoid", (1.1, 0.8, 0.7), 1 / 16),
         ("torus", (1.0, 0.4), 1 / 16)]


@pytest.mark.parametrize("kind,params,dx", CASES)
def test_band_bit_exact(kind, params, dx):
    torch, pkg = require_cuda()
    g = pkg.Band(kind, params, dx)
    ob = build_band(oracle_surface(kind, params), dx)
    assert (g.nb, g.ng) == (ob.nb, ob.ng)
    ijk, cp, base = g.export()
    kB = gpu_keys(ijk[: g.nb], ob.n)
    kG = gpu_keys(ijk[g.nb:], ob.n)
    assert np.array_equal(np.sort(kB), ob.keys)
    assert np.array_equal(np.sort(kG), ob.ghost_keys)
    idx = ob.index_in_bplus(np.concatenate([kB, kG]))
    assert np.all(idx >= 0)
    # closest points: same formulas, same rounding -> identical bits
    assert np.array_equal(cp, ob.cp[idx])
    from oracle.band import stencil
    obase, _ = stencil(ob.cp[idx], ob.lo, ob.dx, 3)
    assert np.array_equal(base, obase)


def test_band_order_is_brick_morton():
    torch, pkg = require_cuda()
    g = pkg.Band("sphere", (), 1 / 32)
    ijk, _, _ = g.export()
    b = ijk[: g.nb] >> 2

    def morton(v):
        out = np.zeros(v.shape[0], np.int64)
        for bit in range(11):
            for a in range(3):
                out |= ((v[:, a] >> bit) & 1).astype(np.int64) << (3 * bit + a)
        return out

    m = morton(b)
    assert np.all(np.diff(m) >= 0)
    loc = (ijk[: g.nb, 0] & 3) | ((ijk[: g.nb, 1] & 3) << 2) | ((ijk[: g.nb, 2] & 3) << 4)
    same = np.diff(m) == 0
    assert np.all(np.diff(loc)[same] > 0)


@pytest.mark.parametrize("row", load_golden("table41.txt")[1:5])
def test_table41_on_gpu(row):
    """Table 4.1 integers from the GPU band and its exported stencil bases."""
    torch, pkg = require_cuda()
    dx, dofs, nnzL, nnzE, nnzM = row
    g = pkg.Band("sphere", (), dx)
    assert g.nb == int(dofs)
    ijk, _, base = g.export()
    n = int(round(4 / dx)) + 1
    keys = gpu_keys(ijk[: g.nb], n)
    ks = np.sort(keys)
    cnt = g.nb
    for a in range(3):
        for s in (-1, 1):
            nb = ijk[: g.nb].copy()
            nb[:, a] += s
            q = gpu_keys(nb, n)
            pos = np.minimum(np.searchsorted(ks, q), ks.size - 1)
            cnt += int((ks[pos] == q).sum())
    assert cnt == int(nnzL)
    assert 64 * g.nb == int(nnzE)
    own = ijk[: g.nb]
    b = base[: g.nb]
    inside = np.all((own >= b) & (own <= b + 3), axis=1)
    assert 64 * g.nb + int((~inside).sum()) == int(nnzM)


def test_reach_error_is_reported():
    torch, pkg = require_cuda()
    with pytest.raises(pkg.capi.CpmError) as e:
        pkg.Band("sphere", (), 0.2)
    assert e.value.status == pkg.capi.CPM_ERR_REACH


def test_band_at_grid_edge_is_rejected():
    torch, pkg = require_cuda()
    with pytest.raises(pkg.capi.CpmError) as e:
        pkg.Band("torus", (1.2, 0.6), 1 / 16)
    assert e.value.status == pkg.capi.CPM_ERR_ARG


def test_bad_arguments():
    torch, pkg = require_cuda()
    with pytest.raises(pkg.capi.CpmError) as e:
        pkg.Band("torus", (0.4, 1.0), 1 / 16)
    assert e.value.status == pkg.capi.CPM_ERR_ARG
    with pytest.raises(pkg.capi.CpmError):
        pkg.Band("sphere", (), -0.1)
