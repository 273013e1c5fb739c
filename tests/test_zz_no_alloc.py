"""cpm_residual_norms_noalloc: the residual norms for callers that cannot allocate.

Callers recording work into a CUDA graph, running under a strict latency budget
or drawing every byte from their own memory pool cannot let the library call
cudaMalloc.  The allocation-free entry point keeps its scratch in a fixed
device array inside the library; this test checks, through the C ABI, that two
calls in a row give the same norms as cpm_residual_norms (which uses the
hierarchy's own buffers), and that a level larger than the fixed scratch is
refused.  The file name makes pytest collect it last.
"""
import math

import numpy as np
import pytest

from helpers import require_cuda

pytestmark = pytest.mark.gpu


def test_noalloc_norms_match_existing_entry_point():
    torch, pkg = require_cuda()
    capi = pkg.capi
    band = pkg.Band("sphere", (), 1 / 32)
    H = pkg.Hierarchy(band, coarsest_dx=1 / 8)
    assert band.nb + band.ng <= capi.CPM_NOALLOC_MAX_POINTS
    rng = np.random.default_rng(7)
    f = torch.from_numpy(rng.uniform(-1, 1, band.nb)).cuda()
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    fmax = float(f.abs().max())
    for call in range(2):  # two calls in a row on the shared scratch
        u = torch.from_numpy(rng.uniform(-1, 1, band.nb)).cuda()
        rel_ref, l2_ref = capi.cpm_residual_norms(H.handle, f.data_ptr(), u.data_ptr(), stream)
        norms.fill_(-1.0)
        capi.cpm_residual_norms_noalloc(H.handle, f.data_ptr(), u.data_ptr(), norms.data_ptr(), stream)
        torch.cuda.synchronize()
        rmax, sumsq = norms.cpu().tolist()
        assert abs(rmax / fmax - rel_ref) <= 1e-12 * rel_ref, (call, rmax / fmax, rel_ref)
        assert abs(math.sqrt(sumsq) - l2_ref) <= 1e-12 * l2_ref, (call, math.sqrt(sumsq), l2_ref)


def test_noalloc_rejects_levels_beyond_the_scratch():
    torch, pkg = require_cuda()
    capi = pkg.capi
    band = pkg.Band("sphere", (), 1 / 128)
    assert band.nb + band.ng > capi.CPM_NOALLOC_MAX_POINTS
    H = pkg.Hierarchy(band, coarsest_dx=1 / 64, coarse_sweeps=1)
    f = torch.zeros(band.nb, dtype=torch.float64, device="cuda")
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.CpmError) as e:
        capi.cpm_residual_norms_noalloc(H.handle, f.data_ptr(), f.data_ptr(), norms.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    assert e.value.status == capi.CPM_ERR_ARG
    assert "1048576" in str(e.value)
