"""The allocation-free moments entry point (ssqcd_moments_noalloc).

Some callers cannot allocate device memory when they need the moments
(stream capture, caller-owned memory pools, allocation-free loops); this
entry point keeps its scratch in a fixed device array.  The test calls it
through the C ABI twice in a row, with different inputs, and checks each
result against the allocating ssqcd_moments.  It lives in a file of its own
that pytest collects last.
"""
import numpy as np
import pytest

from tests._lib import gpu_module

import synthetic
from oracle import contour

pytestmark = pytest.mark.gpu


def _case(seed, dims, N, M, L, beta):
    g = synthetic.rng(seed)
    V = synthetic.volume(dims)
    y = g.standard_normal((L, N, V, 4, 3)) + 1j * g.standard_normal((L, N, V, 4, 3))
    z = contour.line_nodes(0.1, 0.05, beta, N)
    zeta = contour.normalise(z, 0.1, 0.05)
    w = contour.weights_closed_form(zeta)
    return y, w, zeta


def test_moments_noalloc_matches_allocating_entry_point_twice():
    import torch
    ss = gpu_module()
    dims = (4, 4, 2, 6)
    lat = ss.create_lattice(dims, 0.1, -1)
    for seed, N, M, L, beta in [(1, 16, 8, 3, 0.3), (2, 32, 16, 2, 0.6)]:
        y, w, zeta = _case(seed, dims, N, M, L, beta)
        ref = ss.moments(lat, w, zeta, y, M)
        yd = torch.from_numpy(y).cuda()
        got = ss.moments_noalloc(w, zeta, yd, M).cpu().numpy()
        torch.cuda.synchronize()
        # same tolerance as the moments parity test: FP64 sums of N terms
        scale = np.sum(np.abs(w)[:, None] * np.abs(zeta)[:, None] ** np.arange(M)[None, :], axis=0)
        for k in range(M):
            assert np.max(np.abs(got[:, k] - ref[:, k])) <= 1e-14 * scale[k] * np.max(np.abs(y)) * 8


def test_moments_noalloc_rejects_oversize():
    import torch
    ss = gpu_module()
    y = torch.zeros((1, 128, 24), dtype=torch.complex128, device="cuda")
    w = np.ones(128, dtype=complex)
    with pytest.raises(ss.SsqcdError) as e:
        ss.moments_noalloc(w, w, y, 64)   # 128 x 64 > 4096
    assert e.value.code == ss.ERR_ARG
