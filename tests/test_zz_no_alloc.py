"""The allocation-free moments entry point (ssqcd_moments_noalloc).

Some callers cannot allocate device memory when they need the moments
(programs that give all device memory to their own pool or arena up front,
loops with a fixed memory budget); this entry point keeps its scratch in a
fixed device array.  The test calls it
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


def test_moments_noalloc_allocates_no_device_memory():
    """After one warm-up call (module load, torch's cached output block), a
    call leaves the device's free memory unchanged: the library allocated
    nothing."""
    import torch
    ss = gpu_module()
    dims = (4, 4, 2, 6)
    y, w, zeta = _case(3, dims, 16, 8, 2, 0.3)
    yd = torch.from_numpy(y).cuda()
    s = ss.moments_noalloc(w, zeta, yd, 8)
    torch.cuda.synchronize()
    del s
    free0, _ = torch.cuda.mem_get_info()
    s = ss.moments_noalloc(w, zeta, yd, 8)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert tuple(s.shape) == (2, 8) + y.shape[2:]


def test_moments_noalloc_rejects_mismatched_shapes():
    import torch
    ss = gpu_module()
    y = torch.zeros((2, 16, 24), dtype=torch.complex128, device="cuda")
    w = np.ones(8, dtype=complex)
    with pytest.raises(ValueError):
        ss.moments_noalloc(w, w, y, 4)            # y has 16 shifts, w 8
    with pytest.raises(ValueError):
        ss.moments_noalloc(np.ones(16, dtype=complex), w, y, 4)   # zeta shorter than w
