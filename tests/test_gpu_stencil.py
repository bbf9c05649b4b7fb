"""Parity of the CUDA Wilson stencil (FP64 and mixed) with the oracle."""
import numpy as np
import pytest

from tests._lib import fp16_rounded_links, gpu_module

import synthetic
from oracle import wilson

pytestmark = pytest.mark.gpu

CASES = [
    ((2, 2, 2, 2), "haar", -1),
    ((4, 4, 4, 4), "haar", -1),
    ((4, 4, 4, 4), "smooth", 1),
    ((3, 2, 5, 4), "haar", -1),     # odd extents, V = 120 < one block
    ((4, 4, 4, 6), "smooth", -1),   # 4^3 x 6
    ((6, 4, 2, 7), "haar", 1),      # V = 336: two blocks plus a ragged tail
    ((1, 1, 2, 3), "haar", -1),     # extents of one: forward = backward = self
]


@pytest.fixture(scope="module")
def ss():
    return gpu_module()


@pytest.mark.parametrize("dims,kind,bc", CASES)
def test_fp64_stencil_matches_oracle(ss, dims, kind, bc):
    kappa = 0.13
    U = synthetic.gauge_field(dims, kind, seed=3, eps=0.4)
    psi = synthetic.gaussian_sources(dims, 3, seed=4)
    lat = ss.create_lattice(dims, kappa, bc)
    ss.upload_gauge(lat, U)
    got = ss.apply_H(lat, psi)
    ref = wilson.apply_H(U, psi, kappa, dims, bc)
    # FP64 bound: every output is a sum of at most 8 x 18 + 1 products of
    # O(1) numbers, so 1e-13 of the largest output magnitude is generous.
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


def test_fp64_stencil_8x4_full_size(ss):
    dims = (8, 8, 8, 8)
    U = synthetic.gauge_field(dims, "smooth", seed=2, eps=0.3)
    psi = synthetic.gaussian_sources(dims, 1, seed=5)
    lat = ss.create_lattice(dims, 0.125, -1)
    ss.upload_gauge(lat, U)
    got = ss.apply_H(lat, psi)
    ref = wilson.apply_H(U, psi, 0.125, dims, -1)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_fp64_stencil_device_tensors(ss):
    import torch
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, "haar", seed=8)
    psi = synthetic.gaussian_sources(dims, 2, seed=9)
    lat = ss.create_lattice(dims, 0.12, -1, stream=torch.cuda.current_stream())
    ss.upload_gauge(lat, torch.from_numpy(U).cuda())
    got = ss.apply_H(lat, torch.from_numpy(psi).cuda()).cpu().numpy()
    ref = wilson.apply_H(U, psi, 0.12, dims, -1)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_fp64_stencil_hermitian_on_gpu(ss):
    # <x, A y> = <A x, y> computed entirely from GPU outputs
    dims = (4, 4, 2, 6)
    U = synthetic.gauge_field(dims, "haar", seed=11)
    lat = ss.create_lattice(dims, 0.2, -1)
    ss.upload_gauge(lat, U)
    x = synthetic.gaussian_sources(dims, 1, seed=12)[0]
    y = synthetic.gaussian_sources(dims, 1, seed=13)[0]
    lhs = np.vdot(x, ss.apply_H(lat, y))
    rhs = np.vdot(ss.apply_H(lat, x), y)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("dims,kind,bc", CASES[:5])
def test_mixed_stencil_matches_oracle_on_fp16_links(ss, dims, kind, bc):
    kappa = 0.135
    U = synthetic.gauge_field(dims, kind, seed=3, eps=0.5)
    psi = synthetic.gaussian_sources(dims, 2, seed=4)
    lat = ss.create_lattice(dims, kappa, bc, precision=ss.MIXED)
    ss.upload_gauge(lat, U)
    got = ss.apply_H_mixed(lat, psi)
    # the oracle on exactly the links the kernel uses, in FP64
    ref16 = wilson.apply_H(fp16_rounded_links(U), psi, kappa, dims, bc)
    # FP32 arithmetic: inputs rounded to 2^-24, sums of ~150 terms
    assert np.max(np.abs(got - ref16)) <= 2e-6 * np.max(np.abs(ref16))
    # and the FP16 links perturb the true operator by ~2^-11 relative
    ref = wilson.apply_H(U, psi, kappa, dims, bc)
    assert np.linalg.norm(got - ref) <= 2e-3 * np.linalg.norm(ref)


@pytest.mark.parametrize("dims,nrhs,bc", [((16, 16, 16, 32), 8, -1), ((5, 3, 4, 6), 3, 1), ((33, 1, 2, 2), 1, -1)])
def test_mixed_stencil_all_rhs_kernel(ss, dims, nrhs, bc):
    """The FP32 stencil variants that share each link load among several
    rhs (paired FP32 arithmetic; the rhs-pair variants 4-7 with two rhs in
    the lanes, between layout conversions, 6-7 with the x-y plane staged in
    shared memory): every variant and every rhs against the oracle on the
    FP16-rounded links, at the 16^3 x 32 size of the stencil measurement
    with 8 rhs (8 x-lines of 16 a tile), an odd lattice with an odd rhs
    count (variants 4-7 fall back to 2-3), and a ragged last block (V = 132
    = 4 x 32 + 4, where 6-7 fall back to 4-5)."""
    kappa = 0.135
    U = synthetic.gauge_field(dims, "smooth", seed=5, eps=0.5)
    psi = synthetic.gaussian_sources(dims, nrhs, seed=6)
    lat = ss.create_lattice(dims, kappa, bc, precision=ss.MIXED)
    ss.upload_gauge(lat, U)
    ref16 = wilson.apply_H(fp16_rounded_links(U), psi, kappa, dims, bc)
    try:
        for variant in (0, 1, 2, 3, 4, 5, 6, 7):
            ss.set_stencil_variant(variant)
            got = ss.apply_H_mixed(lat, psi)
            for r in range(nrhs):
                assert np.max(np.abs(got[r] - ref16[r])) <= 2e-6 * np.max(np.abs(ref16[r])), (variant, r)
    finally:
        ss.set_stencil_variant(-1)
    # the autotuner: the first tuned application times every variant and
    # keeps the fastest; the result is the same operator
    got = ss.apply_H_mixed(lat, psi)
    chosen, us = ss.stencil_tuning(lat, nrhs)
    timed = [t for t in us if t > 0]
    tiled = 128 % dims[0] == 0 and dims[1] % (128 // dims[0]) == 0
    assert len(timed) == ((8 if tiled else 6) if nrhs % 2 == 0 else 4)
    assert 0 <= chosen <= 7 and us[chosen] == min(timed)
    assert np.max(np.abs(got - ref16)) <= 2e-6 * np.max(np.abs(ref16))
    with pytest.raises(ss.SsqcdError):
        ss.set_stencil_variant(8)
