"""Mixed-precision path: FP32 stencil and shifted CG with FP16 (SSQCD_MIXED)
or FP32 (SSQCD_MIXED_F32LINKS) 12-parameter links, FP64 reliable updates of
the seed residual, FP64 moments and Rayleigh-Ritz.

The reference for the solver is the oracle run on exactly the links the
kernels see (rows 0 and 1 rounded, row 2 rebuilt), in FP64; the eigenpairs
are compared with the dense spectrum of the true operator, with the
accuracy the reduced-precision operator allows stated in each assertion."""
import json
import os

import numpy as np
import pytest

from tests._lib import fp16_rounded_links, gpu_module

import synthetic
from oracle import contour, shifted_cg as oscg, wilson

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "windows.json")
EPS32 = 2.0 ** -24


def fp32_rounded_links(U):
    r01 = U[..., :2, :]
    r01 = r01.real.astype(np.float32).astype(np.float64) + 1j * r01.imag.astype(np.float32).astype(np.float64)
    r2 = np.conj(np.cross(r01[..., 0, :], r01[..., 1, :]))
    return np.concatenate([r01, r2[..., None, :]], axis=-2)


@pytest.fixture(scope="module")
def ss():
    return gpu_module()


@pytest.mark.parametrize("dims,kind,bc", [((4, 4, 4, 4), "haar", -1), ((3, 2, 5, 4), "smooth", 1)])
def test_fp32_link_stencil_matches_oracle(ss, dims, kind, bc):
    U = synthetic.gauge_field(dims, kind, seed=3, eps=0.5)
    psi = synthetic.gaussian_sources(dims, 2, seed=4)
    lat = ss.create_lattice(dims, 0.135, bc, precision=2)
    ss.upload_gauge(lat, U)
    got = ss.apply_H_mixed(lat, psi)
    ref = wilson.apply_H(fp32_rounded_links(U), psi, 0.135, dims, bc)
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision,rounding", [(1, fp16_rounded_links), (2, fp32_rounded_links)])
def test_mixed_shifted_cg_against_oracle_on_rounded_links(ss, precision, rounding):
    reliable = 0
    import torch
    dims, kappa, bc, N, L = (4, 4, 4, 4), 0.13, -1, 8, 2
    U = synthetic.gauge_field(dims, "haar", seed=7)
    v = synthetic.gaussian_sources(dims, L, seed=8)
    z = contour.line_nodes(0.38, 0.02, 0.5, N)
    tol = 1e-6
    lat = ss.create_lattice(dims, kappa, bc, precision=precision, stream=torch.cuda.Stream())
    ss.upload_gauge(lat, U)
    code, y, iters, xi, seed_iters = ss.shifted_cg(lat, z, v, tol=tol, precision=precision,
                                                    reliable_every=reliable)
    assert code == ss.OK
    Ut = rounding(U)
    A = lambda x: wilson.apply_H(Ut, x, kappa, dims, bc)
    for l in range(L):
        ref = oscg.shifted_cg(A, v[l], z, tol=tol)
        vn = np.linalg.norm(v[l])
        for j in range(N):
            r_gpu = v[l] - (z[j] * y[l, j] - A(y[l, j]))
            r_orc = v[l] - (z[j] * ref["y"][j] - A(ref["y"][j]))
            # FP32 recurrences: the true residual exceeds the recursive one by
            # ~ iterations x eps32 x ||A|| x ||y|| (factor 4 as in the FP64 test)
            drift = 4 * int(iters[l, j]) * EPS32 * (1 + 8 * kappa) * np.linalg.norm(y[l, j])
            assert np.linalg.norm(r_gpu) <= tol * vn + drift
            bound = (np.linalg.norm(r_gpu) + np.linalg.norm(r_orc)) / abs(z[j].imag)
            assert np.linalg.norm(y[l, j] - ref["y"][j]) <= bound * (1 + 1e-6)


@pytest.mark.parametrize("precision,relerr_max,res_max", [(1, 1e-6, 1e-3), (2, 1e-6, 2e-4)])
def test_mixed_eigenpairs_accuracy_stated(ss, precision, relerr_max, res_max):
    # The FP16 links perturb A by ~3e-4 and FP32 links by ~1e-7 (relative);
    # the mixed solve then yields eigenvalues to ~1e-8 and residuals ~1e-4 /
    # ~5e-5 on this case -- the bounds asserted are 10-100x looser.
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, "haar", seed=1)
    src = synthetic.gaussian_sources(dims, 3, seed=100)
    lat = ss.create_lattice(dims, 0.13, -1, precision=precision)
    ss.upload_gauge(lat, U)
    res = ss.ss_solve(lat, (0.374, 0.3930), 16, 8, src, beta=0.3, nprime=14, tol=1e-7)
    assert res.status == ss.OK, res.error
    ev, vec, rs, st = ss.ss_eigpairs(res)
    lam = np.array(json.load(open(GOLDEN))["haar_4x4x4x4_k0.13_s1"]["lowest_abs"])
    exact = np.sort(lam[(lam >= 0.374) & (lam <= 0.3930)])
    assert len(ev) == len(exact) == 8
    assert np.max(np.abs(ev - exact) / exact) <= relerr_max
    assert np.max(rs) <= res_max
    # residuals reported by the library are those of the true FP64 operator
    r = wilson.apply_H(U, vec[0], 0.13, dims, -1) - ev[0] * vec[0]
    assert abs(np.linalg.norm(r) - rs[0]) <= 1e-10 + 1e-6 * rs[0]


@pytest.mark.parametrize("precision", [1, 2])
def test_reliable_updates_keep_the_solve_valid(ss, precision):
    # FP64 reliable updates of the seed residual (while it is above the
    # reduced-precision operator's error) leave the eigenpairs at the stated
    # accuracy and are counted.
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, "haar", seed=1)
    src = synthetic.gaussian_sources(dims, 3, seed=100)
    lat = ss.create_lattice(dims, 0.13, -1, precision=precision)
    ss.upload_gauge(lat, U)
    res = ss.ss_solve(lat, (0.374, 0.3930), 16, 8, src, beta=0.3, nprime=14, tol=1e-7, reliable_every=16)
    assert res.status == ss.OK, res.error
    ev, _, rs, st = ss.ss_eigpairs(res, want_vectors=False)
    lam = np.array(json.load(open(GOLDEN))["haar_4x4x4x4_k0.13_s1"]["lowest_abs"])
    exact = np.sort(lam[(lam >= 0.374) & (lam <= 0.3930)])
    assert len(ev) == len(exact) == 8
    assert np.max(np.abs(ev - exact) / exact) <= 1e-6
    assert st["reliable_updates"] >= 1


def test_fp64_seed_fp32_shift_vectors_against_oracle(ss):
    # SSQCD_FP64_SHIFT32 keeps the operator and the seed recurrence in FP64
    # and stores y and p-hat in FP32: the true residual then exceeds tol by at
    # most the FP32 rounding of the updates, ~ iterations x eps32 x ||zI - A|| x ||y||.
    import torch
    dims, kappa, bc, N, L = (4, 4, 4, 4), 0.13, -1, 8, 2
    U = synthetic.gauge_field(dims, "haar", seed=7)
    v = synthetic.gaussian_sources(dims, L, seed=8)
    z = contour.line_nodes(0.38, 0.02, 0.5, N)
    tol = 1e-6
    lat = ss.create_lattice(dims, kappa, bc, precision=ss.FP64, stream=torch.cuda.Stream())
    ss.upload_gauge(lat, U)
    code, y, iters, xi, seed_iters = ss.shifted_cg(lat, z, v, tol=tol, precision=ss.FP64_SHIFT32)
    assert code == ss.OK
    code64, y64, iters64, _, seed64 = ss.shifted_cg(lat, z, v, tol=tol, precision=ss.FP64)
    assert code64 == ss.OK
    # the seed recurrence is the FP64 one: identical stopping iterations
    assert seed_iters == seed64
    assert np.array_equal(iters, iters64)
    A = lambda x: wilson.apply_H(U, x, kappa, dims, bc)
    for l in range(L):
        ref = oscg.shifted_cg(A, v[l], z, tol=tol)
        vn = np.linalg.norm(v[l])
        for j in range(N):
            r_gpu = v[l] - (z[j] * y[l, j] - A(y[l, j]))
            r_orc = v[l] - (z[j] * ref["y"][j] - A(ref["y"][j]))
            drift = 4 * int(iters[l, j]) * EPS32 * (abs(z[j]) + 1 + 8 * kappa) * np.linalg.norm(y[l, j])
            assert np.linalg.norm(r_gpu) <= tol * vn + drift
            bound = (np.linalg.norm(r_gpu) + np.linalg.norm(r_orc)) / abs(z[j].imag)
            assert np.linalg.norm(y[l, j] - ref["y"][j]) <= bound * (1 + 1e-6)
