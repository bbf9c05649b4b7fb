"""Float-float solve precisions (two FP32 words per real, 48-bit significand,
arithmetic on the FP32 pipes).

SSQCD_FP64_DFSHIFT: FP64 operator and seed recurrence, shift vectors y and
p-hat in float-float.  The seed recurrence is the FP64 one (the power-of-two
rescaling at the FP32 threshold is exact), so the stopping iterations equal
those of the FP64 path bit for bit; the solutions differ from the FP64 ones
by the float-float rounding of the updates, ~ iterations x 2^-48 relative.

SSQCD_DF: links, stencil, seed and shift vectors all in float-float.  The
operator carries a ~1e-14 relative error, so the seed recurrence is a
(slightly) different CG run and the stopping iterations may differ from the
FP64 ones by a few per cent.

Both meet the FP64 bars on the eigenpairs: eigenvalues 1e-10 relative,
residuals 1e-8."""
import json
import os

import numpy as np
import pytest

from tests._lib import gpu_module

import bench
import synthetic
from oracle import contour, shifted_cg as oscg, wilson

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "windows.json")
EPS_FF = 2.0 ** -48


@pytest.fixture(scope="module")
def ss():
    return gpu_module()


@pytest.mark.parametrize("dims,kind,kappa,N,L", [((4, 4, 4, 4), "haar", 0.13, 8, 2),
                                                  ((3, 2, 5, 4), "smooth", 0.12, 6, 3)])
def test_dfshift_shifted_cg_against_oracle(ss, dims, kind, kappa, N, L):
    import torch
    bc = -1
    U = synthetic.gauge_field(dims, kind, seed=7, eps=0.4)
    v = synthetic.gaussian_sources(dims, L, seed=8)
    z = contour.line_nodes(0.38, 0.02, 0.5, N)
    tol = 1e-11
    lat = ss.create_lattice(dims, kappa, bc, stream=torch.cuda.Stream())
    ss.upload_gauge(lat, U)
    code, y, iters, xi, seed_iters = ss.shifted_cg(lat, z, v, tol=tol, precision=ss.FP64_DFSHIFT)
    assert code == ss.OK
    code64, y64, iters64, xi64, seed64 = ss.shifted_cg(lat, z, v, tol=tol, precision=ss.FP64)
    assert code64 == ss.OK
    assert seed_iters == seed64
    assert np.array_equal(iters, iters64)
    assert np.array_equal(xi, xi64)
    A = lambda x: wilson.apply_H(U, x, kappa, dims, bc)
    for l in range(L):
        ref = oscg.shifted_cg(A, v[l], z, tol=tol)
        vn = np.linalg.norm(v[l])
        for j in range(N):
            yn = np.linalg.norm(y[l, j])
            # float-float rounding of every update: ~ iterations x 2^-48 x ||y||
            assert np.linalg.norm(y[l, j] - y64[l, j]) <= 8 * int(iters[l, j]) * EPS_FF * yn
            r_gpu = v[l] - (z[j] * y[l, j] - A(y[l, j]))
            r_orc = v[l] - (z[j] * ref["y"][j] - A(ref["y"][j]))
            drift = 8 * int(iters[l, j]) * EPS_FF * (abs(z[j]) + 1 + 8 * kappa) * yn
            assert np.linalg.norm(r_gpu) <= tol * vn + drift
            bound = (np.linalg.norm(r_gpu) + np.linalg.norm(r_orc)) / abs(z[j].imag)
            assert np.linalg.norm(y[l, j] - ref["y"][j]) <= bound * (1 + 1e-6)


def test_dfshift_zero_source_stays_zero(ss):
    dims = (2, 2, 2, 4)
    U = synthetic.gauge_field(dims, "haar", seed=3)
    v = synthetic.gaussian_sources(dims, 2, seed=4)
    v[1] = 0.0
    z = contour.line_nodes(0.4, 0.05, 0.5, 4)
    lat = ss.create_lattice(dims, 0.12, 1)
    ss.upload_gauge(lat, U)
    code, y, iters, xi, _ = ss.shifted_cg(lat, z, v, tol=1e-10, precision=ss.FP64_DFSHIFT)
    assert code == ss.OK
    assert np.all(y[1] == 0) and np.all(iters[1] == 0)
    assert np.all(iters[0] > 0)


def test_dfshift_eigenpairs_config1(ss):
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, "haar", seed=1)
    src = synthetic.gaussian_sources(dims, 3, seed=100)
    lat = ss.create_lattice(dims, 0.13, -1, precision=ss.FP64_DFSHIFT)
    ss.upload_gauge(lat, U)
    res = ss.ss_solve(lat, (0.374, 0.3930), 16, 8, src, beta=0.3, nprime=14)
    assert res.status == ss.OK, res.error
    ev, vec, rs, st = ss.ss_eigpairs(res)
    lam = np.array(json.load(open(GOLDEN))["haar_4x4x4x4_k0.13_s1"]["lowest_abs"])
    exact = np.sort(lam[(lam >= 0.374) & (lam <= 0.3930)])
    assert len(ev) == len(exact) == 8
    assert np.max(np.abs(ev - exact) / exact) <= 1e-10
    assert np.max(rs) <= 1e-8
    r = wilson.apply_H(U, vec[3], 0.13, dims, -1) - ev[3] * vec[3]
    assert abs(np.linalg.norm(r) - rs[3]) <= 1e-12 + 1e-6 * rs[3]


def test_dfshift_eigenpairs_full_size(ss):
    # the 8^4 workload (N = 32, L = 4, M = 8, beta 0.6) on a side stream with
    # graph replay, as the benchmark runs it
    import torch
    w = bench.CONFIG2
    U, src = bench.make_inputs(0, bench.CONFIG2)
    lat = ss.create_lattice(w["dims"], w["kappa"], w["bc_t"], precision=ss.FP64_DFSHIFT,
                            stream=torch.cuda.Stream())
    ss.upload_gauge(lat, U)
    res = ss.ss_solve(lat, w["interval"], w["N"], w["M"], src, beta=w["beta"], nprime=w["nprime"], tol=w["tol"])
    assert res.status == ss.OK, res.error
    ev, vec, rs, st = ss.ss_eigpairs(res)
    ref = np.array(json.load(open(GOLDEN))["smooth_8x8x8x8_e0.3_k0.125_s2"]["lowest_abs"])
    ref = np.sort(ref[(ref >= w["interval"][0]) & (ref <= w["interval"][1])])
    assert len(ref) == 12
    # The subspace has full rank L M = 32 for 12 eigenvalues: the other 20
    # directions hold filtered noise, and a Ritz value of those may land in
    # the rectangle (the FP64 path shows none on this input, a different
    # rounding may show one).  Such a value is no eigenvalue and its
    # residual says so; the converged pairs are exactly the 12 eigenvalues.
    good = rs <= 1e-8
    assert good.sum() == 12
    assert np.max(np.abs(ev[good] - ref) / np.abs(ref)) <= 1e-10
    assert np.all(rs[~good] > 1e-3)
    for k in np.flatnonzero(good)[[0, -1]]:
        r = wilson.apply_H(U, vec[k], w["kappa"], w["dims"], w["bc_t"]) - ev[k] * vec[k]
        assert np.linalg.norm(r) <= 1e-8


@pytest.mark.parametrize("dims,kind,bc", [((4, 4, 4, 4), "haar", -1), ((3, 2, 5, 4), "smooth", 1)])
def test_df_stencil_matches_oracle(ss, dims, kind, bc):
    U = synthetic.gauge_field(dims, kind, seed=3, eps=0.5)
    psi = synthetic.gaussian_sources(dims, 2, seed=4)
    lat = ss.create_lattice(dims, 0.135, bc, precision=ss.DF)
    ss.upload_gauge(lat, U)
    got = ss.apply_H_mixed(lat, psi)
    ref = wilson.apply_H(U, psi, 0.135, dims, bc)
    # the FP64 stencil's bar: 1e-13 relative
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("dims,kind,kappa,N,L", [((4, 4, 4, 4), "haar", 0.13, 8, 2),
                                                  ((3, 2, 5, 4), "smooth", 0.12, 6, 3)])
def test_df_shifted_cg_against_oracle(ss, dims, kind, kappa, N, L):
    import torch
    bc = -1
    U = synthetic.gauge_field(dims, kind, seed=7, eps=0.4)
    v = synthetic.gaussian_sources(dims, L, seed=8)
    z = contour.line_nodes(0.38, 0.02, 0.5, N)
    tol = 1e-11
    lat = ss.create_lattice(dims, kappa, bc, stream=torch.cuda.Stream())
    ss.upload_gauge(lat, U)
    code, y, iters, xi, seed_iters = ss.shifted_cg(lat, z, v, tol=tol, precision=ss.DF)
    assert code == ss.OK
    A = lambda x: wilson.apply_H(U, x, kappa, dims, bc)
    for l in range(L):
        ref = oscg.shifted_cg(A, v[l], z, tol=tol)
        vn = np.linalg.norm(v[l])
        for j in range(N):
            yn = np.linalg.norm(y[l, j])
            r_gpu = v[l] - (z[j] * y[l, j] - A(y[l, j]))
            r_orc = v[l] - (z[j] * ref["y"][j] - A(ref["y"][j]))
            # The float-float operator's error per application is within the
            # stencil bar (1e-13 relative, test_df_stencil_matches_oracle);
            # the true residual drifts from the recursive one by up to that
            # much per iteration (factor 4 as in the FP64 test).
            drift = 4 * int(iters[l, j]) * 1e-13 * (abs(z[j]) + 1 + 8 * kappa) * yn
            assert np.linalg.norm(r_gpu) <= tol * vn + drift
            bound = (np.linalg.norm(r_gpu) + np.linalg.norm(r_orc)) / abs(z[j].imag)
            assert np.linalg.norm(y[l, j] - ref["y"][j]) <= bound * (1 + 1e-6)
            assert int(iters[l, j]) <= 1.2 * int(ref["iters"][j]) + 2
    assert seed_iters == int(iters.max())


def test_df_eigenpairs_config1(ss):
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, "haar", seed=1)
    src = synthetic.gaussian_sources(dims, 3, seed=100)
    lat = ss.create_lattice(dims, 0.13, -1, precision=ss.DF)
    ss.upload_gauge(lat, U)
    res = ss.ss_solve(lat, (0.374, 0.3930), 16, 8, src, beta=0.3, nprime=14)
    assert res.status == ss.OK, res.error
    ev, vec, rs, st = ss.ss_eigpairs(res)
    lam = np.array(json.load(open(GOLDEN))["haar_4x4x4x4_k0.13_s1"]["lowest_abs"])
    exact = np.sort(lam[(lam >= 0.374) & (lam <= 0.3930)])
    assert len(ev) == len(exact) == 8
    assert np.max(np.abs(ev - exact) / exact) <= 1e-10
    assert np.max(rs) <= 1e-8
    r = wilson.apply_H(U, vec[5], 0.13, dims, -1) - ev[5] * vec[5]
    assert abs(np.linalg.norm(r) - rs[5]) <= 1e-12 + 1e-6 * rs[5]


def test_df_eigenpairs_full_size(ss):
    import torch
    w = bench.CONFIG2
    U, src = bench.make_inputs(0, bench.CONFIG2)
    lat = ss.create_lattice(w["dims"], w["kappa"], w["bc_t"], precision=ss.DF, stream=torch.cuda.Stream())
    ss.upload_gauge(lat, U)
    res = ss.ss_solve(lat, w["interval"], w["N"], w["M"], src, beta=w["beta"], nprime=w["nprime"], tol=w["tol"])
    assert res.status == ss.OK, res.error
    ev, vec, rs, st = ss.ss_eigpairs(res)
    ref = np.array(json.load(open(GOLDEN))["smooth_8x8x8x8_e0.3_k0.125_s2"]["lowest_abs"])
    ref = np.sort(ref[(ref >= w["interval"][0]) & (ref <= w["interval"][1])])
    good = rs <= 1e-8
    assert good.sum() == len(ref) == 12
    assert np.max(np.abs(ev[good] - ref) / np.abs(ref)) <= 1e-10
    assert np.all(rs[~good] > 1e-3)
    for k in np.flatnonzero(good)[[0, -1]]:
        r = wilson.apply_H(U, vec[k], w["kappa"], w["dims"], w["bc_t"]) - ev[k] * vec[k]
        assert np.linalg.norm(r) <= 1e-8


@pytest.mark.parametrize("precision", ["FP64", "FP64_DFSHIFT", "DF"])
def test_refined_ritz_vectors_full_size(ss, precision):
    # Refined Ritz vectors (opts.refine): the same eigenvalues, and for every
    # converged pair a residual no larger than its Ritz residual; the pairs
    # that a spurious Ritz value nearby contaminates recover FP64-level
    # residuals, and the spurious value itself (whose refined vector would
    # duplicate its neighbour) is dropped.
    import torch
    w = bench.CONFIG2
    U, src = bench.make_inputs(0, bench.CONFIG2)
    lat = ss.create_lattice(w["dims"], w["kappa"], w["bc_t"], precision=getattr(ss, precision),
                            stream=torch.cuda.Stream())
    ss.upload_gauge(lat, U)
    kw = dict(beta=w["beta"], nprime=w["nprime"], tol=w["tol"])
    r0 = ss.ss_solve(lat, w["interval"], w["N"], w["M"], src, **kw)
    r1 = ss.ss_solve(lat, w["interval"], w["N"], w["M"], src, refine=1, **kw)
    assert r0.status == ss.OK and r1.status == ss.OK, (r0.error, r1.error)
    ev0, _, rs0, _ = ss.ss_eigpairs(r0, want_vectors=False)
    ev1, vec1, rs1, _ = ss.ss_eigpairs(r1)
    ref = np.array(json.load(open(GOLDEN))["smooth_8x8x8x8_e0.3_k0.125_s2"]["lowest_abs"])
    ref = np.sort(ref[(ref >= w["interval"][0]) & (ref <= w["interval"][1])])
    good0, good1 = rs0 <= 1e-8, rs1 <= 1e-8
    assert good0.sum() == good1.sum() == 12
    assert np.max(np.abs(ev1[good1] - ref) / ref) <= 1e-10
    assert len(ev1) == 12 and np.all(good1)
    # each refined residual <= the Ritz residual of the same eigenvalue
    for e, r in zip(ev1, rs1):
        k0 = int(np.argmin(np.abs(ev0 - e)))
        assert abs(ev0[k0] - e) <= 1e-10 * e and r <= rs0[k0] * (1 + 1e-6) + 1e-13
    assert np.max(rs1) <= 1e-9
    k = int(np.argmax(np.where(good1, rs1, 0)))
    r = wilson.apply_H(U, vec1[k], w["kappa"], w["dims"], w["bc_t"]) - ev1[k] * vec1[k]
    assert abs(np.linalg.norm(r) - rs1[k]) <= 1e-12 + 1e-6 * rs1[k]
