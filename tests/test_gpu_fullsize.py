"""Parity at the benchmark's full size (8^4, N = 32, L = 4) in the launch
configuration bench.py times (side stream, CUDA-graph replay): outputs the
oracle can check one by one -- eigenvalues against the independent ARPACK
spectrum of the oracle operator, eigenvector residuals and sampled
shifted-CG residuals recomputed with the oracle operator."""
import json
import os

import numpy as np
import pytest

from tests._lib import gpu_module

import bench
import synthetic
from oracle import contour, wilson

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "windows.json")


@pytest.fixture(scope="module")
def setup():
    import torch
    ss = gpu_module()
    w = bench.CONFIG2
    U, src = bench.make_inputs(0, bench.CONFIG2)
    stream = torch.cuda.Stream()
    lat = ss.create_lattice(w["dims"], w["kappa"], w["bc_t"], stream=stream)
    ss.upload_gauge(lat, U)
    return ss, w, U, src, lat


def test_eigenpairs_full_size(setup):
    ss, w, U, src, lat = setup
    res = ss.ss_solve(lat, w["interval"], w["N"], w["M"], src, beta=w["beta"], nprime=w["nprime"], tol=w["tol"])
    assert res.status == ss.OK, res.error
    ev, vec, rs, st = ss.ss_eigpairs(res)
    ref = np.array(json.load(open(GOLDEN))["smooth_8x8x8x8_e0.3_k0.125_s2"]["lowest_abs"])
    ref = np.sort(ref[(ref >= w["interval"][0]) & (ref <= w["interval"][1])])
    assert len(ref) == 12
    # The subspace has full rank L M = 32 for 12 eigenvalues: the other 20
    # directions hold filtered noise, and a Ritz value of those may land in
    # the rectangle depending on rounding; its residual marks it (the paper's
    # acceptance is by position; the converged pairs are the 12 eigenvalues).
    good = rs <= 1e-8
    assert good.sum() == 12
    assert np.all(rs[~good] > 1e-3)
    ev, vec, rs = ev[good], vec[good], rs[good]
    assert np.max(np.abs(ev - ref) / np.abs(ref)) <= 1e-10
    for k in (0, 5, 11):
        r = wilson.apply_H(U, vec[k], w["kappa"], w["dims"], w["bc_t"]) - ev[k] * vec[k]
        assert np.linalg.norm(r) <= 1e-8
        assert abs(np.linalg.norm(r) - rs[k]) <= 1e-12 + 1e-6 * rs[k]


def test_shifted_cg_full_size_sampled(setup):
    ss, w, U, src, lat = setup
    gamma, rho = contour.window_from_interval(*w["interval"], w["N"], w["nprime"])
    z = contour.line_nodes(gamma, rho, w["beta"], w["N"])
    code, y, iters, xi, seed_iters = ss.shifted_cg(lat, z, src, tol=w["tol"])
    assert code == ss.OK
    normA = 1.0 + 8.0 * w["kappa"]
    for l, j in [(0, 0), (1, 7), (2, 16), (3, 31)]:
        v = src[l]
        r = v - (z[j] * y[l, j] - wilson.apply_H(U, y[l, j], w["kappa"], w["dims"], w["bc_t"]))
        drift = 4 * int(iters[l, j]) * 2.2e-16 * normA * np.linalg.norm(y[l, j])
        assert np.linalg.norm(r) <= w["tol"] * np.linalg.norm(v) + drift
    assert seed_iters == int(iters.max())


GOLDEN12 = os.path.join(os.path.dirname(__file__), "golden", "window_12.json")


@pytest.mark.parametrize("precision", ["FP64", "FP64_DFSHIFT"])
def test_eigenpairs_12x12x12x12(precision):
    # A larger lattice (n = 248832, the 12^4 size of the batched configuration):
    # the lowest positive cluster of the seeded eps = 0.4 field (12
    # eigenvalues in [0.0864, 0.0898], next one 0.1495), against the ARPACK
    # spectrum of the oracle operator; residuals recomputed by the oracle.
    import torch
    ss = gpu_module()
    g = json.load(open(GOLDEN12))["smooth_12x12x12x12_e0.4_k0.13_s3"]
    dims, kappa, bc = tuple(g["dims"]), g["kappa"], g["bc_t"]
    U = synthetic.gauge_field(dims, g["kind"], seed=g["seed"], eps=g["eps"])
    src = synthetic.gaussian_sources(dims, 4, seed=400)
    lat = ss.create_lattice(dims, kappa, bc, precision=getattr(ss, precision), stream=torch.cuda.Stream())
    ss.upload_gauge(lat, U)
    # the core interval brackets the cluster with both ends in spectral gaps;
    # the contour (rho = 0.0075, beta 0.3) stays far from the next clusters
    interval = (0.085, 0.091)
    res = ss.ss_solve(lat, interval, 32, 8, src, beta=0.3, nprime=16)
    assert res.status == ss.OK, res.error
    ev, vec, rs, st = ss.ss_eigpairs(res)
    lam = np.array(g["lowest_abs"])
    ref = np.sort(lam[(lam >= interval[0]) & (lam <= interval[1])])
    assert len(ref) == 12
    good = rs <= 1e-8
    assert good.sum() == 12
    assert np.all(rs[~good] > 1e-3)
    ev, vec, rs = ev[good], vec[good], rs[good]
    assert np.max(np.abs(ev - ref) / ref) <= 1e-10
    for k in (0, 11):
        r = wilson.apply_H(U, vec[k], kappa, dims, bc) - ev[k] * vec[k]
        assert np.linalg.norm(r) <= 1e-8
        assert abs(np.linalg.norm(r) - rs[k]) <= 1e-12 + 1e-6 * rs[k]


def test_shifted_cg_16x16x16x32_true_residuals():
    # The lattice shape of the mixed configuration (n = 1572864; 16^3 x 32,
    # kappa 0.135, eps 0.5): the operator against the oracle's, and the true
    # residual of every shifted solution recomputed by the oracle operator
    # (float-float shift vectors; the stopping rule is 1e-10 relative).
    import torch
    ss = gpu_module()
    dims, kappa = (16, 16, 16, 32), 0.135
    U = synthetic.gauge_field(dims, "smooth", seed=4, eps=0.5)
    v = synthetic.gaussian_sources(dims, 2, seed=301)
    z = np.array([0.1 + 0.01j, 0.1 - 0.01j, 0.005j, 0.05 + 0.002j])
    lat = ss.create_lattice(dims, kappa, -1, precision=ss.FP64_DFSHIFT, stream=torch.cuda.Stream())
    ss.upload_gauge(lat, U)
    A = lambda x: wilson.apply_H(U, x, kappa, dims, -1)
    got = ss.apply_H(lat, v[:1])[0]
    ref = A(v[0])
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    code, y, iters, xi, seed_iters = ss.shifted_cg(lat, z, v, tol=1e-10, precision=ss.FP64_DFSHIFT)
    assert code == ss.OK
    for l in range(2):
        vn = np.linalg.norm(v[l])
        for j in range(len(z)):
            r = v[l] - (z[j] * y[l, j] - A(y[l, j]))
            drift = 8 * int(iters[l, j]) * 2.0 ** -48 * (abs(z[j]) + 1 + 8 * kappa) * np.linalg.norm(y[l, j])
            assert np.linalg.norm(r) <= 1e-10 * vn + drift
