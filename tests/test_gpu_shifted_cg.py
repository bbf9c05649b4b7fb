"""Parity of the CUDA shifted CG and moments with the oracle."""
import numpy as np
import pytest

from tests._lib import gpu_module

import synthetic
from oracle import contour, moments as omoments, shifted_cg as oscg, wilson

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    return gpu_module()


def _problem(dims, kind, kappa, bc, L, seed):
    U = synthetic.gauge_field(dims, kind, seed=seed, eps=0.3)
    v = synthetic.gaussian_sources(dims, L, seed=seed + 100)
    return U, v


@pytest.mark.parametrize("dims,kind,kappa,N,L,beta,side_stream", [
    ((2, 2, 2, 2), "haar", 0.13, 8, 1, 0.3, False),
    ((4, 4, 4, 4), "haar", 0.13, 16, 2, 0.3, True),     # CUDA-graph replay of the loop
    ((3, 2, 4, 6), "smooth", 0.125, 12, 3, 0.5, False),  # direct launches (legacy stream)
])
def test_shifted_cg_matches_oracle(ss, dims, kind, kappa, N, L, beta, side_stream):
    import torch
    bc = -1
    U, v = _problem(dims, kind, kappa, bc, L, seed=7)
    gamma, rho = 0.38, 0.02
    z = contour.line_nodes(gamma, rho, beta, N)
    lat = ss.create_lattice(dims, kappa, bc, stream=torch.cuda.Stream() if side_stream else None)
    ss.upload_gauge(lat, U)
    code, y, iters, xi, seed_iters = ss.shifted_cg(lat, z, v, tol=1e-12)
    assert code == ss.OK
    A = lambda x: wilson.apply_H(U, x, kappa, dims, bc)
    normA = 1.0 + 8.0 * kappa
    for l in range(L):
        ref = oscg.shifted_cg(A, v[l], z, tol=1e-12)
        vn = np.linalg.norm(v[l])
        for j in range(N):
            r_gpu = v[l] - (z[j] * y[l, j] - A(y[l, j]))
            r_orc = v[l] - (z[j] * ref["y"][j] - A(ref["y"][j]))
            # The stopping rule bounds the recursive residual by tol ||v||; the
            # true residual may exceed it by the rounding drift of the
            # recurrences, ~ iterations x eps x ||A|| x ||y|| (a factor 4 covers
            # the growth of ||y|| along the iteration).
            drift = 4 * int(iters[l, j]) * 2.2e-16 * normA * np.linalg.norm(y[l, j])
            assert np.linalg.norm(r_gpu) <= 1e-12 * vn + drift
            # y - y_exact = (z I - A)^{-1} r and ||(z I - A)^{-1}|| <= 1/|Im z|
            bound = (np.linalg.norm(r_gpu) + np.linalg.norm(r_orc)) / abs(z[j].imag)
            assert np.linalg.norm(y[l, j] - ref["y"][j]) <= bound * (1 + 1e-6)
            # The freeze iteration is not unique in floating point: CG on the
            # indefinite seed loses orthogonality at a rate set by rounding,
            # so two correct runs stop a few per cent apart.  Both meet the
            # stopping rule (checked above through the true residual); here
            # only a gross slowdown would be a defect.
            assert int(iters[l, j]) <= 1.2 * int(ref["iters"][j]) + 2
    assert seed_iters == int(iters.max())


def test_shifted_cg_zero_source_and_real_seed(ss):
    dims = (2, 2, 2, 4)
    U, v = _problem(dims, "haar", 0.12, -1, 2, seed=3)
    v[1] = 0.0
    z = contour.line_nodes(0.0, 0.5, 0.4, 8)
    lat = ss.create_lattice(dims, 0.12, -1)
    ss.upload_gauge(lat, U)
    code, y, iters, xi, _ = ss.shifted_cg(lat, z, v, sigma=2.5, tol=1e-12)
    assert code == ss.OK
    assert np.all(y[1] == 0) and np.all(iters[1] == 0)
    A = lambda x: wilson.apply_H(U, x, 0.12, dims, -1)
    ref = oscg.shifted_cg(A, v[0], z, sigma=2.5, tol=1e-12)
    for j in range(len(z)):
        assert np.linalg.norm(y[0, j] - ref["y"][j]) <= 2.5e-12 * np.linalg.norm(v[0]) / abs(z[j].imag)


def test_shifted_cg_max_iter_reports_noconv(ss):
    dims = (4, 4, 4, 4)
    U, v = _problem(dims, "haar", 0.13, -1, 1, seed=5)
    z = contour.line_nodes(0.38, 0.02, 0.3, 8)
    lat = ss.create_lattice(dims, 0.13, -1)
    ss.upload_gauge(lat, U)
    code, y, iters, xi, seed_iters = ss.shifted_cg(lat, z, v, tol=1e-12, max_iter=32)
    assert code == ss.ERR_NOCONV
    assert seed_iters == 32


def test_moments_match_oracle(ss):
    dims = (4, 2, 2, 6)
    g = synthetic.rng(9)
    N, M, L = 16, 8, 3
    V = synthetic.volume(dims)
    y = g.standard_normal((L, N, V, 4, 3)) + 1j * g.standard_normal((L, N, V, 4, 3))
    z = contour.line_nodes(0.1, 0.05, 0.3, N)
    zeta = contour.normalise(z, 0.1, 0.05)
    w = contour.weights_closed_form(zeta)
    lat = ss.create_lattice(dims, 0.1, -1)
    s = ss.moments(lat, w, zeta, y, M)
    for l in range(L):
        ref = omoments.moments(y[l], w, zeta, M)
        scale = np.sum(np.abs(w)[:, None] * np.abs(zeta)[:, None] ** np.arange(M)[None, :], axis=0)
        for k in range(M):
            assert np.max(np.abs(s[l, k] - ref[k])) <= 1e-14 * scale[k] * np.max(np.abs(y)) * 8


@pytest.mark.parametrize("prec", ["FP64", "DF"])
def test_seed_breakdown_returns_status(ss, prec):
    """The seed matrix K = sigma I - A with sigma = 0 (Section 4) is
    indefinite, so CG on it can break down.  Free field (U = 1), periodic
    time, kappa = 1/16: the constant spinor with colour-0 components in spin 0
    (gamma5 = +1) and spin 2 (gamma5 = -1) is a sum of a +lambda and a -lambda
    eigenvector of equal norm (lambda = 1 - 8 kappa = 1/2), so (v, K v) = 0
    exactly in binary arithmetic, at the first iteration.  Built on the
    host; the solve must return SSQCD_ERR_BREAKDOWN (no fault, no hang)."""
    dims, kappa, bc = (4, 4, 4, 4), 1.0 / 16.0, +1
    U = synthetic.unit_gauge(dims)
    V = synthetic.volume(dims)
    v = np.zeros((1, V, 4, 3), dtype=np.complex128)
    v[0, :, 0, 0] = 1.0
    v[0, :, 2, 0] = 1.0
    Av = wilson.apply_H(U, v[0], kappa, dims, bc)
    assert np.vdot(v[0], Av) == 0.0
    assert np.allclose(Av[:, 0, 0], 0.5) and np.allclose(Av[:, 2, 0], -0.5)
    with pytest.raises(oscg.Breakdown):
        oscg.shifted_cg(lambda x: wilson.apply_H(U, x, kappa, dims, bc), v[0],
                        contour.line_nodes(0.5, 0.05, 0.3, 8), tol=1e-12)
    lat = ss.create_lattice(dims, kappa, bc, precision=getattr(ss, prec))
    ss.upload_gauge(lat, U)
    z = contour.line_nodes(0.5, 0.05, 0.3, 8)
    code, *_ = ss.shifted_cg(lat, z, v, tol=1e-12, precision=getattr(ss, prec))
    assert code == ss.ERR_BREAKDOWN
    res = ss.ss_solve(lat, (0.45, 0.55), 8, 4, v, beta=0.3, nprime=4)
    assert res.status == ss.ERR_BREAKDOWN
    # the context stays usable: a regular solve afterwards succeeds
    w = synthetic.gaussian_sources(dims, 1, seed=5)
    code, *_ = ss.shifted_cg(lat, z, w, tol=1e-10, precision=getattr(ss, prec))
    assert code == ss.OK
