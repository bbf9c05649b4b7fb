"""Pins of the oracle's shifted CG against dense solves and invariants."""
import numpy as np
import pytest

import synthetic
from oracle import contour, shifted_cg, wilson


def _setup(dims=(2, 2, 2, 2), kappa=0.12, seed=1):
    U = synthetic.gauge_field(dims, "haar", seed=seed)
    Hd = wilson.dense_H(U, kappa, dims, -1)
    v = synthetic.gaussian_sources(dims, 1, seed=seed + 10)[0]
    return U, Hd, v


def test_diagonal_special_case():
    # A diagonal: (z I - A) y = v has y = v / (z - d) exactly.
    g = synthetic.rng(3)
    d = np.concatenate([g.uniform(-2, -0.1, 30), g.uniform(0.1, 2, 30)])
    v = g.standard_normal(60) + 1j * g.standard_normal(60)
    z = contour.line_nodes(0.0, 0.5, 0.3, 8)
    out = shifted_cg.shifted_cg(lambda x: d * x, v, z, tol=1e-13)
    for j, zj in enumerate(z):
        assert np.allclose(out["y"][j], v / (zj - d), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("beta", [0.2, 0.6])
def test_against_dense_solve(beta):
    U, Hd, v = _setup()
    z = contour.line_nodes(0.05, 0.3, beta, 16)
    out = shifted_cg.shifted_cg(lambda x: (Hd @ x.reshape(-1)).reshape(x.shape), v, z, tol=1e-12)
    vn = np.linalg.norm(v)
    n = Hd.shape[0]
    for j, zj in enumerate(z):
        A = zj * np.eye(n) - Hd
        exact = np.linalg.solve(A, v.reshape(-1))
        yj = out["y"][j].reshape(-1)
        true_res = np.linalg.norm(v.reshape(-1) - A @ yj) / vn
        assert true_res <= 1.5e-12
        cond = np.linalg.cond(A)
        assert np.linalg.norm(yj - exact) <= 2 * cond * 1e-12 * np.linalg.norm(exact)


def test_collinear_residuals():
    # Section 2.2: r^sigma_k = xi^sigma_k r_k at every iteration.
    U, Hd, v = _setup(seed=4)
    z = contour.line_nodes(-0.02, 0.25, 0.4, 8)
    A = lambda x: (Hd @ x.reshape(-1)).reshape(x.shape)
    out = shifted_cg.shifted_cg(A, v, z, tol=1e-10, history=True)
    vn = np.linalg.norm(v)
    for k in range(1, 8):
        r = out["hist_r"][k]
        for j, zj in enumerate(z):
            y = out["hist_y"][k][j]
            true = v - (zj * y - A(y))
            assert np.linalg.norm(true - out["hist_xi"][k][j] * r) <= 1e-12 * vn


def test_seed_shift_reproduces_plain_cg():
    # A shift equal to the seed shift has xi = 1 and y equal to CG's iterate.
    U, Hd, v = _setup(seed=5)
    sigma = 3.0   # sigma I - A positive definite: plain CG
    A = lambda x: (Hd @ x.reshape(-1)).reshape(x.shape)
    out = shifted_cg.shifted_cg(A, v, np.array([sigma, sigma + 0.5j]), sigma=sigma, tol=1e-12)
    assert np.allclose(out["xi"][0], np.abs(out["xi"][0]))
    exact = np.linalg.solve(sigma * np.eye(Hd.shape[0]) - Hd, v.reshape(-1))
    assert np.allclose(out["y"][0].reshape(-1), exact, rtol=1e-10)


def test_matrix_free_operator_and_stop_rule():
    dims = (2, 2, 2, 4)
    U = synthetic.gauge_field(dims, "smooth", seed=2, eps=0.5)
    v = synthetic.gaussian_sources(dims, 1, seed=3)[0]
    z = contour.line_nodes(0.0, 0.2, 0.3, 8)
    A = lambda x: wilson.apply_H(U, x, 0.125, dims, -1)
    out = shifted_cg.shifted_cg(A, v, z, tol=1e-12)
    vn = np.linalg.norm(v)
    for j, zj in enumerate(z):
        r = v - (zj * out["y"][j] - A(out["y"][j]))
        assert np.linalg.norm(r) / vn < 1.5e-12
    assert out["matvecs"] == out["iters"].max()


def test_breakdown_detected():
    # K = -A with A = diag(1, -1) and v = (1, 1): (p, K p) = 0 at once.
    v = np.array([1.0, 1.0], dtype=complex)
    with pytest.raises(shifted_cg.Breakdown):
        shifted_cg.shifted_cg(lambda x: np.array([1.0, -1.0]) * x, v, np.array([0.1j]))
