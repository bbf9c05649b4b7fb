"""Pins of the oracle's Rayleigh-Ritz, Hankel and full pipeline."""
import json
import os

import numpy as np
import pytest

import synthetic
from oracle import contour, hankel, moments, rayleigh_ritz, ss, wilson

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "windows.json")


def _dense(dims=(2, 2, 2, 2), kappa=0.13, seed=2):
    U = synthetic.gauge_field(dims, "haar", seed=seed)
    return U, wilson.dense_H(U, kappa, dims, -1)


def test_exact_invariant_subspace():
    # S spanning k eigenvectors exactly: Ritz pairs are those eigenpairs.
    U, Hd = _dense()
    lam, X = np.linalg.eigh(Hd)
    idx = [10, 11, 40, 41, 100]
    g = synthetic.rng(3)
    S = X[:, idx] @ (g.standard_normal((5, 7)) + 1j * g.standard_normal((5, 7)))
    theta, Xr, res, rank = rayleigh_ritz.rayleigh_ritz(lambda Q: Hd @ Q, S, rank_tol=1e-12)
    assert rank == 5
    assert np.allclose(theta, lam[idx], atol=1e-13)
    assert np.max(res) < 1e-12
    # Ritz vectors equal the eigenvectors up to phase
    for k, i in enumerate(idx):
        assert abs(abs(np.vdot(X[:, i], Xr[:, k])) - 1) < 1e-12


def test_residual_definition_section4():
    U, Hd = _dense()
    g = synthetic.rng(5)
    S = g.standard_normal((Hd.shape[0], 6)) + 1j * g.standard_normal((Hd.shape[0], 6))
    theta, Xr, res, _ = rayleigh_ritz.rayleigh_ritz(lambda Q: Hd @ Q, S)
    for k in range(len(theta)):
        x = Xr[:, k] / np.linalg.norm(Xr[:, k])
        assert np.isclose(res[k], np.linalg.norm(Hd @ x - theta[k] * x), rtol=1e-10)


def test_accept_interval():
    assert list(rayleigh_ritz.accept([0.1, 0.2, 0.3, 0.4], 0.15, 0.3)) == [False, True, True, False]


def test_hankel_pencil_with_exact_moments():
    U, Hd = _dense(seed=4)
    lam = np.linalg.eigvalsh(Hd)
    pos = np.sort(lam[lam > 0])
    a, b = pos[0] - 0.005, 0.5 * (pos[2] + pos[3])
    N, L, M = 32, 2, 6
    gamma, rho = contour.window_from_interval(a, b, N, N)
    z = contour.line_nodes(gamma, rho, 0.2, N)
    zeta = contour.normalise(z, gamma, rho)
    w = contour.weights_closed_form(zeta)
    V = synthetic.gaussian_sources((2, 2, 2, 2), L, seed=6).reshape(L, -1).T
    n = Hd.shape[0]
    ys = [np.stack([np.linalg.solve(zj * np.eye(n) - Hd, V[:, l]) for zj in z]) for l in range(L)]
    s = np.stack([np.stack([moments.moments(ys[l], w, zeta, 2 * M)[k] for l in range(L)], axis=1)
                  for k in range(2 * M)])
    eta = hankel.block_hankel_eigs(V, s, rank_tol=1e-10)
    lam_h = gamma + rho * eta
    inside = np.sort(lam_h[(np.abs(lam_h.imag) < 1e-6) & (lam_h.real >= a) & (lam_h.real <= b)].real)
    exact = lam[(lam >= a) & (lam <= b)]
    assert len(inside) == len(exact) == 3
    assert np.max(np.abs(inside - exact) / exact) < 1e-8


def test_pipeline_small_lattice_against_dense():
    dims = (2, 2, 2, 4)
    U = synthetic.gauge_field(dims, "haar", seed=1)
    v = synthetic.gaussian_sources(dims, 2, seed=2)
    lam = np.linalg.eigvalsh(wilson.dense_H(U, 0.13, dims, -1))
    pos = np.sort(lam[lam > 0])
    a, b = pos[0] - 0.01, 0.5 * (pos[3] + pos[4])
    out = ss.ss_solve(U, dims, 0.13, -1, (a, b), 16, 8, v, beta=0.3, Nprime=12)
    exact = lam[(lam >= a) & (lam <= b)]
    assert len(out["evals"]) == len(exact) == 4
    assert np.max(np.abs(out["evals"] - exact) / exact) < 1e-10
    assert np.max(out["residuals"]) < 1e-8


@pytest.mark.slow
def test_pipeline_4x4_config_against_dense():
    # 4^4 Haar links, kappa 0.13, the eight smallest positive eigenvalues.
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, "haar", seed=1)
    v = synthetic.gaussian_sources(dims, 3, seed=100)
    out = ss.ss_solve(U, dims, 0.13, -1, (0.374, 0.3930), 16, 8, v, beta=0.3, Nprime=14)
    lam = np.array(json.load(open(GOLDEN))["haar_4x4x4x4_k0.13_s1"]["lowest_abs"])
    exact = lam[(lam >= 0.374) & (lam <= 0.3930)]
    assert len(out["evals"]) == len(exact) == 8
    assert np.max(np.abs(out["evals"] - exact) / exact) < 1e-10
    assert np.max(out["residuals"]) < 1e-8


def test_hankel_blocks_hermitian_psd_on_conjugate_symmetric_contours():
    # With Hermitian A and nodes closed under conjugation (weights conjugate
    # too, since P has real coefficients), mu_k = V^H s_k is Hermitian and
    # the block Hankel matrix H = [mu_{i+j}] is positive semidefinite (the
    # filter P(0)/P(x) is positive on the real axis): the reading the GPU
    # extraction reduces through two Hermitian eigenproblems.
    U, Hd = _dense(seed=5)
    lam = np.linalg.eigvalsh(Hd)
    pos = np.sort(lam[lam > 0])
    a, b = pos[0] - 0.005, 0.5 * (pos[2] + pos[3])
    N, L, M = 16, 2, 4
    for path in ("lines", "circle"):
        gamma, rho = contour.window_from_interval(a, b, N, N // 2)
        if path == "lines":
            z = contour.line_nodes(gamma, rho, 0.3, N)
        else:
            z = contour.circle_nodes(gamma, rho, N)
        zeta = contour.normalise(z, gamma, rho)
        w = contour.weights_closed_form(zeta)
        V = synthetic.gaussian_sources((2, 2, 2, 2), L, seed=8).reshape(L, -1).T
        n = Hd.shape[0]
        ys = [np.stack([np.linalg.solve(zj * np.eye(n) - Hd, V[:, l]) for zj in z]) for l in range(L)]
        s = np.stack([np.stack([moments.moments(ys[l], w, zeta, 2 * M)[k] for l in range(L)], axis=1)
                      for k in range(2 * M)])
        mu = np.stack([V.conj().T @ s[k] for k in range(2 * M)])
        scale = np.max(np.abs(mu))
        assert np.max(np.abs(mu - mu.conj().transpose(0, 2, 1))) <= 1e-12 * scale
        H = np.block([[mu[i + j] for j in range(M)] for i in range(M)])
        h = np.linalg.eigvalsh(0.5 * (H + H.conj().T))
        assert h.min() >= -1e-12 * h.max()


def test_refined_ritz_properties():
    # (1) an exact invariant subspace gives eigenvectors; (2) on a perturbed
    # subspace the refined residual never exceeds the Ritz residual and
    # equals the smallest singular value of A Q - theta Q (brute force).
    U, Hd = _dense(seed=6)
    lam, Vecs = np.linalg.eigh(Hd)
    n = Hd.shape[0]
    A = lambda X: Hd @ X
    S = Vecs[:, 10:14] @ np.diag([1.0, 0.5, 2.0, 1.5])
    th, X, res = rayleigh_ritz.refined_ritz(A, S, lam[10:14])
    assert np.max(np.abs(th - lam[10:14])) <= 1e-12
    assert np.max(res) <= 1e-12
    g = np.random.default_rng(3)
    E = g.standard_normal((n, 6)) + 1j * g.standard_normal((n, 6))
    S2 = Vecs[:, 10:16] + 1e-6 * E
    th_r, X_r, res_r, _ = rayleigh_ritz.rayleigh_ritz(A, S2)
    th_f, X_f, res_f = rayleigh_ritz.refined_ritz(A, S2, th_r)
    assert np.all(res_f <= res_r * (1 + 1e-10) + 1e-15)
    Q, _ = rayleigh_ritz.orthonormal_basis(S2)
    for k in range(len(th_r)):
        smin = np.linalg.svd(Hd @ Q - th_r[k] * Q, compute_uv=False)[-1]
        x = X_f[:, k]
        assert np.linalg.norm(Hd @ x - th_r[k] * x) <= smin * (1 + 1e-8) + 1e-15
