"""Pin of the oracle's moments against the filtered eigen-expansion."""
import numpy as np

import synthetic
from oracle import contour, moments, wilson


def test_moments_equal_filtered_expansion():
    # Section 2.1: s_hat_k = sum_l f_k(eta_l) alpha_l x_l / rho.
    dims = (2, 2, 2, 2)
    U = synthetic.gauge_field(dims, "haar", seed=2)
    Hd = wilson.dense_H(U, 0.13, dims, -1)
    lam, X = np.linalg.eigh(Hd)
    v = synthetic.gaussian_sources(dims, 1, seed=4)[0].reshape(-1)
    gamma, rho, beta, N, M = 0.1, 0.3, 0.4, 16, 6
    z = contour.line_nodes(gamma, rho, beta, N)
    zeta = contour.normalise(z, gamma, rho)
    w = contour.weights_closed_form(zeta)
    n = Hd.shape[0]
    y = np.stack([np.linalg.solve(zj * np.eye(n) - Hd, v) for zj in z])
    s = moments.moments(y, w, zeta, M)
    alpha = X.conj().T @ v
    eta = (lam - gamma) / rho
    for k in range(M):
        fk = contour.filter_function(zeta, w, k, eta)
        ref = X @ (fk * alpha) / rho
        assert np.linalg.norm(s[k] - ref) <= 1e-12 * np.linalg.norm(ref)


def test_block_layout_source_major():
    g = synthetic.rng(1)
    ys = g.standard_normal((2, 4, 10)) + 0j
    zeta = np.array([0.5, -0.5, 0.2j, -0.2j])
    w = np.array([1.0, 2.0, 3.0, 4.0]) + 0j
    S = moments.block_moment_matrix(ys, w, zeta, 3)
    assert S.shape == (10, 6)
    assert np.allclose(S[:, 1 * 3 + 2], sum(w[j] * zeta[j] ** 2 * ys[1, j] for j in range(4)))
