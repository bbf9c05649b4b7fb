"""The identity the library's Krylov-basis form rests on, checked on the
oracle's own shifted CG (Section 2.2): every shifted solution is a fixed
combination of the seed residuals,

    p^j_k = sum_{s <= k} (prod_{m=s}^{k-1} beta^j_m) xi^j_s r_s,
    y_j   = sum_k alpha^j_k p^j_k = sum_s xi^j_s g_j(s) r_s,
    g_j(s) = alpha^j_s + beta^j_s g_j(s + 1),  g_j(K_j) = 0,

with alpha^j_k = alpha_k xi_{k+1} / xi_k, beta^j_k = (xi_{k+1} / xi_k)^2 beta_k
and K_j the number of updates of shift j, so the moments of Eq. 2 are one
combination of the stored residuals.  (The library keeps p-hat = p / xi;
the same identity with its coefficients a_j = alpha_k xi_{k+1},
b_j = beta_k xi_{k+1} / xi_k.)"""
import numpy as np

import synthetic
from oracle import contour, moments as omoments, shifted_cg, wilson


def _case(N=12):
    dims, kappa = (2, 2, 2, 4), 0.12
    U = synthetic.gauge_field(dims, "haar", seed=7)
    v = synthetic.gaussian_sources(dims, 1, seed=8)[0]
    A = lambda x: wilson.apply_H(U, x, kappa, dims, -1)
    lam = np.linalg.eigvalsh(wilson.dense_H(U, kappa, dims, -1))
    pos = np.sort(lam[lam > 0])
    gamma, rho = contour.window_from_interval(pos[0] - 0.01, 0.5 * (pos[3] + pos[4]), N, N // 2)
    z = contour.line_nodes(gamma, rho, 0.3, N)
    return A, v, z, gamma, rho


def _coefficients(out, N):
    """c[j][s]: coefficient of r_s in y_j, from the backward recurrence."""
    xi = np.array(out["hist_xi"])          # [K + 1][N], xi^j_k
    alpha = np.array(out["hist_alpha"])    # [K]
    beta = np.array(out["hist_beta"])      # [K]
    K = len(alpha)
    c = np.zeros((N, K + 1), dtype=np.complex128)
    for j in range(N):
        Kj = int(out["iters"][j])
        g = 0.0
        for s in range(Kj - 1, -1, -1):
            ratio = xi[s + 1, j] / xi[s, j]
            a_js = alpha[s] * ratio
            b_js = ratio ** 2 * beta[s]
            g = a_js + b_js * g
            c[j, s] = xi[s, j] * g
    return c


def test_solutions_are_combinations_of_the_seed_residuals():
    A, v, z, _, _ = _case()
    out = shifted_cg.shifted_cg(A, v, z, tol=1e-12, history=True)
    R = np.array(out["hist_r"])            # [K + 1][...]
    c = _coefficients(out, len(z))
    for j in range(len(z)):
        y = np.tensordot(c[j], R, axes=1)
        assert np.linalg.norm(y - out["y"][j]) <= 1e-12 * np.linalg.norm(out["y"][j])
        # and it solves its system to the CG tolerance
        r = v - (z[j] * y - A(y))
        assert np.linalg.norm(r) <= 2e-12 * np.linalg.norm(v)


def test_moments_are_one_combination_of_the_seed_residuals():
    A, v, z, gamma, rho = _case()
    M = 6
    zeta = contour.normalise(z, gamma, rho)
    w = contour.weights_closed_form(zeta)
    out = shifted_cg.shifted_cg(A, v, z, tol=1e-12, history=True)
    R = np.array(out["hist_r"])
    c = _coefficients(out, len(z))
    ref = omoments.moments(out["y"], w, zeta, M)
    for k in range(M):
        Gk = np.sum((w * zeta ** k)[:, None] * c, axis=0)  # coefficient of r_s in s_hat_k
        s_k = np.tensordot(Gk, R, axes=1)
        scale = np.sum(np.abs(w) * np.abs(zeta) ** k) * np.max(np.linalg.norm(out["y"].reshape(len(z), -1), axis=1))
        assert np.linalg.norm(s_k - ref[k]) <= 1e-13 * scale


def test_a_frozen_shift_stops_contributing():
    # shifts that freeze early take no residual past their last update
    A, v, z, _, _ = _case()
    out = shifted_cg.shifted_cg(A, v, z, tol=1e-12, history=True)
    c = _coefficients(out, len(z))
    for j in range(len(z)):
        Kj = int(out["iters"][j])
        assert np.all(c[j, Kj:] == 0)
        assert abs(c[j, Kj - 1]) > 0
    assert len(set(int(i) for i in out["iters"])) > 1  # the shifts freeze at different iterations


def test_moment_coefficients_are_real_on_a_conjugate_closed_contour():
    # The line pair of a real centre (Section 3) holds each point's conjugate,
    # with the conjugate weight; the seed's CG scalars are real (Hermitian A,
    # real seed shift), so the coefficient of r_s in s_hat_k is real and the
    # moments are the real parts' combination.  Off the real axis (a complex
    # centre) the coefficients are not real.
    A, v, z, gamma, rho = _case()
    M = 6
    zeta = contour.normalise(z, gamma, rho)
    w = contour.weights_closed_form(zeta)
    out = shifted_cg.shifted_cg(A, v, z, tol=1e-12, history=True)
    R = np.array(out["hist_r"])
    c = _coefficients(out, len(z))
    ref = omoments.moments(out["y"], w, zeta, M)
    for k in range(M):
        Gk = np.sum((w * zeta ** k)[:, None] * c, axis=0)
        big = np.sum(np.abs((w * zeta ** k)[:, None] * c), axis=0)
        assert np.all(np.abs(Gk.imag) <= 1e-13 * np.max(big))
        s_k = np.tensordot(Gk.real, R, axes=1)
        scale = np.sum(np.abs(w) * np.abs(zeta) ** k) * np.max(np.linalg.norm(out["y"].reshape(len(z), -1), axis=1))
        assert np.linalg.norm(s_k - ref[k]) <= 1e-13 * scale
    zc = z + 0.05j * rho
    outc = shifted_cg.shifted_cg(A, v, zc, tol=1e-12, history=True)
    cc = _coefficients(outc, len(zc))
    Gc = np.sum((w * zeta ** 1)[:, None] * cc, axis=0)
    assert np.max(np.abs(Gc.imag)) > 1e-3 * np.max(np.abs(Gc))
