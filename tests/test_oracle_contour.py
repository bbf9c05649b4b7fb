"""Pins of the oracle's quadrature nodes, weights and filter function."""
import numpy as np
import pytest

from oracle import contour


@pytest.mark.parametrize("N", [8, 16, 32, 64])
def test_circle_weights_are_zeta_over_N(N):
    # Section 2.1 prints w_j = (z_j - gamma)/N for C; normalised by rho this
    # is zeta_j / N, which must be the unique solution of the Section 3 system.
    z = contour.circle_nodes(0.3, 2.0, N)
    zeta = contour.normalise(z, 0.3, 2.0)
    w = contour.weights_closed_form(zeta)
    assert np.max(np.abs(w - zeta / N)) < 1e-14


@pytest.mark.parametrize("N,k", [(16, 0), (16, 5), (32, 0), (32, 7), (64, 3)])
def test_circle_filter_closed_form(N, k):
    # Section 2.1: on the unit circle f_k(x) = x^k / (1 + x^N).
    zeta = contour.normalise(contour.circle_nodes(0.0, 1.0, N), 0.0, 1.0)
    w = contour.weights_closed_form(zeta)
    x = np.array([0.0, 0.3, -0.7, 0.95, 1.2, -1.5, 3.0, 0.2 + 0.1j])
    f = contour.filter_function(zeta, w, k, x)
    assert np.allclose(f, x ** k / (1 + x ** N), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("N,beta", [(8, 0.2), (12, 0.6), (16, 0.3), (16, 1.0)])
def test_line_weights_closed_form_matches_linear_system(N, beta):
    z = contour.line_nodes(0.1, 0.5, beta, N)
    zeta = contour.normalise(z, 0.1, 0.5)
    w1 = contour.weights_moment_system(zeta)
    w2 = contour.weights_closed_form(zeta)
    assert np.max(np.abs(w1 - w2)) <= 1e-10 * np.max(np.abs(w2))
    # the defining equations themselves (the k = 0 row has power -1)
    assert abs(np.sum(w2 / zeta) - 1.0) < 1e-12
    for m in range(0, N - 1):
        assert abs(np.sum(w2 * zeta ** m)) < 1e-11


@pytest.mark.parametrize("N,beta", [(32, 0.2), (64, 0.3)])
def test_line_weights_satisfy_system_at_large_N(N, beta):
    zeta = contour.normalise(contour.line_nodes(0.0, 1.0, beta, N), 0.0, 1.0)
    w = contour.weights_closed_form(zeta)
    assert abs(np.sum(w / zeta) - 1.0) < 1e-9
    scale = np.sum(np.abs(w) * np.abs(zeta) ** (N - 2))
    for m in range(0, N - 1):
        assert abs(np.sum(w * zeta ** m)) < 1e-12 * max(1.0, scale)


@pytest.mark.parametrize("N,beta,k", [(16, 0.2, 0), (16, 0.6, 3), (32, 0.4, 0), (32, 0.4, 10)])
def test_filter_equals_polynomial_ratio(N, beta, k):
    # f_k(x) = x^k P(0) / P(x) for k <= N - 1 (partial fractions).
    zeta = contour.normalise(contour.line_nodes(0.0, 1.0, beta, N), 0.0, 1.0)
    w = contour.weights_closed_form(zeta)
    x = np.linspace(-1.5, 1.5, 41) + 1e-3
    f = contour.filter_function(zeta, w, k, x)
    P = lambda t: np.prod(t[:, None] - zeta[None, :], axis=1)
    ref = x ** k * P(np.zeros(1))[0] / P(x.astype(complex))
    assert np.allclose(f, ref, rtol=1e-10, atol=1e-14)


def test_line_nodes_geometry():
    N, g, r, b = 16, 0.2, 0.5, 0.3
    z = contour.line_nodes(g, r, b, N)
    assert np.allclose(z[0::2].imag, b * r) and np.allclose(z[1::2].imag, -b * r)
    xs = (z[0::2].real - g) / r
    assert np.isclose(xs[0], -1) and np.isclose(xs[-1], 1)
    assert np.allclose(np.diff(xs), xs[1] - xs[0])
    assert np.allclose(z[0::2].real, z[1::2].real)


def test_window_mapping_core_rectangle():
    # The N' central points (N'/2 per line) span the accepted interval.
    N, Np = 32, 16
    g, r = contour.window_from_interval(-0.1, 0.3, N, Np)
    z = contour.line_nodes(g, r, 0.2, N)
    xr = np.sort(np.unique(np.round(z.real, 14)))
    centre = xr[(N // 2 - Np // 2) // 2:(N // 2 + Np // 2) // 2]
    assert len(centre) == Np // 2
    assert np.isclose(centre[0], -0.1) and np.isclose(centre[-1], 0.3)


def test_filter_f0_section3_shape():
    # Section 3: f_0 on L+- has no plateau; it is largest at the centre and
    # decays beyond the ends, faster for smaller beta.
    N = 32
    vals = {}
    for beta in (0.2, 0.6, 1.0, 1.4):
        zeta = contour.normalise(contour.line_nodes(0.0, 1.0, beta, N), 0.0, 1.0)
        w = contour.weights_closed_form(zeta)
        f = np.abs(contour.filter_function(zeta, w, 0, np.array([0.0, 0.5, 1.5, 3.0])))
        assert f[0] > f[2] > f[3]
        vals[beta] = f
    assert vals[0.2][2] < vals[1.4][2]


def test_point_reuse_matches_table2():
    # Section 4, Table 2: six adjacent line pairs (N = 32, N' = 16) need 102
    # quadrature points, four circles 128 (no reuse).
    import json, os
    facts = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")))
    t = facts["table2_line_pairs"]
    wins = contour.tiled_windows(-0.1, 0.1, t["windows"], t["N"], t["Nprime"])
    zs = [contour.line_nodes(g, r, 0.2, t["N"]) for g, r, _, _ in wins]
    assert contour.distinct_points(zs) == t["points"]
    # the cores tile the interval and all windows share rho
    assert np.isclose(wins[0][2], -0.1) and np.isclose(wins[-1][3], 0.1)
    assert all(np.isclose(w_[1], wins[0][1]) for w_ in wins)
    c = facts["table2_circles"]
    circ = [contour.circle_nodes(0.03 * k, 0.01, c["N"]) for k in range(c["circles"])]
    assert contour.distinct_points(circ) == c["points"]
