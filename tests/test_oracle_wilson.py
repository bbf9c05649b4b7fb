"""Pins of the oracle's Wilson operator against facts independent of it."""
import numpy as np
import pytest

import synthetic
from oracle import wilson


def test_clifford_algebra():
    gam, g5 = wilson.gamma_matrices()
    eye = np.eye(4)
    for mu in range(4):
        assert np.allclose(gam[mu], gam[mu].conj().T)
        for nu in range(4):
            anti = gam[mu] @ gam[nu] + gam[nu] @ gam[mu]
            assert np.allclose(anti, 2.0 * eye * (mu == nu))
        assert np.allclose(g5 @ gam[mu] + gam[mu] @ g5, 0)
    assert np.allclose(g5, g5.conj().T)
    assert np.allclose(g5 @ g5, eye)
    # chiral basis: gamma5 diagonal with two +1 and two -1
    assert np.allclose(g5, np.diag(np.diag(g5)))
    assert sorted(np.diag(g5).real) == [-1, -1, 1, 1]


def test_dimension_count_section4():
    # Section 4: a 12^3 x 24 lattice gives a 497,664 dimensional matrix.
    assert 12 * synthetic.volume((12, 12, 12, 24)) == 497664


@pytest.mark.parametrize("dims,bc", [((2, 2, 2, 2), -1), ((4, 2, 2, 4), 1), ((3, 2, 2, 4), -1)])
def test_hermitian_and_gamma5_hermitian(dims, bc):
    U = synthetic.gauge_field(dims, "haar", seed=1)
    kappa = 0.13
    x = synthetic.gaussian_sources(dims, 1, seed=2)[0]
    y = synthetic.gaussian_sources(dims, 1, seed=3)[0]
    Hx = wilson.apply_H(U, x, kappa, dims, bc)
    Hy = wilson.apply_H(U, y, kappa, dims, bc)
    lhs = np.vdot(x, Hy)
    rhs = np.vdot(Hx, y)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # gamma5 (I - kappa D) gamma5 = (I - kappa D)^H
    Mx = wilson.apply_M(U, x, kappa, dims, bc)
    g5My = wilson.apply_gamma5(wilson.apply_M(U, wilson.apply_gamma5(y), kappa, dims, bc))
    assert abs(np.vdot(x, g5My) - np.vdot(Mx, y)) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(y) * 10


def test_dense_matches_matrix_free():
    dims = (2, 2, 2, 2)
    U = synthetic.gauge_field(dims, "haar", seed=5)
    Hd = wilson.dense_H(U, 0.11, dims, -1)
    assert np.allclose(Hd, Hd.conj().T, atol=1e-14)
    x = synthetic.gaussian_sources(dims, 1, seed=6)[0]
    assert np.allclose(Hd @ x.reshape(-1), wilson.apply_H(U, x, 0.11, dims, -1).reshape(-1), atol=1e-13)


def test_gauge_covariance():
    dims = (2, 4, 2, 4)
    bc = -1
    U = synthetic.gauge_field(dims, "haar", seed=7)
    g = synthetic.random_gauge_transform(dims, seed=8)
    fwd, _, _, _ = wilson.neighbours(dims, bc)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = g @ U[mu] @ np.conj(np.swapaxes(g[fwd[mu]], -1, -2))
    psi = synthetic.gaussian_sources(dims, 1, seed=9)[0]
    gpsi = np.einsum("sab,sib->sia", g, psi)
    lhs = wilson.apply_H(Ug, gpsi, 0.12, dims, bc)
    rhs = np.einsum("sab,sib->sia", g, wilson.apply_H(U, psi, 0.12, dims, bc))
    assert np.allclose(lhs, rhs, atol=1e-13)


@pytest.mark.parametrize("bc", [1, -1])
def test_free_field_plane_wave_symbol(bc):
    # On a plane wave exp(i p.x) chi the free operator acts as the 4x4
    # symbol gamma5 (1 - 2 kappa sum cos p + 2 i kappa sum gamma_mu sin p_mu).
    dims = (4, 2, 2, 4)
    kappa = 0.125
    U = synthetic.unit_gauge(dims)
    coords = wilson.site_coords(dims)
    P = wilson.free_field_momenta(dims, bc)
    g = synthetic.rng(11)
    for p in P[[1, 5, 11, 30]]:
        chi = g.standard_normal((4, 3)) + 1j * g.standard_normal((4, 3))
        phase = np.exp(1j * coords @ p)
        psi = phase[:, None, None] * chi[None]
        out = wilson.apply_H(U, psi, kappa, dims, bc)
        expect = phase[:, None, None] * (wilson.free_field_symbol(p, kappa) @ chi)[None]
        assert np.allclose(out, expect, atol=1e-13)


@pytest.mark.parametrize("dims,bc", [((2, 2, 2, 2), -1), ((2, 2, 2, 2), 1), ((4, 2, 2, 4), -1)])
def test_free_field_spectrum(dims, bc):
    kappa = 0.125
    U = synthetic.unit_gauge(dims)
    ev = np.linalg.eigvalsh(wilson.dense_H(U, kappa, dims, bc))
    ref = wilson.free_field_spectrum(dims, kappa, bc)
    assert np.max(np.abs(ev - ref)) < 1e-13


def test_spectrum_gauge_invariant():
    dims = (2, 2, 2, 2)
    U = synthetic.gauge_field(dims, "smooth", seed=3, eps=0.5)
    g = synthetic.random_gauge_transform(dims, seed=4)
    fwd, _, _, _ = wilson.neighbours(dims, -1)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = g @ U[mu] @ np.conj(np.swapaxes(g[fwd[mu]], -1, -2))
    e1 = np.linalg.eigvalsh(wilson.dense_H(U, 0.13, dims, -1))
    e2 = np.linalg.eigvalsh(wilson.dense_H(Ug, 0.13, dims, -1))
    assert np.max(np.abs(e1 - e2)) < 1e-13


def test_synthetic_links_are_su3():
    for kind in ("haar", "smooth"):
        U = synthetic.gauge_field((2, 2, 2, 2), kind, seed=1, eps=0.3)
        uu = U @ np.conj(np.swapaxes(U, -1, -2))
        assert np.allclose(uu, np.eye(3), atol=1e-14)
        assert np.allclose(np.linalg.det(U), 1.0, atol=1e-14)
