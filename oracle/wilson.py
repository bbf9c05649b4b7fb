"""Oracle: the Hermitian Wilson fermion matrix A = gamma5 (I - kappa D).

Test infrastructure (see ``oracle/__init__``).  Section 4 of the paper
defines A = gamma5 (I - kappa D) with D the Wilson hopping matrix, which it
does not write out.  The reading used here (and by the CUDA path):

    (D psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                        + (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu) ],

Wilson parameter r = 1, DeGrand-Rossi (chiral) gamma basis with
gamma5 = gamma1 gamma2 gamma3 gamma4, periodic boundaries in x, y, z and a
sign ``bc_t`` (+1 periodic, -1 antiperiodic) on hops that wrap in t.

Everything here is written as whole-array numpy gathers and einsums over the
full 4x4 spin matrices (no spin projection, no blocking), so it can be read
against the formula above.

Pins (tests/test_oracle_wilson.py): Clifford algebra of the gamma matrices;
Hermiticity of A and gamma5-Hermiticity of I - kappa D; gauge covariance;
the free-field plane-wave symbol and its closed-form spectrum
+-sqrt((1 - 2 kappa sum cos p)^2 + 4 kappa^2 sum sin^2 p) with multiplicity
six; the dimension count n = 12 V of Section 4.
"""
from __future__ import annotations

import numpy as np


def gamma_matrices():
    """(gamma_1..gamma_4, gamma_5) in the DeGrand-Rossi basis."""
    i = 1j
    g1 = np.array([[0, 0, 0, i], [0, 0, i, 0], [0, -i, 0, 0], [-i, 0, 0, 0]], dtype=np.complex128)
    g2 = np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]], dtype=np.complex128)
    g3 = np.array([[0, 0, i, 0], [0, 0, 0, -i], [-i, 0, 0, 0], [0, i, 0, 0]], dtype=np.complex128)
    g4 = np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]], dtype=np.complex128)
    g5 = g1 @ g2 @ g3 @ g4
    return (g1, g2, g3, g4), g5


def site_coords(dims):
    """Integer coordinates (V, 4) of every site, x fastest."""
    X, Y, Z, T = dims
    s = np.arange(X * Y * Z * T)
    return np.stack([s % X, (s // X) % Y, (s // (X * Y)) % Z, s // (X * Y * Z)], axis=1)


def site_index(coords, dims):
    X, Y, Z, T = dims
    c = np.asarray(coords)
    return c[..., 0] + X * (c[..., 1] + Y * (c[..., 2] + Z * c[..., 3]))


def neighbours(dims, bc_t):
    """Forward/backward neighbour index and boundary sign per direction.

    Returns ``fwd, bwd, sfwd, sbwd`` with shapes (4, V): ``fwd[mu, s]`` is the
    site s + mu (periodic wrap) and ``sfwd[mu, s]`` is ``bc_t`` when that hop
    wraps around the t boundary, 1 otherwise; likewise for s - mu."""
    dims = tuple(int(d) for d in dims)
    c = site_coords(dims)
    V = c.shape[0]
    fwd = np.empty((4, V), dtype=np.int64)
    bwd = np.empty((4, V), dtype=np.int64)
    sfwd = np.ones((4, V))
    sbwd = np.ones((4, V))
    for mu in range(4):
        cf = c.copy()
        cf[:, mu] = (c[:, mu] + 1) % dims[mu]
        cb = c.copy()
        cb[:, mu] = (c[:, mu] - 1) % dims[mu]
        fwd[mu] = site_index(cf, dims)
        bwd[mu] = site_index(cb, dims)
        if mu == 3:
            sfwd[mu, c[:, 3] == dims[3] - 1] = bc_t
            sbwd[mu, c[:, 3] == 0] = bc_t
    return fwd, bwd, sfwd, sbwd


def apply_D(U, psi, dims, bc_t):
    """Wilson hopping term D psi for psi of shape (..., V, 4, 3)."""
    gam, _ = gamma_matrices()
    eye = np.eye(4)
    fwd, bwd, sfwd, sbwd = neighbours(dims, bc_t)
    out = np.zeros_like(psi)
    for mu in range(4):
        # forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
        pf = psi[..., fwd[mu], :, :] * sfwd[mu][:, None, None]
        t = np.einsum("sab,...sib->...sia", U[mu], pf)
        out += np.einsum("ij,...sja->...sia", eye - gam[mu], t)
        # backward: (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu)
        pb = psi[..., bwd[mu], :, :] * sbwd[mu][:, None, None]
        ub = U[mu][bwd[mu]]
        t = np.einsum("sba,...sib->...sia", np.conj(ub), pb)
        out += np.einsum("ij,...sja->...sia", eye + gam[mu], t)
    return out


def apply_gamma5(psi):
    _, g5 = gamma_matrices()
    return np.einsum("ij,...sja->...sia", g5, psi)


def apply_M(U, psi, kappa, dims, bc_t):
    """Wilson matrix (I - kappa D) psi."""
    return psi - kappa * apply_D(U, psi, dims, bc_t)


def apply_H(U, psi, kappa, dims, bc_t):
    """Hermitian fermion matrix A psi = gamma5 (I - kappa D) psi (Section 4)."""
    return apply_gamma5(apply_M(U, psi, kappa, dims, bc_t))


def dense_H(U, kappa, dims, bc_t):
    """A as a dense n x n matrix (n = 12 V), in the flat (site, spin, colour)
    ordering of ``psi.reshape(-1)``.  Intended for V <= 256."""
    V = U.shape[1]
    n = 12 * V
    basis = np.eye(n, dtype=np.complex128).reshape(n, V, 4, 3)
    cols = apply_H(U, basis, kappa, dims, bc_t).reshape(n, n)
    return np.ascontiguousarray(cols.T)


def free_field_momenta(dims, bc_t):
    """All lattice momenta p (V, 4): 2 pi n / L_mu, and (2n + 1) pi / T in t
    when the time boundary is antiperiodic."""
    axes = []
    for mu, L in enumerate(dims):
        k = np.arange(L)
        if mu == 3 and bc_t == -1:
            axes.append((2 * k + 1) * np.pi / L)
        else:
            axes.append(2 * k * np.pi / L)
    grid = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.reshape(-1) for g in grid], axis=1)


def free_field_spectrum(dims, kappa, bc_t):
    """Closed-form eigenvalues of A for unit links, sorted ascending.

    For a plane wave of momentum p, (I - kappa D) acts as
    m(p) + i sum_mu gamma_mu s_mu(p) with m = 1 - 2 kappa sum cos p_mu and
    s_mu = 2 kappa sin p_mu, so A^2 = m^2 + sum s^2 and A has +-sqrt(.) each
    twice in spin space, times three colours."""
    p = free_field_momenta(dims, bc_t)
    m = 1.0 - 2.0 * kappa * np.cos(p).sum(axis=1)
    e = np.sqrt(m * m + (4.0 * kappa * kappa) * (np.sin(p) ** 2).sum(axis=1))
    return np.sort(np.concatenate([np.repeat(e, 6), -np.repeat(e, 6)]))


def free_field_symbol(p, kappa):
    """4x4 spin matrix of A on the plane wave exp(i p.x) chi (unit links,
    forward hop with (1 - gamma_mu)):  gamma5 (m + i sum gamma_mu s_mu)."""
    gam, g5 = gamma_matrices()
    m = 1.0 - 2.0 * kappa * np.cos(p).sum()
    mat = m * np.eye(4, dtype=np.complex128)
    for mu in range(4):
        mat = mat + 1j * 2.0 * kappa * np.sin(p[mu]) * gam[mu]
    return g5 @ mat
