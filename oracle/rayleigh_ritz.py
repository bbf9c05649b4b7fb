"""Oracle: Rayleigh-Ritz extraction from the moment block (Section 2.1).

Test infrastructure (see ``oracle/__init__``).

The paper builds an orthonormal basis Q of span(S_hat) and takes the Ritz
pairs of (Q^H A Q, Q^H Q); with Q orthonormal Q^H Q = I and this is an
ordinary Hermitian eigenproblem.  The paper does not say how S_hat is
orthogonalised; the oracle uses the SVD and keeps the left singular vectors
whose singular value exceeds ``rank_tol`` times the largest (S_hat is
numerically rank deficient whenever M L exceeds the number of eigenvalues
the filter lets through).  Eigenvector x_l = Q w_l with ||x_l|| = 1 and the
residual res_l = ||A x_l - theta_l x_l||_2, both as defined in Section 4.
Accepted pairs are those whose Ritz value lies in the core interval formed
by the N' central quadrature points (Section 3).

Pins (tests/test_oracle_rayleigh_ritz.py): Ritz values against a dense
eigendecomposition of A; residuals recomputed independently; a matrix with
known eigenvectors spanning S_hat exactly.
"""
from __future__ import annotations

import numpy as np


def orthonormal_basis(S, rank_tol=1e-14):
    U, sv, _ = np.linalg.svd(S, full_matrices=False)
    if sv.size == 0 or sv[0] == 0.0:
        return U[:, :0], sv
    r = int(np.count_nonzero(sv > rank_tol * sv[0]))
    return U[:, :r], sv


def rayleigh_ritz(apply_A_cols, S, rank_tol=1e-14):
    """Ritz pairs of A on span(S).

    ``apply_A_cols(X)`` applies A to every column of the n x m matrix X.
    Returns (theta ascending, X with unit columns, residuals, rank)."""
    Q, _ = orthonormal_basis(S, rank_tol)
    AQ = apply_A_cols(Q)
    At = Q.conj().T @ AQ
    At = 0.5 * (At + At.conj().T)
    theta, W = np.linalg.eigh(At)
    X = Q @ W
    AX = apply_A_cols(X)
    res = np.linalg.norm(AX - X * theta[None, :], axis=0) / np.linalg.norm(X, axis=0)
    return theta, X, res, Q.shape[1]


def accept(theta, lo, hi):
    """Mask of Ritz values inside the core interval [lo, hi]."""
    theta = np.asarray(theta)
    return (theta >= lo) & (theta <= hi)


def refined_ritz(apply_A_cols, S, thetas, rank_tol=1e-14):
    """Refined Ritz vectors (Jia's refined projection; an extension, not in
    the paper): for each given Ritz value theta, the unit vector x of span(S)
    that minimises ||(A - theta) x||_2, i.e. x = Q v with v the right
    singular vector of the smallest singular value of A Q - theta Q.
    Returns (Rayleigh quotients x^H A x, X with unit columns, residuals
    ||A x - (x^H A x) x||_2)."""
    Q, _ = orthonormal_basis(S, rank_tol)
    AQ = apply_A_cols(Q)
    X = np.empty((Q.shape[0], len(thetas)), dtype=np.complex128)
    rq = np.empty(len(thetas))
    res = np.empty(len(thetas))
    for k, th in enumerate(thetas):
        _, _, Vh = np.linalg.svd(AQ - th * Q, full_matrices=False)
        x = Q @ Vh[-1].conj()
        x = x / np.linalg.norm(x)
        Ax = apply_A_cols(x[:, None])[:, 0]
        rq[k] = np.real(np.vdot(x, Ax))
        res[k] = np.linalg.norm(Ax - rq[k] * x)
        X[:, k] = x
    return rq, X, res
