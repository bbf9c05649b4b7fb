"""Oracle: moment-based (Hankel pencil) extraction (Section 2.1).

Test infrastructure (see ``oracle/__init__``).

Section 2.1 forms mu_k = v^H s_k, the Hankel matrix H_m = [mu_{i+j-2}] and
the shifted one H^<_m = [mu_{i+j-1}]; the pencil (H^<_m, H_m) has the
eigenvalues inside the contour.  With the normalised moments of Eq. 2 the
pencil returns eta = (lambda - gamma)/rho.  The block version (L sources)
uses the L x L blocks mu_k = V^H s_hat_k.  H_m is truncated to its numerical
rank (singular values above ``rank_tol`` times the largest) before the
pencil is reduced to a standard eigenproblem.

Used as an independent cross-check of the Rayleigh-Ritz path; it needs the
moments up to k = 2M - 1.

Pin: for exact solves and M L at least the number of eigenvalues the
filter passes, the pencil eigenvalues inside the window match a dense
eigendecomposition (tests/test_oracle_rayleigh_ritz.py).
"""
from __future__ import annotations

import numpy as np


def block_hankel_eigs(V, s_hat, rank_tol=1e-12):
    """V: n x L sources; s_hat: (2M, n, L) moments.  Returns eta values."""
    K2 = s_hat.shape[0]
    M = K2 // 2
    L = V.shape[1]
    mu = np.stack([V.conj().T @ s_hat[k] for k in range(K2)])
    H = np.zeros((M * L, M * L), dtype=np.complex128)
    Hs = np.zeros_like(H)
    for i in range(M):
        for j in range(M):
            H[i * L:(i + 1) * L, j * L:(j + 1) * L] = mu[i + j]
            Hs[i * L:(i + 1) * L, j * L:(j + 1) * L] = mu[i + j + 1]
    U, sv, Vh = np.linalg.svd(H)
    r = int(np.count_nonzero(sv > rank_tol * sv[0]))
    Ur, Vr = U[:, :r], Vh[:r].conj().T
    small = (Ur.conj().T @ Hs @ Vr) / sv[:r][:, None]
    return np.linalg.eigvals(small)
