"""Oracle: quadrature moments s_hat_k (Eq. 2) and their block form.

Test infrastructure (see ``oracle/__init__``).

    s_hat_k = sum_{j=0}^{N-1} w_j zeta_j^k y_j,   y_j = (z_j I - A)^{-1} v,

k = 0..M-1 (Eq. 2).  With L sources v_1..v_L (the block variant, Section
2.1) the columns of S_hat (n x M L) are ordered source-major:
column l*M + k holds s_hat_k for source l.

Pin (tests/test_oracle_moments.py): with exact solves, s_hat_k equals the
filtered eigen-expansion sum_l f_k(eta_l) alpha_l x_l / rho of Section 2.1
(eta_l = (lambda_l - gamma)/rho, v = sum_l alpha_l x_l), built from a dense
eigendecomposition and the closed-form filter.
"""
from __future__ import annotations

import numpy as np


def moments(y, w, zeta, M):
    """s_hat_k for k = 0..M-1 from the N shifted solutions y (N, ...)."""
    y = np.asarray(y)
    out = np.zeros((M,) + y.shape[1:], dtype=np.complex128)
    for k in range(M):
        for j in range(len(w)):
            out[k] += w[j] * zeta[j] ** k * y[j]
    return out


def block_moment_matrix(ys, w, zeta, M):
    """S_hat (n x M L) from per-source solutions ``ys`` (L, N, ...)."""
    cols = []
    for y in ys:
        s = moments(y, w, zeta, M)
        for k in range(M):
            cols.append(s[k].reshape(-1))
    return np.stack(cols, axis=1)
