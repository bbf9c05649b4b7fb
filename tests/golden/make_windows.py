"""Write ``windows.json``: the low-lying spectrum of the seeded gauge fields.

Run: ``python tests/golden/make_windows.py``.  Uses only the oracle's Wilson
operator, the seeded input generators and dense/ARPACK eigensolvers; the
CUDA path plays no part.  The stored eigenvalues fix the accepted intervals
of the workloads (an interval that brackets a chosen set of low-lying
eigenvalues, with its ends in spectral gaps) and serve as independent
eigenvalue references for the parity tests.
"""
import json
import os
import sys
import time

import numpy as np
import scipy.sparse.linalg as sla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synthetic  # noqa: E402
from oracle import wilson  # noqa: E402


def low_spectrum_dense(dims, kind, seed, eps, kappa, bc, count):
    U = synthetic.gauge_field(dims, kind, seed=seed, eps=eps)
    lam = np.linalg.eigvalsh(wilson.dense_H(U, kappa, dims, bc))
    return np.sort(lam[np.argsort(np.abs(lam))[:count]])


def low_spectrum_arpack(dims, kind, seed, eps, kappa, bc, count):
    """Eigenvalues of A nearest zero from the smallest eigenvalues of A^2;
    signs recovered by Rayleigh quotients of A on the eigenvectors."""
    U = synthetic.gauge_field(dims, kind, seed=seed, eps=eps)
    V = U.shape[1]
    n = 12 * V
    A = lambda x: wilson.apply_H(U, x.reshape(-1, V, 4, 3), kappa, dims, bc).reshape(x.shape)
    op = sla.LinearOperator((n, n), matvec=lambda x: A(A(x)), dtype=np.complex128)
    w2, X = sla.eigsh(op, k=count, which="SA", tol=1e-12, ncv=max(3 * count, 80), maxiter=100000)
    # A is block diagonal on each eigenspace of A^2 with eigenvalues +-sqrt(w2);
    # diagonalise A on the returned subspace to split the two signs.
    AX = np.stack([A(X[:, i]) for i in range(count)], axis=1)
    small = X.conj().T @ AX
    lam, W = np.linalg.eigh(0.5 * (small + small.conj().T))
    Y = X @ W
    res = np.linalg.norm(np.stack([A(Y[:, i]) for i in range(count)], axis=1) - Y * lam, axis=0)
    return np.sort(lam), float(res.max())


def main():
    out = {}
    t = time.time()
    out["haar_4x4x4x4_k0.13_s1"] = {
        "dims": [4, 4, 4, 4], "kind": "haar", "seed": 1, "eps": 0.0, "kappa": 0.13, "bc_t": -1,
        "lowest_abs": low_spectrum_dense((4, 4, 4, 4), "haar", 1, 0.0, 0.13, -1, 40).tolist(),
        "method": "dense eigvalsh",
    }
    print("4^4 done", time.time() - t, flush=True)
    lam, res = low_spectrum_arpack((8, 8, 8, 8), "smooth", 2, 0.3, 0.125, -1, 64)
    out["smooth_8x8x8x8_e0.3_k0.125_s2"] = {
        "dims": [8, 8, 8, 8], "kind": "smooth", "seed": 2, "eps": 0.3, "kappa": 0.125, "bc_t": -1,
        "lowest_abs": lam.tolist(), "max_residual": res, "method": "ARPACK on A^2, signs split on the subspace",
    }
    print("8^4 done", time.time() - t, res, flush=True)
    with open(os.path.join(HERE, "windows.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
