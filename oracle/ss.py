"""Oracle: the whole Sakurai-Sugiura / Rayleigh-Ritz pipeline.

Test infrastructure (see ``oracle/__init__``).  Steps, in the paper's order:

1. window: gamma = (a + b)/2 and rho such that the N' central quadrature
   points span the accepted interval [a, b] (Section 3);
2. nodes z_j on L+- with gap beta (Section 3) or on the circle C
   (Section 2.1), normalised zeta_j, weights w_j;
3. for each source v_l: shifted CG for all (z_j I - A) y_j = v_l with seed
   shift sigma (Section 2.2, default sigma = 0 as in Section 4);
4. moments s_hat_k, k < M, per source (Eq. 2), block S_hat (n x M L);
5. Rayleigh-Ritz on span(S_hat) and acceptance of Ritz values in [a, b]
   (Section 2.1, Section 3; for C, inside the circle).

The parity of every stage is pinned in its own module; this driver only
chains them.
"""
from __future__ import annotations

import numpy as np

from . import contour, moments as mom, rayleigh_ritz as rr, shifted_cg as scg, wilson


def ss_solve(U, dims, kappa, bc_t, interval, N, M, sources, beta=0.3, Nprime=None,
             tol=1e-12, sigma=0.0, rank_tol=1e-14, path="line", max_iter=100000, windows=1):
    dims = tuple(int(d) for d in dims)
    a, b = float(interval[0]), float(interval[1])
    if Nprime is None:
        Nprime = N // 2
    if windows > 1:
        return _ss_windows(U, dims, kappa, bc_t, (a, b), N, M, sources, beta, Nprime, tol, sigma,
                           rank_tol, max_iter, windows)
    if path == "line":
        gamma, rho = contour.window_from_interval(a, b, N, Nprime)
        z = contour.line_nodes(gamma, rho, beta, N)
        lo, hi = a, b
    elif path == "circle":
        gamma, rho = 0.5 * (a + b), 0.5 * (b - a)
        z = contour.circle_nodes(gamma, rho, N)
        lo, hi = a, b
    else:
        raise ValueError(path)
    zeta = contour.normalise(z, gamma, rho)
    w = contour.weights_closed_form(zeta)

    def A(x):
        return wilson.apply_H(U, x, kappa, dims, bc_t)

    V = U.shape[1]
    sources = np.asarray(sources).reshape(-1, V, 4, 3)
    ys, iters, matvecs = [], [], 0
    for v in sources:
        out = scg.shifted_cg(A, v, z, sigma=sigma, tol=tol, max_iter=max_iter)
        ys.append(out["y"])
        iters.append(out["iters"])
        matvecs += out["matvecs"]
    S = mom.block_moment_matrix(ys, w, zeta, M)

    def A_cols(X):
        Xf = X.T.reshape(X.shape[1], V, 4, 3)
        return A(Xf).reshape(X.shape[1], -1).T

    theta, X, res, rank = rr.rayleigh_ritz(A_cols, S, rank_tol)
    keep = rr.accept(theta, lo, hi)
    return {
        "evals": theta[keep], "evecs": X[:, keep], "residuals": res[keep],
        "ritz_all": theta, "res_all": res, "rank": rank,
        "gamma": gamma, "rho": rho, "z": z, "zeta": zeta, "w": w,
        "iters": np.array(iters), "matvecs": matvecs, "S": S, "ys": ys,
    }


def _ss_windows(U, dims, kappa, bc_t, interval, N, M, sources, beta, Nprime, tol, sigma, rank_tol,
                max_iter, K):
    """Several adjacent windows (Section 3): each window is solved as a
    single window and accepts the Ritz values in its share [lo, hi) of the
    interval (the last one [lo, hi]).  The shared quadrature points are
    solved again here; the CUDA path solves each distinct point once."""
    a, b = interval
    evals, evecs, res, zs = [], [], [], []
    for k, (gamma, rho, lo, hi) in enumerate(contour.tiled_windows(a, b, K, N, Nprime)):
        out = ss_solve(U, dims, kappa, bc_t, (lo, hi), N, M, sources, beta=beta, Nprime=Nprime, tol=tol,
                       sigma=sigma, rank_tol=rank_tol, max_iter=max_iter)
        keep = out["evals"] < hi if k < K - 1 else np.ones(len(out["evals"]), dtype=bool)
        evals.append(out["evals"][keep])
        evecs.append(out["evecs"][:, keep])
        res.append(out["residuals"][keep])
        zs.append(out["z"])
    order = np.argsort(np.concatenate(evals))
    return {"evals": np.concatenate(evals)[order], "evecs": np.concatenate(evecs, axis=1)[:, order],
            "residuals": np.concatenate(res)[order], "points": contour.distinct_points(zs)}
