"""Oracle: the shifted CG method with a real seed shift (Section 2.2).

Test infrastructure (see ``oracle/__init__``).

Problem: (z_j I - A) y_j = v for every quadrature point z_j, A Hermitian.
Section 2.2 observes that with a real seed shift sigma the seed matrix
K = sigma I - A is Hermitian, so plain CG can run on K, and that by the
shift invariance of Krylov subspaces (Eq. 5) each shifted residual is a
scalar multiple of the seed residual, r^j_k = xi^j_k r_k.  Writing
z_j I - A = K + s_j I with s_j = z_j - sigma, every shifted solution then
follows from the seed's one matrix-vector product per iteration.  The
paper does not print the shifted-CG recurrences (it cites them); the ones
below are the standard multi-shift CG recurrences that keep r^j_k = xi^j_k r_k
(the paper's own stopping test ||r^j_k|| / ||v|| <= tol is then
|xi^j_k| ||r_k|| / ||v|| <= tol):

    seed CG on K:   alpha_k = (r_k, r_k) / (p_k, K p_k)
                    r_{k+1} = r_k - alpha_k K p_k
                    beta_k  = (r_{k+1}, r_{k+1}) / (r_k, r_k)
                    p_{k+1} = r_{k+1} + beta_k p_k
    shift j:        xi_{k+1} = xi_k xi_{k-1} alpha_{k-1} /
                        [ alpha_k beta_{k-1} (xi_{k-1} - xi_k)
                          + xi_{k-1} alpha_{k-1} (1 + s_j alpha_k) ]
                    alpha^j_k = alpha_k xi_{k+1} / xi_k
                    beta^j_k  = (xi_{k+1} / xi_k)^2 beta_k
                    y_j      += alpha^j_k p^j_k
                    p^j_{k+1} = xi_{k+1} r_{k+1} + beta^j_k p^j_k
    start:          r_0 = p_0 = p^j_0 = v, y_j = 0,
                    xi_0 = xi_{-1} = 1, alpha_{-1} = 1, beta_{-1} = 0.

A shift stops updating once |xi^j_{k+1}| ||r_{k+1}|| <= tol ||v||; the loop
ends when every shift has stopped.  With sigma = 0 (the paper's choice,
Section 4) K is indefinite and (p, K p) can vanish; the paper gives no
breakdown test, and the oracle raises ``Breakdown`` when
|(p, K p)| < 1e-30 (r_k, r_k) (in CG ||p_k|| >= ||r_k||, so this is at least
as strict as a test against ||p_k||^2).

Pins (tests/test_oracle_shifted_cg.py): every y_j against a dense solve;
the true residual of every shift against the tolerance; the collinearity
v - (z_j I - A) y_j^(k) = xi^j_k r_k at every early iteration (Eq. 5 and the
text after it); a diagonal A, where the solutions are v / (z_j - d); a shift
equal to the seed shift reproducing plain CG.
"""
from __future__ import annotations

import numpy as np


class Breakdown(ArithmeticError):
    """(p, K p) vanished: CG on the indefinite seed system cannot proceed."""


class NoConvergence(RuntimeError):
    pass


def _dot(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def shifted_cg(apply_A, v, z, sigma=0.0, tol=1e-12, max_iter=100000, history=False):
    """Solve (z_j I - A) y_j = v for all j from one CG run on sigma I - A.

    ``apply_A(x)`` returns A x for an array shaped like ``v``.  Returns a dict
    with ``y`` (N, *v.shape), ``iters`` (per-shift iteration count at which it
    stopped), ``xi`` (final xi per shift), ``matvecs``, and, when
    ``history`` is set, per-iteration lists of ``r`` and ``xi``
    (``hist_r[k]`` = r_k, ``hist_xi[k][j]`` = xi^j_k), ``hist_y``
    (y_j after k updates) and the seed scalars ``hist_alpha[k]`` = alpha_k,
    ``hist_beta[k]`` = beta_k."""
    z = np.asarray(z, dtype=np.complex128)
    N = len(z)
    s = z - sigma

    def apply_K(x):
        return sigma * x - apply_A(x)

    vnorm = np.sqrt(_dot(v, v).real)
    r = v.astype(np.complex128).copy()
    p = r.copy()
    rr = _dot(r, r).real
    y = np.zeros((N,) + v.shape, dtype=np.complex128)
    pj = np.broadcast_to(r, (N,) + v.shape).copy()
    xi_cur = np.ones(N, dtype=np.complex128)
    xi_prev = np.ones(N, dtype=np.complex128)
    alpha_prev, beta_prev = 1.0, 0.0
    active = np.ones(N, dtype=bool)
    iters = np.zeros(N, dtype=np.int64)
    out = {"hist_r": [], "hist_xi": [], "hist_y": [], "hist_alpha": [], "hist_beta": []} if history else {}
    if history:
        out["hist_r"].append(r.copy())
        out["hist_xi"].append(xi_cur.copy())
        out["hist_y"].append(y.copy())
    k = 0
    while active.any():
        if k >= max_iter:
            raise NoConvergence(f"{int(active.sum())} shifts not converged after {k} iterations")
        q = apply_K(p)
        pq = _dot(p, q).real
        if not abs(pq) >= 1e-30 * rr:
            raise Breakdown(f"(p, K p) = {pq} at iteration {k}")
        alpha = rr / pq
        xi_next = xi_cur.copy()
        for j in np.nonzero(active)[0]:
            den = (alpha * beta_prev * (xi_prev[j] - xi_cur[j])
                   + xi_prev[j] * alpha_prev * (1.0 + s[j] * alpha))
            xi_next[j] = xi_cur[j] * xi_prev[j] * alpha_prev / den
            y[j] += (alpha * xi_next[j] / xi_cur[j]) * pj[j]
        r = r - alpha * q
        rr_new = _dot(r, r).real
        beta = rr_new / rr
        for j in np.nonzero(active)[0]:
            beta_j = (xi_next[j] / xi_cur[j]) ** 2 * beta
            pj[j] = xi_next[j] * r + beta_j * pj[j]
        p = r + beta * p
        k += 1
        for j in np.nonzero(active)[0]:
            xi_prev[j] = xi_cur[j]
            xi_cur[j] = xi_next[j]
            iters[j] = k
            if abs(xi_cur[j]) * np.sqrt(rr_new) <= tol * vnorm:
                active[j] = False
        alpha_prev, beta_prev, rr = alpha, beta, rr_new
        if history:
            out["hist_r"].append(r.copy())
            out["hist_xi"].append(xi_cur.copy())
            out["hist_y"].append(y.copy())
            out["hist_alpha"].append(alpha)
            out["hist_beta"].append(beta)
    out.update(y=y, iters=iters, xi=xi_cur, matvecs=k)
    return out
