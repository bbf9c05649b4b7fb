"""Oracle: quadrature nodes, weights and the filter function.

Test infrastructure (see ``oracle/__init__``).

* Circle C (Section 2.1): z_j = gamma + rho exp(2 pi i (j + 1/2) / N),
  j = 0..N-1.  The paper prints the weights as (z_j - gamma)/N; in the
  normalised variable zeta_j = (z_j - gamma)/rho (the form Eq. 2, the filter
  identity f_k(x) = x^k/(1 + x^N) and the line-pair weight system all use)
  they are zeta_j / N.  The factor rho between the two is a uniform scale of
  every moment and cancels in the extracted eigenpairs.
* Line pair L+- (Section 3): z = gamma + rho (x +- i beta), -1 <= x <= 1,
  N/2 equally spaced points per line; even j on L+, odd j on L-.  The points
  include both ends, x_i = -1 + 2 i / (N/2 - 1).
* Weights on L+- (Section 3): the paper defines them as the solution of
  sum_j w_j zeta_j^(k-1) = 1 for k = 0 and 0 for k = 1..N-1, i.e. the power
  -1 has weight one and the powers 0..N-2 vanish.  ``weights_moment_system``
  solves that linear system as written.  Its matrix is a Vandermonde matrix
  whose condition number reaches ~1e18 at N = 64, so ``weights_closed_form``
  gives the same solution in closed form: with P(zeta) = prod_k (zeta - zeta_k),
  w_j = -P(0) / P'(zeta_j).  (Residues of zeta^m / P(zeta) sum to zero for
  m <= N - 2, and those of 1/(zeta P(zeta)) give the k = 0 row.)
* Filter function (Eq. 3): f_k(x) = sum_j w_j zeta_j^k / (zeta_j - x).

Several windows (Section 3): adjacent line pairs with the same N, rho and
beta, shifted along the real axis so that their cores tile an interval;
their nodes are then shared except for N' - 2 per new window.

Pins (tests/test_oracle_contour.py): on circle nodes the closed form returns
zeta_j / N, and the filter equals x^k / (1 + x^N), both printed in
Section 2.1; closed form against the linear solve on line nodes for N <= 16;
the filter against x^k P(0)/P(x); node geometry (Im z = +-beta rho, even/odd
line assignment, equal spacing).
"""
from __future__ import annotations

import numpy as np


def line_abscissae(N: int) -> np.ndarray:
    """x_i, i = 0..N/2-1: N/2 equally spaced points on [-1, 1], ends included."""
    if N < 4 or N % 2:
        raise ValueError("N must be even and >= 4")
    h = N // 2
    return -1.0 + 2.0 * np.arange(h) / (h - 1)


def line_nodes(gamma: float, rho: float, beta: float, N: int) -> np.ndarray:
    """Quadrature points z_j on L+- (even j on L+, odd j on L-)."""
    x = line_abscissae(N)
    z = np.empty(N, dtype=np.complex128)
    z[0::2] = gamma + rho * (x + 1j * beta)
    z[1::2] = gamma + rho * (x - 1j * beta)
    return z


def circle_nodes(gamma: complex, rho: float, N: int) -> np.ndarray:
    """Quadrature points z_j on the circle C."""
    j = np.arange(N)
    return gamma + rho * np.exp(2j * np.pi * (j + 0.5) / N)


def normalise(z: np.ndarray, gamma: complex, rho: float) -> np.ndarray:
    """zeta_j = (z_j - gamma) / rho."""
    return (np.asarray(z) - gamma) / rho


def weights_moment_system(zeta: np.ndarray) -> np.ndarray:
    """Solve sum_j w_j zeta_j^(k-1) = delta_{k0}, k = 0..N-1, directly."""
    N = len(zeta)
    powers = np.arange(-1, N - 1)
    A = zeta[None, :] ** powers[:, None]
    rhs = np.zeros(N, dtype=np.complex128)
    rhs[0] = 1.0
    return np.linalg.solve(A, rhs)


def weights_closed_form(zeta: np.ndarray) -> np.ndarray:
    """w_j = -P(0)/P'(zeta_j), P(zeta) = prod_k (zeta - zeta_k).

    Written as w_j = zeta_j * prod_{k != j} (-zeta_k)/(zeta_j - zeta_k) so that
    each factor is O(1) and nothing overflows at large N."""
    zeta = np.asarray(zeta, dtype=np.complex128)
    N = len(zeta)
    w = np.empty(N, dtype=np.complex128)
    for j in range(N):
        others = np.delete(zeta, j)
        w[j] = zeta[j] * np.prod(-others / (zeta[j] - others))
    return w


def filter_function(zeta: np.ndarray, w: np.ndarray, k: int, x) -> np.ndarray:
    """f_k(x) = sum_j w_j zeta_j^k / (zeta_j - x)  (Eq. 3)."""
    x = np.asarray(x, dtype=np.complex128)
    return np.sum((w * zeta ** k)[None, :] / (zeta[None, :] - x.reshape(-1, 1)), axis=1).reshape(x.shape)


def core_half_width(N: int, Nprime: int) -> float:
    """Half-width, in units of rho, of the rectangle formed by the Nprime
    central quadrature points (Nprime/2 per line, Section 3)."""
    if Nprime < 4 or Nprime % 2 or Nprime > N:
        raise ValueError("Nprime must be even, >= 4 and <= N")
    return (Nprime // 2 - 1) / (N // 2 - 1)


def window_from_interval(a: float, b: float, N: int, Nprime: int):
    """Map an accepted interval [a, b] to (gamma, rho): the Nprime central
    points span [a, b] exactly, gamma = (a + b)/2."""
    if not b > a:
        raise ValueError("interval must have b > a")
    gamma = 0.5 * (a + b)
    rho = 0.5 * (b - a) / core_half_width(N, Nprime)
    return gamma, rho


def tiled_windows(a: float, b: float, K: int, N: int, Nprime: int):
    """K adjacent line-pair windows with the same N, rho (Section 3): the
    window cores (N' central points) tile [a, b]; window k is returned as
    (gamma_k, rho, lo_k, hi_k).  Neighbouring windows are N' - 2 points
    apart, so their nodes coincide except for N' - 2 new points."""
    core = (b - a) / K
    out = []
    for k in range(K):
        lo, hi = a + k * core, a + (k + 1) * core
        gamma, rho = window_from_interval(lo, hi, N, Nprime)
        out.append((gamma, rho, lo, hi))
    return out


def distinct_points(zs, decimals=12):
    """Number of distinct quadrature points among several node sets."""
    allz = np.concatenate([np.asarray(z) for z in zs])
    return len(np.unique(np.round(allz.real, decimals) + 1j * np.round(allz.imag, decimals)))
