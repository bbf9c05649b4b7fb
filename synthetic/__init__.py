"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds input generation only -- none of the eigensolver's
arithmetic.  Every generator takes an explicit ``numpy.random.Generator``
(PCG64) or an integer seed so that both sides of a parity test receive
bit-identical inputs.

Array conventions (the same ones the C-ABI uses at its boundary):

* lattice ``dims = (X, Y, Z, T)``; site index ``s = x + X*(y + Y*(z + Z*t))``
  (x fastest), ``V = X*Y*Z*T``;
* gauge field ``U``: complex128 array of shape ``(4, V, 3, 3)``, ``U[mu, s]``
  is the SU(3) link from site ``s`` to ``s + mu_hat`` (mu = 0..3 = x, y, z, t);
* spinor field: complex128 ``(V, 4, 3)`` (site, spin, colour); a block of
  ``L`` sources is ``(L, V, 4, 3)``.

The gauge fields stand in for the paper's 12^3 x 24 Wilson configuration
(Section 4), which is not available: Haar-random links (a "hot" field) and
smooth links ``exp(i eps G)`` projected to SU(3) with Hermitian Gaussian
``G`` (small ``eps`` approaches the free field).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng", "volume", "haar_su3", "smooth_su3", "gauge_field", "unit_gauge",
    "gaussian_sources", "random_gauge_transform",
]


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator for ``seed``."""
    return np.random.Generator(np.random.PCG64(seed))


def volume(dims) -> int:
    X, Y, Z, T = (int(d) for d in dims)
    return X * Y * Z * T


def _complex_gaussian(g: np.random.Generator, shape) -> np.ndarray:
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) / np.sqrt(2.0)


def _fix_det(u: np.ndarray) -> np.ndarray:
    """Divide unitary 3x3 matrices by the principal cube root of their det."""
    det = np.linalg.det(u)
    phase = np.exp(-1j * np.angle(det) / 3.0)
    return u * phase[..., None, None]


def haar_su3(g: np.random.Generator, count: int) -> np.ndarray:
    """``count`` Haar-random SU(3) matrices: QR of a complex Gaussian 3x3,
    the diagonal phases of R moved into Q, then det fixed to 1."""
    a = _complex_gaussian(g, (count, 3, 3))
    q, r = np.linalg.qr(a)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[:, None, :]
    return _fix_det(q)


def smooth_su3(g: np.random.Generator, count: int, eps: float) -> np.ndarray:
    """``count`` links ``proj_SU(3)(exp(i eps G))`` with ``G = (X + X^H)/2``,
    X complex Gaussian.  exp of a Hermitian argument is formed through its
    eigendecomposition (so it is unitary to rounding); a polar step removes
    the remaining rounding and the det is fixed to 1."""
    x = _complex_gaussian(g, (count, 3, 3))
    h = 0.5 * (x + np.conj(np.swapaxes(x, -1, -2)))
    lam, vec = np.linalg.eigh(h)
    u = (vec * np.exp(1j * eps * lam)[:, None, :]) @ np.conj(np.swapaxes(vec, -1, -2))
    w, _, vh = np.linalg.svd(u)
    return _fix_det(w @ vh)


def gauge_field(dims, kind: str = "haar", seed: int = 0, eps: float = 0.3) -> np.ndarray:
    """Gauge field of shape (4, V, 3, 3); ``kind`` is "haar", "smooth" or "unit"."""
    V = volume(dims)
    if kind == "unit":
        return unit_gauge(dims)
    g = rng(seed)
    if kind == "haar":
        links = haar_su3(g, 4 * V)
    elif kind == "smooth":
        links = smooth_su3(g, 4 * V, eps)
    else:
        raise ValueError(f"unknown gauge kind {kind!r}")
    return np.ascontiguousarray(links.reshape(4, V, 3, 3))


def unit_gauge(dims) -> np.ndarray:
    """Free field: every link is the 3x3 identity."""
    V = volume(dims)
    u = np.zeros((4, V, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def gaussian_sources(dims, L: int, seed: int) -> np.ndarray:
    """``L`` complex Gaussian source vectors, shape (L, V, 4, 3)."""
    V = volume(dims)
    return np.ascontiguousarray(_complex_gaussian(rng(seed), (L, V, 4, 3)))


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """One Haar SU(3) matrix per site, shape (V, 3, 3)."""
    return haar_su3(rng(seed), volume(dims))
