"""End-to-end parity of the CUDA eigensolver with the oracle and with dense
/ ARPACK eigenvalues of the oracle operator."""
import json
import os

import numpy as np
import pytest

from tests._lib import gpu_module

import synthetic
from oracle import ss as oss

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "windows.json")

# 4^4 Haar links, kappa = 0.13: the interval brackets the eight smallest
# positive eigenvalues (0.3783 .. 0.3924; the next is 0.3935).
CFG1 = dict(dims=(4, 4, 4, 4), kind="haar", seed=1, eps=0.0, kappa=0.13, bc=-1,
            interval=(0.374, 0.3930), N=16, M=8, L=3, nprime=14, beta=0.3, src_seed=100)


@pytest.fixture(scope="module")
def ss():
    return gpu_module()


def _reference_spectrum(key):
    return np.array(json.load(open(GOLDEN))[key]["lowest_abs"])


def test_config1_against_oracle_and_dense(ss):
    c = CFG1
    U = synthetic.gauge_field(c["dims"], c["kind"], seed=c["seed"])
    src = synthetic.gaussian_sources(c["dims"], c["L"], seed=c["src_seed"])
    lat = ss.create_lattice(c["dims"], c["kappa"], c["bc"])
    ss.upload_gauge(lat, U)
    res = ss.ss_solve(lat, c["interval"], c["N"], c["M"], src, beta=c["beta"], nprime=c["nprime"])
    assert res.status == ss.OK, res.error
    ev, vec, rs, st = ss.ss_eigpairs(res)
    ref = oss.ss_solve(U, c["dims"], c["kappa"], c["bc"], c["interval"], c["N"], c["M"], src,
                       beta=c["beta"], Nprime=c["nprime"])
    exact = _reference_spectrum("haar_4x4x4x4_k0.13_s1")
    exact = exact[(exact >= c["interval"][0]) & (exact <= c["interval"][1])]
    assert len(exact) == 8
    assert len(ev) == len(ref["evals"]) == 8
    assert np.max(np.abs(ev - ref["evals"]) / np.abs(ref["evals"])) <= 1e-10
    assert np.max(np.abs(ev - exact) / np.abs(exact)) <= 1e-10
    assert np.max(rs) <= 1e-8
    assert st["rank"] == ref["rank"]
    # eigenvectors: residual recomputed by the oracle operator
    from oracle import wilson
    for k in range(len(ev)):
        x = vec[k]
        assert abs(np.linalg.norm(x) - 1.0) < 1e-12
        r = wilson.apply_H(U, x, c["kappa"], c["dims"], c["bc"]) - ev[k] * x
        assert abs(np.linalg.norm(r) - rs[k]) <= 1e-12 + 1e-6 * rs[k]
    # iteration counts are not unique in floating point (see the shifted-CG test)
    assert st["iterations"] <= 1.2 * int(ref["iters"].max()) + 2


def test_hankel_extraction_config1(ss):
    # Block Hankel pencil of the GPU moments (2M = 16 <= N): eigenvalues only,
    # accuracy bounded by the conditioning of the Hankel matrix.  Against the
    # exact spectrum and against the oracle's own Hankel extraction (SVD
    # reduction, numpy eig) of the oracle's moments of the same solve.
    c = CFG1
    U = synthetic.gauge_field(c["dims"], c["kind"], seed=c["seed"])
    src = synthetic.gaussian_sources(c["dims"], c["L"], seed=c["src_seed"])
    lat = ss.create_lattice(c["dims"], c["kappa"], c["bc"])
    ss.upload_gauge(lat, U)
    res = ss.ss_solve(lat, c["interval"], c["N"], c["M"], src, beta=c["beta"], nprime=c["nprime"],
                      extract=ss.EXTRACT_HANKEL)
    assert res.status == ss.OK, res.error
    ev, vec, rs, st = ss.ss_eigpairs(res, want_vectors=False)
    assert np.all(np.isnan(rs)) and st["matvecs_rr"] == 0
    exact = _reference_spectrum("haar_4x4x4x4_k0.13_s1")
    exact = np.sort(exact[(exact >= c["interval"][0]) & (exact <= c["interval"][1])])
    assert len(ev) == len(exact) == 8
    # the oracle's Hankel extraction of this case reaches 1.51e-5 (its own
    # moments, shifted CG at tol 1e-12), the conditioning of the Hankel matrix
    # (smallest kept eigenvalue ~1.4e-11 of the largest); the GPU reduction
    # (Hermitian eigendecomposition of H) reaches the same
    assert np.max(np.abs(ev - exact) / exact) <= 2e-5
    # the oracle's Hankel extraction on its own shifted-CG moments
    from oracle import contour, hankel, moments, shifted_cg, wilson
    a, b = c["interval"]
    g, r = contour.window_from_interval(a, b, c["N"], c["nprime"])
    z = contour.line_nodes(g, r, c["beta"], c["N"])
    zeta = contour.normalise(z, g, r)
    w = contour.weights_closed_form(zeta)
    A = lambda x: wilson.apply_H(U, x, c["kappa"], c["dims"], c["bc"])
    M2 = 2 * c["M"]
    ys = [shifted_cg.shifted_cg(A, v, z, tol=1e-12)["y"] for v in src]
    S = np.stack([np.stack([moments.moments(ys[l], w, zeta, M2)[k].reshape(-1) for l in range(c["L"])], axis=1)
                  for k in range(M2)])
    lam_o = g + r * hankel.block_hankel_eigs(src.reshape(c["L"], -1).T, S, rank_tol=1e-12)
    lam_o = np.sort(lam_o[(np.abs(lam_o.imag) < 1e-6) & (lam_o.real >= a) & (lam_o.real <= b)].real)
    assert len(lam_o) == 8
    # the two reductions of (nearly) the same moments agree far below their
    # common error against the exact spectrum
    assert np.max(np.abs(ev - lam_o) / lam_o) <= 1e-8
    with pytest.raises(Exception):
        ss.ss_eigpairs(res, want_vectors=True)
