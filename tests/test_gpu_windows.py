"""Multi-window tiling with point reuse and the circle contour, against the
oracle (same readings) and the dense spectrum."""
import json
import os

import numpy as np
import pytest

from tests._lib import gpu_module

import synthetic
from oracle import ss as oss

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "windows.json")


@pytest.fixture(scope="module")
def setup():
    import torch
    ss = gpu_module()
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, "haar", seed=1)
    src = synthetic.gaussian_sources(dims, 3, seed=100)
    lat = ss.create_lattice(dims, 0.13, -1, stream=torch.cuda.Stream())
    ss.upload_gauge(lat, U)
    lam = np.array(json.load(open(GOLDEN))["haar_4x4x4x4_k0.13_s1"]["lowest_abs"])
    return ss, dims, U, src, lat, lam


def test_two_windows_reuse_points_and_match_oracle(setup):
    ss, dims, U, src, lat, lam = setup
    a, b, N, M, Np, K = 0.374, 0.3930, 16, 8, 12, 2
    res = ss.ss_solve(lat, (a, b), N, M, src, beta=0.3, nprime=Np, windows=K)
    assert res.status == ss.OK, res.error
    ev, vec, rs, st = ss.ss_eigpairs(res)
    assert st["points"] == N + (K - 1) * (Np - 2)     # Section 3: shift by N' - 2 points
    ref = oss.ss_solve(U, dims, 0.13, -1, (a, b), N, M, src, beta=0.3, Nprime=Np, windows=K)
    assert ref["points"] == st["points"]
    exact = np.sort(lam[(lam >= a) & (lam <= b)])
    assert len(ev) == len(ref["evals"]) == len(exact) == 8
    assert np.max(np.abs(ev - ref["evals"]) / ref["evals"]) <= 1e-10
    assert np.max(np.abs(ev - exact) / exact) <= 1e-10
    assert np.max(rs) <= 1e-8


def test_circle_contour_matches_oracle(setup):
    ss, dims, U, src, lat, lam = setup
    a, b, N, M = 0.374, 0.3930, 32, 8
    res = ss.ss_solve(lat, (a, b), N, M, src, path=ss.PATH_CIRCLE)
    assert res.status == ss.OK, res.error
    ev, vec, rs, st = ss.ss_eigpairs(res)
    ref = oss.ss_solve(U, dims, 0.13, -1, (a, b), N, M, src, path="circle")
    assert len(ev) == len(ref["evals"])
    assert np.max(np.abs(ev - ref["evals"]) / ref["evals"]) <= 1e-10
    exact = np.sort(lam[(lam >= a) & (lam <= b)])
    good = rs <= 1e-8
    # every well-resolved Ritz pair is an eigenpair of the dense spectrum
    for e in ev[good]:
        assert np.min(np.abs(exact - e)) / e <= 1e-10


def test_window_list_one_seed_run_matches_separate_windows(setup):
    """ssqcd_ss_solve_windows: a window on each side of the spectral gap
    around zero out of one shifted-CG run.  Each window's points, moments and
    Rayleigh-Ritz are those of its own solve, so the eigenvalues equal the
    separate solves' and the oracle's, and the dense spectrum's to 1e-10;
    running the sources one at a time (source_block = 1) changes only the
    rounding."""
    ss, dims, U, src, lat, lam = setup
    wins = [(-0.3932, -0.3785), (0.374, 0.3930)]
    N, M, Np = 16, 8, 14
    res = ss.ss_solve_windows(lat, wins, N, M, src, beta=0.3, nprime=Np)
    assert res.status == ss.OK, res.error
    ev, vec, rs, st = ss.ss_eigpairs(res)
    assert st["points"] == 2 * N
    exact = np.sort(np.concatenate([lam[(lam >= a) & (lam <= b)] for a, b in wins]))
    assert len(exact) == 16 and len(ev) == 16
    assert np.max(np.abs(ev - exact) / np.abs(exact)) <= 1e-10
    assert np.max(rs) <= 1e-8
    assert st["n_converged"] == 16 == st["n_accepted"]
    sep = []
    for a, b in wins:
        r1 = ss.ss_solve(lat, (a, b), N, M, src, beta=0.3, nprime=Np)
        assert r1.status == ss.OK, r1.error
        e1, _, _, _ = ss.ss_eigpairs(r1, want_vectors=False)
        ref = oss.ss_solve(U, dims, 0.13, -1, (a, b), N, M, src, beta=0.3, Nprime=Np)
        assert np.max(np.abs(e1 - ref["evals"]) / np.abs(ref["evals"])) <= 1e-10
        sep.append(e1)
    sep = np.sort(np.concatenate(sep))
    assert np.max(np.abs(ev - sep) / np.abs(sep)) <= 1e-12
    res_b = ss.ss_solve_windows(lat, wins, N, M, src, beta=0.3, nprime=Np, source_block=1)
    assert res_b.status == ss.OK, res_b.error
    eb, _, rb, stb = ss.ss_eigpairs(res_b, want_vectors=False)
    assert len(eb) == 16
    assert np.max(np.abs(eb - ev) / np.abs(ev)) <= 1e-11
    assert np.max(rb) <= 1e-8
    # the blocks' runs side by side on their own streams (block_streams):
    # every source's arithmetic is the same, so the result is bit-identical
    for bs in (2, 3):
        res_s = ss.ss_solve_windows(lat, wins, N, M, src, beta=0.3, nprime=Np, source_block=1, block_streams=bs)
        assert res_s.status == ss.OK, res_s.error
        es, _, rss, sts = ss.ss_eigpairs(res_s, want_vectors=False)
        assert np.array_equal(es, eb) and np.array_equal(rss, rb)
        assert sts["iterations"] == stb["iterations"]


def test_window_list_rejects_bad_intervals(setup):
    ss, dims, U, src, lat, lam = setup
    with pytest.raises(ss.SsqcdError):
        ss.ss_solve_windows(lat, [(0.39, 0.38)], 16, 8, src)
    with pytest.raises(ss.SsqcdError):
        ss.ss_solve_windows(lat, [], 16, 8, src)
