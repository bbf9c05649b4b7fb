"""The benchmark's headline workload (16^3 x 32, kappa 0.135, smooth links
eps 0.5, L = 8, M = 16, two line-pair windows of N = 32 points on the two
sides of the spectral gap, source blocks of two) in the launch configuration
bench.py times.  The oracle cannot solve a lattice of this size, so the
eigenpairs are certified by what the paper and the mathematics fix:

* every accepted pair's residual ||A x - theta x|| recomputed on the host
  with the oracle's Wilson operator is <= 1e-8 (Section 4's residual), and
  for a Hermitian A such a residual puts an eigenvalue of A within
  ||r||^2 / gap of theta (Kato-Temple), checked against the gap to the
  neighbouring computed eigenvalues;
* the eigenvectors are orthonormal;
* the same windows solved at another beta (another filter, another
  iteration count) give the same eigenvalue set: the count of eigenvalues
  in the windows does not depend on the contour;
* the float-float solve gives the same eigenvalues.
"""
import numpy as np
import pytest

from tests._lib import gpu_module

import bench
from oracle import wilson

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run():
    import torch
    ss = gpu_module()
    w = bench.WORKLOAD
    U, src = bench.make_inputs(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    lat = ss.create_lattice(w["dims"], w["kappa"], w["bc_t"], stream=stream)
    ss.upload_gauge(lat, torch.from_numpy(U).cuda())
    src_d = torch.from_numpy(src).cuda()
    ev, rs, st, vec = bench.windows_step(ss, lat, src_d, w, want_vectors=True)
    yield ss, w, U, src_d, lat, stream, ev, rs, st, vec
    torch.cuda.set_stream(torch.cuda.default_stream())


def test_config3_eigenpairs_certified_by_oracle_residuals(run):
    ss, w, U, src_d, lat, stream, ev, rs, st, vec = run
    good = rs <= 1e-8
    assert good.sum() == 48, (ev, rs)
    assert st["n_converged"] == 48 and st["n_accepted"] == len(ev)
    # the spurious Ritz values of the filtered noise (residual ~0.5) are the
    # only other accepted values
    assert np.all(rs[~good] > 1e-2)
    X = vec[good]
    theta = ev[good]
    V = X.shape[1]
    G = X.reshape(len(theta), -1).conj() @ X.reshape(len(theta), -1).T
    assert np.max(np.abs(np.diag(G) - 1.0)) <= 1e-10
    # within a window the Ritz vectors are orthonormal by construction; across
    # windows two eigenvectors' overlap is bounded by (||r_i|| + ||r_j||) /
    # |theta_i - theta_j| (A Hermitian)
    rsg = rs[good]
    off = np.abs(G - np.diag(np.diag(G)))
    bound = 1e-10 + (rsg[:, None] + rsg[None, :]) / np.maximum(np.abs(theta[:, None] - theta[None, :]), 1e-300)
    np.fill_diagonal(bound, np.inf)
    assert np.all(off <= bound)
    res = np.empty(len(theta))
    for i0 in range(0, len(theta), 8):
        AX = wilson.apply_H(U, X[i0:i0 + 8], w["kappa"], w["dims"], w["bc_t"])
        R = AX - theta[i0:i0 + 8, None, None, None] * X[i0:i0 + 8]
        res[i0:i0 + 8] = np.linalg.norm(R.reshape(len(R), -1), axis=1)
    assert np.max(res) <= 1e-8, res
    # the library's residuals are the same numbers
    assert np.max(np.abs(res - rs[good])) <= 1e-9
    # Kato-Temple: theta is within ||r||^2 / gap of an eigenvalue of A (gap to
    # the neighbouring computed eigenvalues, all > 1e-5 here)
    srt = np.sort(theta)
    gaps = np.minimum(np.r_[np.inf, np.diff(srt)], np.r_[np.diff(srt), np.inf])
    order = np.argsort(theta)
    bound = res[order] ** 2 / gaps
    assert np.min(gaps) > 1e-5
    assert np.max(bound / np.abs(srt)) <= 1e-10
    # 24 eigenvalues on each side of the gap, in the two windows
    (a0, b0), (a1, b1) = w["windows"]
    assert np.sum((theta >= a0) & (theta <= b0)) == 24
    assert np.sum((theta >= a1) & (theta <= b1)) == 24


def test_config3_same_eigenvalues_at_another_beta_and_in_float_float(run):
    import torch
    ss, w, U, src_d, lat, stream, ev, rs, st, vec = run
    ref = np.sort(ev[rs <= 1e-8])
    w2 = dict(w, beta=0.25)
    ev2, rs2, st2 = bench.windows_step(ss, lat, src_d, w2)
    assert st2["iterations"] != st["iterations"]
    got = np.sort(ev2[rs2 <= 1e-7])
    assert len(got) == len(ref) == 48
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-10
    lat_df = ss.create_lattice(w["dims"], w["kappa"], w["bc_t"], precision=ss.DF, stream=stream)
    ss.upload_gauge(lat_df, torch.from_numpy(U).cuda())
    ev3, rs3, st3 = bench.windows_step(ss, lat_df, src_d, w)
    # float-float (48-bit significand) residuals sit at 1e-10 .. 1e-8; a pair
    # next to a spurious Ritz value can land just above 1e-8 with some
    # summation orders, so the set is compared at 1e-7 and at least 46 of
    # the 48 must meet 1e-8
    got3 = np.sort(ev3[rs3 <= 1e-7])
    assert len(got3) == 48 and np.sum(rs3 <= 1e-8) >= 46
    assert np.max(np.abs(got3 - ref) / np.abs(ref)) <= 1e-10
