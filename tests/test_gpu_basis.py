"""The Krylov-basis form of the shifted CG (stored seed residuals, moments
formed once from the backward coefficient recurrences) against the oracle's
shifted CG and moments (Section 2.2, Eq. 2), against the per-iteration
update form, and across the switch to the update form at the memory cap."""
import numpy as np
import pytest

from tests._lib import gpu_module

import bench
import synthetic
from oracle import contour, moments as omoments, shifted_cg, wilson

pytestmark = pytest.mark.gpu

DIMS, KAPPA, BC = (4, 4, 4, 4), 0.13, -1
N, M, L, NPRIME, BETA = 16, 8, 2, 8, 0.3


@pytest.fixture(scope="module")
def case():
    ss = gpu_module()
    U = synthetic.gauge_field(DIMS, "haar", seed=1)
    v = synthetic.gaussian_sources(DIMS, L, seed=5)
    lam = np.linalg.eigvalsh(wilson.dense_H(U, KAPPA, DIMS, BC))
    pos = np.sort(lam[lam > 0])
    a, b = pos[0] - 0.005, 0.5 * (pos[5] + pos[6])
    gamma, rho = contour.window_from_interval(a, b, N, NPRIME)
    z = contour.line_nodes(gamma, rho, BETA, N)
    zeta = contour.normalise(z, gamma, rho)
    w = contour.weights_closed_form(zeta)
    A = lambda x: wilson.apply_H(U, x, KAPPA, DIMS, BC)
    ref = []
    for l in range(L):
        y = shifted_cg.shifted_cg(A, v[l], z, tol=1e-12)["y"]
        ref.append(omoments.moments(y, w, zeta, M))
    # bound on |s_gpu - s_oracle| per moment: both solutions are converged
    # to 1e-12 relative, |y_gpu - y_ref| <= 2.5e-12 |v| / |Im z_j| (the
    # distance of z_j from the real spectrum), summed with the weights
    bound = [sum(abs(w[j]) * abs(zeta[j]) ** k * 2.5e-12 / abs(z[j].imag) for j in range(N)) for k in range(M)]
    return ss, U, v, (a, b), np.array(ref), np.array(bound)


def _check_moments(s, ref, bound, v):
    for l in range(L):
        vn = np.linalg.norm(v[l])
        for k in range(M):
            assert np.linalg.norm(s[l, k] - ref[l, k]) <= bound[k] * vn, (l, k)


@pytest.mark.parametrize("precision_name", ["FP64", "DF"])
def test_basis_moments_match_oracle(case, precision_name):
    ss, U, v, iv, ref, bound = case
    prec = getattr(ss, precision_name)
    lat = ss.create_lattice(DIMS, KAPPA, BC, precision=prec)
    ss.upload_gauge(lat, U)
    s, st = ss.ss_moments(lat, iv, N, M, v, beta=BETA, nprime=NPRIME)
    assert st["basis"] == 1 and st["basis_bytes"] > 0
    # float-float residuals carry 48 bits: 32 x the FP64 rounding
    _check_moments(s, ref, bound * (1.0 if prec == ss.FP64 else 32.0), v)


def test_basis_and_update_forms_agree(case):
    ss, U, v, iv, ref, bound = case
    lat = ss.create_lattice(DIMS, KAPPA, BC)
    ss.upload_gauge(lat, U)
    sb, stb = ss.ss_moments(lat, iv, N, M, v, beta=BETA, nprime=NPRIME, basis=1)
    su, stu = ss.ss_moments(lat, iv, N, M, v, beta=BETA, nprime=NPRIME, basis=0)
    assert stb["basis"] == 1 and stu["basis"] == 0
    # one seed recurrence, bit for bit: the same iteration counts
    assert stb["iterations"] == stu["iterations"]
    assert stb["shift_updates"] == stu["shift_updates"]
    _check_moments(su, ref, bound, v)
    # the two forms differ only in the rounding of the final combination
    for l in range(L):
        for k in range(M):
            assert np.linalg.norm(sb[l, k] - su[l, k]) <= 1e-13 * np.linalg.norm(su[l, k]) + 1e-3 * bound[k]


def test_switch_to_updates_at_the_memory_cap(case):
    ss, U, v, iv, ref, bound = case
    lat = ss.create_lattice(DIMS, KAPPA, BC)
    ss.upload_gauge(lat, U)
    n = 12 * synthetic.volume(DIMS)
    block = 16 * L * n * 16
    # room for the two first blocks only: the switch comes after 16 iterations
    s, st = ss.ss_moments(lat, iv, N, M, v, beta=BETA, nprime=NPRIME, basis=1, basis_max_bytes=2.5 * block)
    assert st["basis"] == 2
    assert st["iterations"] > 32
    _check_moments(s, ref, bound, v)
    # and the whole solve through the switch, against the update form and
    # the dense spectrum (the Ritz values nearest the window's edge are the
    # least accurate: the filter there is ~1/2)
    out = {}
    for cap in (2.5 * block, 0.0):
        res = ss.ss_solve(lat, iv, N, M, v, beta=BETA, nprime=NPRIME, basis=1 if cap else 0, basis_max_bytes=cap)
        assert res.status == ss.OK, res.error
        ev, vec, rs, st2 = ss.ss_eigpairs(res)
        assert st2["basis"] == (2 if cap else 0)
        out[cap] = (ev, rs)
    (e2, r2), (e0, r0) = out[2.5 * block], out[0.0]
    lam = np.linalg.eigvalsh(wilson.dense_H(U, KAPPA, DIMS, BC))
    inside = lam[(lam >= iv[0]) & (lam <= iv[1])]
    assert len(e2) == len(e0) == len(inside)
    assert np.max(np.abs(e2 - e0)) <= 1e-12 * np.max(np.abs(inside))
    assert np.max(np.abs(e2 - inside) / np.maximum(r2, 1e-14)) <= 1.0  # |theta - lambda| <= ||A x - theta x||
    assert np.max(np.abs(r2 - r0)) <= 1e-3 * np.max(r0) + 1e-14


def test_basis_eigenpairs_full_size_match_update_form():
    import torch
    ss = gpu_module()
    w = bench.CONFIG2
    U, src = bench.make_inputs(0, bench.CONFIG2)
    lat = ss.create_lattice(w["dims"], w["kappa"], w["bc_t"], stream=torch.cuda.Stream())
    ss.upload_gauge(lat, U)
    out = {}
    for basis in (1, 0):
        res = ss.ss_solve(lat, w["interval"], w["N"], w["M"], src, beta=w["beta"], nprime=w["nprime"], tol=w["tol"],
                          basis=basis)
        assert res.status == ss.OK, res.error
        ev, vec, rs, st = ss.ss_eigpairs(res, want_vectors=False)
        assert st["basis"] == basis
        out[basis] = (ev, rs, st)
    (e1, r1, s1), (e0, r0, s0) = out[1], out[0]
    assert s1["iterations"] == s0["iterations"]
    good1, good0 = e1[r1 <= 1e-8], e0[r0 <= 1e-8]
    assert len(good1) == len(good0) >= 12
    assert np.max(np.abs(good1 - good0)) <= 1e-12 * np.max(np.abs(good0))


def test_switch_to_updates_float_float(case):
    # the same switch with float-float residuals and shift vectors (SSQCD_DF)
    ss, U, v, iv, ref, bound = case
    lat = ss.create_lattice(DIMS, KAPPA, BC, precision=ss.DF)
    ss.upload_gauge(lat, U)
    n = 12 * synthetic.volume(DIMS)
    block = 16 * L * n * 16
    s, st = ss.ss_moments(lat, iv, N, M, v, beta=BETA, nprime=NPRIME, basis=1, basis_max_bytes=2.5 * block)
    assert st["basis"] == 2
    _check_moments(s, ref, bound * 32.0, v)


def test_zero_source_has_zero_moments(case):
    # a zero source starts frozen: no residual of it enters, its moments are 0
    ss, U, v, iv, ref, bound = case
    lat = ss.create_lattice(DIMS, KAPPA, BC)
    ss.upload_gauge(lat, U)
    v2 = v.copy()
    v2[1] = 0.0
    s, st = ss.ss_moments(lat, iv, N, M, v2, beta=BETA, nprime=NPRIME)
    assert st["basis"] == 1
    assert np.all(s[1] == 0.0)
    for k in range(M):
        assert np.linalg.norm(s[0, k] - ref[0, k]) <= bound[k] * np.linalg.norm(v[0])
