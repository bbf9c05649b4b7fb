"""Moments with real coefficients (the line pair about a real centre is
closed under conjugation, so the coefficient of every stored residual is
real): the library's combination with real coefficients against the same
moments combined with the complex coefficients (SSQCD_REAL_MOMENTS=0, read
once by the library, so that case runs in a child process), and against the
oracle's Eq. 2 sums; FP64 and float-float lattices; the circle contour,
whose points are not exact conjugates, keeps the complex combination."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from tests._lib import gpu_module

import synthetic
from oracle import contour, moments as omoments, shifted_cg, wilson

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASE = dict(dims=(4, 4, 4, 4), kappa=0.13, bc=-1, seed=1, src_seed=100, L=2, interval=(0.374, 0.3930), N=16, M=8,
            beta=0.3, nprime=12)

CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    sys.path.insert(0, {root!r})
    import paper_1004_0292_gb300 as ss
    import synthetic
    c = {case!r}
    U = synthetic.gauge_field(c["dims"], "haar", seed=c["seed"])
    src = synthetic.gaussian_sources(c["dims"], c["L"], seed=c["src_seed"])
    for name, prec in (("fp64", ss.FP64), ("df", ss.DF)):
        lat = ss.create_lattice(c["dims"], c["kappa"], c["bc"], precision=prec)
        ss.upload_gauge(lat, U)
        s, st = ss.ss_moments(lat, c["interval"], c["N"], c["M"], src, beta=c["beta"], nprime=c["nprime"])
        np.save({out!r} + "_" + name + ".npy", s)
        print("REAL_" + name, st["real_moments"])
""")


def _moments(ss, prec, path=None):
    c = CASE
    U = synthetic.gauge_field(c["dims"], "haar", seed=c["seed"])
    src = synthetic.gaussian_sources(c["dims"], c["L"], seed=c["src_seed"])
    lat = ss.create_lattice(c["dims"], c["kappa"], c["bc"], precision=prec)
    ss.upload_gauge(lat, U)
    kw = {} if path is None else dict(path=path)
    return ss.ss_moments(lat, c["interval"], c["N"], c["M"], src, beta=c["beta"], nprime=c["nprime"], **kw)


def test_real_coefficient_moments_match_complex_and_oracle(tmp_path):
    ss = gpu_module()
    out = str(tmp_path / "complex")
    env = dict(os.environ, SSQCD_REAL_MOMENTS="0")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, case=CASE, out=out)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    flags = dict(l.split(" ", 1) for l in r.stdout.strip().splitlines() if " " in l)
    assert flags["REAL_fp64"] == "0" and flags["REAL_df"] == "0"
    # the oracle's Eq. 2 sums over its own shifted-CG solutions
    c = CASE
    U = synthetic.gauge_field(c["dims"], "haar", seed=c["seed"])
    src = synthetic.gaussian_sources(c["dims"], c["L"], seed=c["src_seed"])
    g, rho = contour.window_from_interval(*c["interval"], c["N"], c["nprime"])
    z = contour.line_nodes(g, rho, c["beta"], c["N"])
    zeta = contour.normalise(z, g, rho)
    w = contour.weights_closed_form(zeta)
    A = lambda x: wilson.apply_H(U, x, c["kappa"], c["dims"], c["bc"])
    ref = np.stack([omoments.moments(shifted_cg.shifted_cg(A, v, z, tol=1e-12)["y"], w, zeta, c["M"]) for v in src])
    # the shifted-CG error bound of each moment (relative tolerance 1e-12 of
    # every shift's system, weighted as in Eq. 2)
    bound = np.array([sum(abs(w[j]) * abs(zeta[j]) ** k * 2.5e-12 / abs(z[j].imag) for j in range(c["N"]))
                      for k in range(c["M"])])
    for name, prec in (("fp64", ss.FP64), ("df", ss.DF)):
        s_real, st = _moments(ss, prec)
        assert st["real_moments"] == 1
        s_cplx = np.load(out + "_" + name + ".npy")
        widen = 1.0 if name == "fp64" else 32.0  # float-float residuals: 48 bits
        for l in range(c["L"]):
            vn = np.linalg.norm(src[l])
            for k in range(c["M"]):
                # against the oracle, within the CG error bound
                assert np.linalg.norm(s_real[l, k] - ref[l, k]) <= widen * bound[k] * vn, (name, l, k)
                # against the complex combination: rounding only
                d = np.linalg.norm(s_real[l, k] - s_cplx[l, k])
                assert d <= 1e-13 * widen * np.linalg.norm(s_cplx[l, k]) + 1e-3 * bound[k] * vn, (name, l, k)


def test_circle_contour_keeps_complex_coefficients():
    ss = gpu_module()
    s, st = _moments(ss, ss.FP64, path=ss.PATH_CIRCLE)
    assert st["real_moments"] == 0
