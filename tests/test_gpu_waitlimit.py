"""The bounded waits of the bulk-copy-fed shift update: with its producer
held idle (SSQCD_TEST_UPDATE_STALL=1, read once by the library, so the case
runs in a child process) the consumers' first wait on a stage runs out; the
kernel sets its error flag and returns, the solve reports SSQCD_ERR_NOCONV
with the wait-limit message, and the context stays usable (a stencil
application afterwards is still correct).  No fault, trap or endless loop
is involved: every wait in the kernel has an iteration limit."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    sys.path.insert(0, {root!r})
    import paper_1004_0292_gb300 as ss
    import synthetic
    from oracle import contour, wilson
    dims = (2, 2, 2, 4)
    U = synthetic.gauge_field(dims, "haar", seed=3)
    v = synthetic.gaussian_sources(dims, 2, seed=4)
    z = contour.line_nodes(0.4, 0.05, 0.5, 4)
    lat = ss.create_lattice(dims, 0.12, 1)
    ss.upload_gauge(lat, U)
    try:
        code, y, iters, xi, _ = ss.shifted_cg(lat, z, v, tol=1e-10, precision=ss.FP64_DFSHIFT)
        msg = ss.lib().ssqcd_last_error().decode()
    except ss.SsqcdError as e:
        code, msg = e.code, str(e)
    print("CODE", code)
    print("MSG", msg)
    got = ss.apply_H(lat, v)
    ref = wilson.apply_H(U, v, 0.12, dims, 1)
    print("STENCIL_OK", bool(np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))))
""")


def test_update_wait_limit_reports_error():
    env = dict(os.environ, SSQCD_TEST_UPDATE_STALL="1")
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = dict(l.split(" ", 1) for l in out.stdout.strip().splitlines() if " " in l)
    assert int(lines["CODE"]) == 4  # SSQCD_ERR_NOCONV
    assert "wait hit its limit" in lines["MSG"]
    assert lines["STENCIL_OK"] == "True"
