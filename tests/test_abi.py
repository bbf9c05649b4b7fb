"""Host-side checks of the C-ABI library (no GPU needed)."""
import ctypes
import subprocess

import numpy as np
import pytest

from tests._lib import built, header_functions

import synthetic
from oracle import contour as ocontour


@pytest.fixture(scope="module")
def ss():
    built()
    import paper_1004_0292_gb300 as ss
    return ss


def test_every_declared_symbol_is_exported(ss):
    names = header_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(ss.library_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and they are dynamic symbols with C linkage
    out = subprocess.run(["nm", "-D", "--defined-only", ss.library_path()], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    assert set(names) <= exported


def test_small_eigh_matches_lapack(ss):
    g = synthetic.rng(4)
    for m in (1, 2, 5, 16, 33, 64):
        x = g.standard_normal((m, m)) + 1j * g.standard_normal((m, m))
        a = x + x.conj().T
        ev, vec = ss.small_eigh(a)
        ref = np.linalg.eigvalsh(a)
        assert np.max(np.abs(ev - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
        assert np.allclose(vec.conj().T @ vec, np.eye(m), atol=1e-13)
        assert np.allclose(a @ vec, vec * ev[None, :], atol=1e-12 * max(1.0, np.max(np.abs(ref))))


def test_small_eigh_degenerate_and_diagonal(ss):
    # repeated eigenvalues and an already tridiagonal / diagonal input
    d = np.array([1.0, 1.0, 1.0, -2.0, 3.0, 3.0])
    q, _ = np.linalg.qr(synthetic.rng(1).standard_normal((6, 6)) + 1j * synthetic.rng(2).standard_normal((6, 6)))
    a = q @ np.diag(d) @ q.conj().T
    ev, vec = ss.small_eigh(a)
    assert np.allclose(ev, np.sort(d), atol=1e-13)
    assert np.allclose(a @ vec, vec * ev[None, :], atol=1e-12)
    ev2, _ = ss.small_eigh(np.diag(d).astype(complex))
    assert np.allclose(ev2, np.sort(d))


@pytest.mark.parametrize("N,beta", [(8, 0.2), (16, 0.5), (32, 0.2), (64, 0.3)])
def test_contour_matches_oracle(ss, N, beta):
    z, w = ss.contour(ss.PATH_LINES, 0.1, 0.02, beta, N)
    zo = ocontour.line_nodes(0.1, 0.02, beta, N)
    wo = ocontour.weights_closed_form(ocontour.normalise(zo, 0.1, 0.02))
    assert np.allclose(z, zo, rtol=0, atol=1e-15)
    assert np.max(np.abs(w - wo)) <= 1e-12 * np.max(np.abs(wo))


def test_contour_circle_weights(ss):
    z, w = ss.contour(ss.PATH_CIRCLE, -0.3, 0.5, 0.0, 32)
    zeta = (z + 0.3) / 0.5
    assert np.allclose(w, zeta / 32, atol=1e-15)


def test_argument_errors(ss):
    with pytest.raises(ss.SsqcdError) as e:
        ss.contour(ss.PATH_LINES, 0.0, 1.0, 0.3, 7)
    assert e.value.code == ss.ERR_ARG
    with pytest.raises(ss.SsqcdError):
        ss.contour(ss.PATH_LINES, 0.0, -1.0, 0.3, 8)
    with pytest.raises(ss.SsqcdError):
        ss.create_lattice((4, 4, 0, 4), 0.1)
    with pytest.raises(ss.SsqcdError):
        ss.create_lattice((4, 4, 4, 4), 0.1, bc_t=0)


def test_struct_layouts_match_the_header(ss, tmp_path):
    # the ctypes mirrors of ssqcd_opts / ssqcd_stats against a C compiler's
    # view of include/ssqcd.h (sizes and every field offset)
    import os
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ssqcd.h"', "int main(void) {"]
    for cname, py in (("ssqcd_opts", ss.Opts), ("ssqcd_stats", ss.Stats)):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c_side = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in (("ssqcd_opts", ss.Opts), ("ssqcd_stats", ss.Stats)):
        assert c_side[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert c_side[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_small_eigh_clustered_and_large(ss):
    # the Rayleigh-Ritz sizes (m up to M L = 128 and beyond) with tight
    # eigenvalue clusters, as the projected matrices of a window have
    g = synthetic.rng(9)
    for m, spread in ((128, 1e-9), (200, 1e-3), (96, 0.0)):
        d = np.concatenate([0.1 + spread * g.standard_normal(m // 2), g.standard_normal(m - m // 2)])
        q, _ = np.linalg.qr(g.standard_normal((m, m)) + 1j * g.standard_normal((m, m)))
        a = q @ np.diag(d) @ q.conj().T
        ev, vec = ss.small_eigh(a)
        assert np.max(np.abs(ev - np.sort(d))) <= 1e-13 * max(1.0, np.max(np.abs(d)))
        assert np.allclose(vec.conj().T @ vec, np.eye(m), atol=1e-12)
        assert np.max(np.abs(a @ vec - vec * ev[None, :])) <= 1e-12 * max(1.0, np.max(np.abs(d)))
