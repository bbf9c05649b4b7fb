"""The arithmetic behind the tensor-core moment combination (csrc/combine_tc.cu),
checked on the CPU with exact integers (no GPU, no library code):

* the 56-bit fixed point of an FP64 element relative to a power-of-two
  scale, and its seven base-256 digits, reconstruct it to within half a
  unit of 2^-56 of the scale, and every digit is exact in bf16;
* a chunk of 256 slot products of two digits stays within 2^24, so an fp32
  accumulator holds it exactly;
* keeping the slice pairs p + q <= 6 of a dot product loses less than
  2^-55 of (scale x coefficient scale x number of terms), and the result
  agrees with the exact (rational) sum to that bound;
* the check program of the GPU test (tests/combine_tc_exact.cu) compiles
  for sm_103a.
"""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def exp_above(x):
    """e with 2^(e-1) <= x < 2^e for x > 0 (0 for x = 0)."""
    return int(np.frexp(x)[1]) if x > 0 else 0


def fixed56(x, e):
    """round(|x| 2^(56 - e)), ties up, as a Python integer; sign separately."""
    v = Fraction(abs(float(x))) * Fraction(2) ** (56 - e)
    return int(v + Fraction(1, 2)), (-1 if x < 0 else 1)


def digits(X):
    return [X >> 48] + [(X >> (48 - 8 * p)) & 255 for p in range(1, 7)]


def bf16_exact(d):
    f = np.float32(d)
    bits = f.view(np.uint32)
    return float((bits & np.uint32(0xFFFF0000)).view(np.float32)) == float(d)


def test_fixed_point_digits_reconstruct_and_are_bf16():
    g = np.random.default_rng(11)
    for _ in range(2000):
        x = (g.random() - 0.5) * 10.0 ** g.uniform(-30, 30)
        e = exp_above(abs(x)) + int(g.integers(0, 3))
        X, sg = fixed56(x, e)
        assert 0 <= X <= 2 ** 56
        d = digits(X)
        assert sum(dp << (48 - 8 * p) for p, dp in enumerate(d)) == X
        assert all(0 <= dp <= 256 for dp in d) and all(bf16_exact(dp) for dp in d)
        err = abs(Fraction(X) * Fraction(2) ** (e - 56) - Fraction(abs(x)))
        assert err <= Fraction(2) ** (e - 57)


def test_chunk_of_256_products_is_exact_in_fp32():
    # the largest digits on both sides: every partial sum an integer <= 2^24
    prods = np.full(256, 256 * 256, dtype=np.int64)
    assert int(prods.sum()) == 2 ** 24
    acc = np.float32(0)
    for p in prods:
        acc = np.float32(acc + np.float32(p))
    assert int(acc) == 2 ** 24
    g = np.random.default_rng(3)
    a = g.integers(-256, 257, 256)
    b = g.integers(-256, 257, 256)
    acc = np.float32(0)
    for u, v in zip(a, b):
        acc = np.float32(acc + np.float32(u * v))
    assert int(acc) == int(np.dot(a, b))


def test_truncated_slice_pairs_match_the_exact_sum():
    g = np.random.default_rng(5)
    K = 300
    r = (g.random(K) - 0.5) * 10.0 ** g.uniform(-6, 0, K)
    c = (g.random(K) - 0.5) * 10.0 ** g.uniform(0, 8, K)
    # one residual element per slot here; its scale is the slot's max
    e = [exp_above(abs(v)) for v in r]
    b = [float(np.ldexp(cv, es)) for cv, es in zip(c, e)]
    gexp = exp_above(max(abs(v) for v in b))
    A = [fixed56(v, es) for v, es in zip(r, e)]
    B = []
    for v in b:
        y = abs(v) * 2.0 ** (56 - gexp)
        B.append((int(np.rint(y)), -1 if v < 0 else 1))
    xh = xl = 0
    for p in range(7):
        for q in range(7 - p):
            s = sum(sa * sb * digits(Xa)[p] * digits(Xb)[q] for (Xa, sa), (Xb, sb) in zip(A, B))
            lv = p + q
            if lv <= 2:
                xh += s << (8 * (2 - lv))
            else:
                xl += s << (8 * (6 - lv))
    got = (Fraction(xh) * Fraction(2) ** -16 + Fraction(xl) * Fraction(2) ** -48) * Fraction(2) ** (gexp - 16)
    exact = sum(Fraction(float(cv)) * Fraction(float(rv)) for cv, rv in zip(c, r))
    bound = Fraction(2) ** (gexp - 55) * K
    assert abs(got - exact) <= bound
    # the kernel's last step, fma(xl, 2^-48, xh 2^-16) times powers of two,
    # rounds that once more (xh < 2^48 is exact in FP64; an fma rounds once)
    assert abs(xh) < 2 ** 48
    v = float(Fraction(float(xl)) * Fraction(2) ** -48 + Fraction(float(xh) * 2.0 ** -16)) * 2.0 ** (gexp - 16)
    assert abs(Fraction(v) - got) <= Fraction(2) ** -52 * abs(got) + abs(Fraction(float(xl)) - xl) * Fraction(2) ** (gexp - 64)
    assert abs(Fraction(v) - exact) <= 2 * bound


def test_check_program_compiles(tmp_path):
    nvcc = next((c for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc")
                 if c and os.path.exists(c)), None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "--expt-relaxed-constexpr", "-c", "-o", str(tmp_path / "cte.o"),
                    os.path.join(ROOT, "tests", "combine_tc_exact.cu")], check=True, timeout=900)
