"""The moment combination on the tensor cores (csrc/combine_tc.cu).

* Exactness of the kernel: tests/combine_tc_exact.cu, built here with nvcc
  for sm_103a, runs the library's kernels on synthetic stored residuals
  (several tiles, a ragged last K-step, five of sixteen outputs, a single
  slot, NaN in the slots that must not be read) and compares them bit for
  bit with a CPU copy of the same integer arithmetic, and with the
  long-double sum.
* In the library: the moments of the line-pair contour with the tensor-core
  combination (the default for FP64 residuals) against the FP64-pipe kernel
  (SSQCD_MOMENTS_TC=0, read once by the library, so in a child process).
"""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

from tests._lib import gpu_module
from tests.test_gpu_real_moments import CASE, CHILD, ROOT, _moments

pytestmark = pytest.mark.gpu


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.fail("nvcc not found")


def test_tensor_core_combination_is_exact(tmp_path):
    exe = str(tmp_path / "combine_tc_exact")
    subprocess.run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "--expt-relaxed-constexpr", "-o", exe, os.path.join(ROOT, "tests", "combine_tc_exact.cu")],
                   check=True, timeout=900)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "checks: passed" in r.stdout, r.stdout[-3000:] + r.stderr[-2000:]
    assert r.stdout.count("bitwise mismatches vs CPU copy: 0 of") == 3, r.stdout


def test_tensor_core_moments_match_the_fp64_pipe_kernel(tmp_path):
    ss = gpu_module()
    out = str(tmp_path / "fp64pipe")
    env = dict(os.environ, SSQCD_MOMENTS_TC="0")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, case=CASE, out=out)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    s_pipe = np.load(out + "_fp64.npy")
    s_tc, st = _moments(ss, ss.FP64)
    assert st["real_moments"] == 1
    for l in range(CASE["L"]):
        for k in range(CASE["M"]):
            ref = np.linalg.norm(s_pipe[l, k])
            # both are the FP64 combination: the tensor-core form within
            # 2^-56 of the operand scales, the FP64 sum within its rounding
            assert np.linalg.norm(s_tc[l, k] - s_pipe[l, k]) <= 1e-12 * ref, (l, k)
