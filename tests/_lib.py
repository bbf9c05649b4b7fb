"""Test helpers: build the library once per session."""
import functools
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@functools.lru_cache(maxsize=1)
def built():
    from paper_1004_0292_gb300 import build
    return build.build()


def header_functions():
    """Names of every function declared in include/*.h."""
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names += re.findall(r"\b(ssqcd_\w+)\s*\(", text)
    return sorted(set(names))


def gpu_module():
    """The binding with the library built; fails (not skips) without a GPU."""
    import pytest
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    built()
    import paper_1004_0292_gb300 as ss
    return ss


def fp16_rounded_links(U):
    """The links the mixed path sees: rows 0 and 1 rounded to FP16 (re, im
    separately), row 2 rebuilt as conj(row0 x row1), all in FP64."""
    import numpy as np
    r01 = U[..., :2, :]
    r01 = (r01.real.astype(np.float16).astype(np.float64)
           + 1j * r01.imag.astype(np.float16).astype(np.float64))
    r2 = np.conj(np.cross(r01[..., 0, :], r01[..., 1, :]))
    return np.concatenate([r01, r2[..., None, :]], axis=-2)
