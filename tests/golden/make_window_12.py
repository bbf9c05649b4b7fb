"""Write ``window_12.json``: the low-lying spectrum of the seeded 12^4 field
(smooth links, eps 0.4, seed 3, kappa 0.13, antiperiodic time).

Run: ``python tests/golden/make_window_12.py`` (ARPACK on A^2 with the
oracle's matrix-free Wilson operator; ~10 minutes on one core).  The CUDA
path plays no part.  The stored eigenvalues place the accepted interval of
the 12^4 parity test and are its eigenvalue reference.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from make_windows import low_spectrum_arpack  # noqa: E402


def main():
    t = time.time()
    dims, kind, seed, eps, kappa, bc = (12, 12, 12, 12), "smooth", 3, 0.4, 0.13, -1
    lam, res = low_spectrum_arpack(dims, kind, seed, eps, kappa, bc, 48)
    out = {"smooth_12x12x12x12_e0.4_k0.13_s3": {
        "dims": list(dims), "kind": kind, "seed": seed, "eps": eps, "kappa": kappa, "bc_t": bc,
        "lowest_abs": lam.tolist(), "max_residual": res,
        "method": "ARPACK on A^2, signs split on the subspace"}}
    with open(os.path.join(HERE, "window_12.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("12^4 done", time.time() - t, res, flush=True)


if __name__ == "__main__":
    main()
