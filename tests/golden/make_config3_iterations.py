"""Write ``config3_iterations.json``: how many shifted-CG iterations the
oracle needs on the 16^3 x 32 workload, for one source.

Workload: 16^3 x 32 lattice, smooth links exp(i 0.5 G) (seed 4), kappa
0.135, antiperiodic time; two line-pair windows (Section 3) on the two sides
of the spectral gap around zero, [-0.1095, -0.0765] and [0.0769, 0.1081],
N = 32 points each (64 shifts), N' = 20, beta = 0.3; source 0 of the eight
complex Gaussian sources (seed 300); tolerance 1e-12 (Section 4).

The oracle's shifted CG (Section 2.2) runs to the end on the host with the
oracle's matrix-free Wilson operator; the file records the seed iterations
and each shift's freeze iteration.  The CUDA path plays no part.  bench.py's
host-side baseline uses the count to scale the oracle's measured cost per
iteration to a whole solve.  Run: ``python
tests/golden/make_config3_iterations.py`` (about two hours on eight cores,
3.2 GB of memory).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synthetic  # noqa: E402
from oracle import contour, shifted_cg, wilson  # noqa: E402

PARAMS = dict(dims=[16, 16, 16, 32], kind="smooth", gauge_seed=4, eps=0.5, kappa=0.135, bc_t=-1,
              windows=[[-0.1095, -0.0765], [0.0769, 0.1081]], N=32, nprime=20, beta=0.3,
              src_seed=300, L=8, source=0, tol=1e-12)


def main():
    p = PARAMS
    t0 = time.time()
    dims = tuple(p["dims"])
    U = synthetic.gauge_field(dims, p["kind"], seed=p["gauge_seed"], eps=p["eps"])
    v = synthetic.gaussian_sources(dims, p["L"], seed=p["src_seed"])[p["source"]]
    z = []
    for a, b in p["windows"]:
        gamma, rho = contour.window_from_interval(a, b, p["N"], p["nprime"])
        z.append(contour.line_nodes(gamma, rho, p["beta"], p["N"]))
    z = np.concatenate(z)
    out = shifted_cg.shifted_cg(lambda x: wilson.apply_H(U, x, p["kappa"], dims, p["bc_t"]), v, z,
                                tol=p["tol"])
    res = {"params": p, "seed_iterations": int(out["matvecs"]),
           "shift_iterations": [int(i) for i in out["iters"]],
           "host_seconds": time.time() - t0,
           "method": "oracle.shifted_cg on the host, oracle.wilson operator"}
    with open(os.path.join(HERE, "config3_iterations.json"), "w") as f:
        json.dump(res, f, indent=1)
    print("done", res["seed_iterations"], res["host_seconds"], flush=True)


if __name__ == "__main__":
    main()
