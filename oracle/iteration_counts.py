"""Writes iteration_counts.json: the iterations the oracle's own fp64
Jacobi-PCG (single-thread pinned build, x0 = 0, Eq. 2 at 1e-10) takes on the
benchmark's full-size systems.  The CPU baseline times a bounded sample of
iterations and scales it by these counts, so that it needs neither the GPU's
counts nor an hours-long CPU solve per run.  Run once (it takes tens of
minutes on one core):  python oracle/iteration_counts.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as O  # noqa: E402

SYSTEMS = {  # name: (dim, degree, cells, jitter, diag_mode, seed, Dirichlet id)
    "2D-P1-jittered-1024": (2, 1, 1024, 1, 1, 1, O.G_X2_Y2),
    "2D-P2-jittered-1024": (2, 2, 1024, 1, 1, 1, O.G_X2_Y2),
    "3D-P1-Kuhn-128": (3, 1, 128, 0, 0, 0, O.G_X2_Y2_2Z2),
    "3D-P2-Kuhn-64": (3, 2, 64, 0, 0, 0, O.G_X2_Y2_2Z2),
}
TOL = 1e-10


def main():
    out = {}
    for name, (dim, deg, cells, jit, dm, seed, gid) in SYSTEMS.items():
        t0 = time.time()
        s = O.System(dim, deg, cells, jit, dm, seed).assemble()
        rp, ci, v = s.k_ii()
        b = s.lift(s.eval_g(gid))[:, 0]
        x, st, it, rel = O.pcg(rp, ci, v, b, tol=TOL)
        out[name] = {"n": len(rp) - 1, "nnz": int(rp[-1]), "tol": TOL, "status": st, "iterations": it,
                     "relres": rel}
        print(name, out[name], f"{time.time() - t0:.0f} s", flush=True)
    with open(os.path.join(HERE, "iteration_counts.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
