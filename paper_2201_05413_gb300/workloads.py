"""Seeded synthetic workloads (input generation only: no arithmetic of the
method lives here).  Shared by the tests, the benchmark and users who want the
same request mixes.

cfg5 serving mix: Poisson arrivals; 70% 2D jittered meshes with n^2 cells,
n log-uniform in [32, 1024]; 30% 3D Kuhn meshes with n^3 cells, n log-uniform
in [16, 128]; P1/P2 50/50; 1-8 right-hand sides; Dirichlet data: harmonic
basis coefficients N(0,1) (2D) or linear coefficients N(0,1) (3D).  Per-request
mesh seed = request index.
"""
from __future__ import annotations

import numpy as np

G_HARMONIC, G_LINEAR = 4, 3


def serving_requests(count, seed=4, rate_per_s=None, max_cells_2d=1024, max_cells_3d=128):
    """List of request dicts (spec, k, gid, coef, t_arrival_s)."""
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for i in range(count):
        if rng.random() < 0.7:
            dim = 2
            cells = int(round(np.exp(rng.uniform(np.log(32), np.log(max_cells_2d)))))
        else:
            dim = 3
            cells = int(round(np.exp(rng.uniform(np.log(16), np.log(max_cells_3d)))))
        degree = 1 if rng.random() < 0.5 else 2
        k = int(rng.integers(1, 9))
        gid = G_HARMONIC if dim == 2 else G_LINEAR
        coef = rng.standard_normal((k, 10 if dim == 2 else 4))
        if rate_per_s:
            t += rng.exponential(1.0 / rate_per_s)
        reqs.append({"dim": dim, "degree": degree, "cells": cells,
                     "jitter": 1 if dim == 2 else 0, "diag_mode": 1 if dim == 2 else 0,
                     "seed": i, "k": k, "gid": gid, "coef": coef, "t": t})
    return reqs


def multi_rhs_coefficients(k, seed=3):
    """cfg4: N(0,1) coefficients of the 10 harmonic-basis functions per column."""
    return np.random.default_rng(seed).standard_normal((k, 10))
