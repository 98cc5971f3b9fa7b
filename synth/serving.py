"""Seeded request stream of the serving workload and its right-hand sides.

The stream is a Poisson process: exponential inter-arrival gaps with the given
mean rate, then for each request a mesh size n from MESHES, a Reynolds number
from REYNOLDS and 1..8 right-hand sides, each drawn uniformly by its own
splitmix64 stream (seed, seed + 1, seed + 2, seed + 3).  A request's
right-hand sides are the body loads of make_problem with homogeneous Dirichlet
conditions: uniform[-1, 1] draws on the non-Dirichlet velocity rows (column j
drawn with seed 1000 * rhs_seed + j), zero on Dirichlet rows and on the
pressure rows.  No arithmetic of the multigrid method lives here.
"""
from __future__ import annotations

import numpy as np

from .rng import exponential, uniform01, uniform_pm1

MESHES = (64, 128, 256, 384, 512)
REYNOLDS = (1.0, 10.0, 100.0)


def serving_stream(n_requests: int, rate: float = 200.0, seed: int = 0, max_nrhs: int = 8):
    """List of requests {t: arrival time in s from the stream's start, n, Re, nrhs, rhs_seed}."""
    t = np.cumsum(exponential(seed, n_requests, rate))
    un = uniform01(seed + 1, n_requests)
    ur = uniform01(seed + 2, n_requests)
    uk = uniform01(seed + 3, n_requests)
    out = []
    for i in range(n_requests):
        out.append(dict(t=float(t[i]), n=MESHES[int(un[i] * len(MESHES))], Re=REYNOLDS[int(ur[i] * len(REYNOLDS))],
                        nrhs=1 + int(uk[i] * max_nrhs), rhs_seed=1000 * seed + i))
    return out


def homogeneous_rhs(prob, nrhs: int, seed: int) -> np.ndarray:
    """N x nrhs body loads for a problem with homogeneous Dirichlet velocity
    conditions (no lifting), the right-hand sides make_problem(..., bc="zero",
    nrhs=nrhs, seed=seed) would draw for it."""
    dim, n_v = prob.dim, prob.n_v
    b = np.zeros((prob.N, nrhs))
    dirichlet = np.asarray(prob.v_dirichlet, dtype=bool)
    for j in range(nrhs):
        bu = uniform_pm1(1000 * seed + j, dim * n_v).reshape(dim, n_v)
        bu[:, dirichlet] = 0.0
        b[:dim * n_v, j] = bu.reshape(-1)
    return b
