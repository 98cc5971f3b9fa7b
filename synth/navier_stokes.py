"""Steady Navier-Stokes lid cavity by Picard iteration (Section 6.2's test systems).

The paper tests AMG on "the last linear system within a converged Picard
sequence" stopped when the 2-norm of the nonlinear residual falls below 1e-8.
Each Picard step is the Oseen problem whose wind is the current discrete
velocity (make_problem with wind_nodal), solved here by a sparse direct solve:
this builds the test systems, it is not part of the multigrid method.
Domain (-1,1)^2, leaky lid u = (1, 0) on y = 1, zero body force, viscosity nu;
the Picard sequence starts from the Stokes solution of the same viscosity.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .q2q1 import make_problem


def _direct_solve(p):
    """Solve p.full_matrix() x = p.b; a singular (pure Dirichlet) system is solved with
    pressure node 0 fixed to 0 (any solution; the velocity is unique)."""
    A = sp.lil_matrix(p.full_matrix())
    b = p.b[:, 0].copy()
    if p.pinned < 0:
        q = p.dim * p.n_v
        A[q, :] = 0.0
        A[q, q] = 1.0
        b[q] = 0.0
    return spla.spsolve(sp.csc_matrix(A), b)


def lid_cavity_problem(n, nu, wind_nodal=None):
    return make_problem(n, 2, -1.0, 1.0, bc="lid", pin=False, nu=nu, wind_nodal=wind_nodal, nrhs=1,
                        body="none", name=f"ns_lid_nu{nu:g}_{n}x{n}")


def picard_lid_cavity(n, nu, tol=1e-8, maxit=300):
    """Picard sequence for the steady lid cavity.  Returns (last_problem, x, history):
    the last linear system solved (an Oseen problem with the previous iterate as
    wind), its solution and the nonlinear residual norms ||b(u_k) - N(u_k) x_k||_2."""
    p = lid_cavity_problem(n, nu)            # Stokes start
    x = _direct_solve(p)
    hist = []
    last = p
    for _ in range(maxit):
        nv = p.n_v
        wind = x[:2 * nv].reshape(2, nv)
        q = lid_cavity_problem(n, nu, wind_nodal=wind)
        r = np.linalg.norm(q.b[:, 0] - q.full_matrix() @ x)
        hist.append(float(r))
        if r < tol:
            break
        x = _direct_solve(q)
        last = q
    return last, x, hist
