"""Oracle: Vanka relaxation (Section 5.1), FP64, CPU.  Test infrastructure only.

The paper's Vanka step is an overlapping block Gauss-Seidel sweep: one block T_i
per pressure dof i, made of the velocity dofs in the columns of row i of B plus
the pressure dof itself, and for each block in turn

    x <- x + omega R_i^T (R_i A R_i^T)^-1 R_i (f - A x)

with R_i the restriction to T_i and omega = 0.5 (Section 6).

Readings (the paper is silent on them):
  * Order.  The paper relaxes every set T_i in turn but names no order.  Reading:
    blocks in the order (color, index), the colors a greedy coloring (index
    order, smallest free color) of the block interaction graph, in which blocks
    i and j are adjacent when a row of A in T_i has an entry in a column of T_j
    or the other way round (overlapping blocks are adjacent).  Blocks of one
    color then neither overlap nor see each other's values through A, so
    relaxing them together gives exactly the sequential result.
  * Dof in no block.  A Dirichlet velocity dof has a zero column in B, so no
    T_i holds it; its row of A is an identity row decoupled from the others,
    and it is relaxed exactly (x_u = f_u) at the start of each sweep.  Any other
    dof in no block (none occurs on the meshes here) is a block of its own.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def vanka_blocks(L):
    """T_i (sorted global dof indices) for every pressure dof i, then the singleton
    blocks of non-Dirichlet dofs in no T_i, and the Dirichlet velocity dofs."""
    nu = L.dim * L.n_v
    B = sp.csr_matrix(L.B)
    blocks = []
    covered = np.zeros(L.N, dtype=bool)
    for i in range(L.n_p):
        cols = np.sort(B.indices[B.indptr[i]:B.indptr[i + 1]])
        T = np.concatenate([cols, [nu + i]]).astype(np.int64)
        covered[T] = True
        blocks.append(T)
    dirichlet = np.flatnonzero(np.tile(np.asarray(L.dirichlet, dtype=bool), L.dim))
    covered[dirichlet] = True
    for u in np.flatnonzero(~covered):
        blocks.append(np.array([u], dtype=np.int64))
    return blocks, dirichlet


def vanka_colors(M, blocks) -> np.ndarray:
    """Greedy coloring of the block interaction graph (see the module docstring)."""
    nb = len(blocks)
    rows = np.concatenate(blocks)
    cols = np.concatenate([np.full(len(T), b) for b, T in enumerate(blocks)])
    E = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(M.shape[0], nb))
    P = abs(sp.csr_matrix(M)) + sp.identity(M.shape[0], format="csr")
    G = (E.T @ P @ E)
    G = sp.csr_matrix(G + G.T)
    colors = np.full(nb, -1, dtype=np.int64)
    for b in range(nb):
        used = {int(colors[j]) for j in G.indices[G.indptr[b]:G.indptr[b + 1]] if j != b and colors[j] >= 0}
        c = 0
        while c in used:
            c += 1
        colors[b] = c
    return colors


def form_vanka(L):
    """Blocks, colors and the dense inverses of the local matrices R_i A R_i^T."""
    M = sp.csr_matrix(L.full_matrix())
    blocks, dirichlet = vanka_blocks(L)
    colors = vanka_colors(M, blocks)
    inv = []
    for T in blocks:
        MT = M[T][:, T].toarray()
        # a numerically singular local matrix (its pressures carry no coupling, as on a
        # coarsest level that keeps only the constant pressure) has no Vanka step.  The
        # test: LU with partial pivoting meets a pivot of at most n eps max|entry| (the
        # pivots of Gauss-Jordan elimination with partial pivoting are the same ones)
        lu, _ = sla.lu_factor(MT, check_finite=False)
        if not np.abs(np.diag(lu)).min() > len(T) * np.finfo(float).eps * np.abs(MT).max():
            raise ValueError("a Vanka block matrix is singular")
        inv.append(np.linalg.inv(MT))
    L.vanka = dict(blocks=blocks, colors=colors, inv=inv, dirichlet=dirichlet, M=M)


def vanka_sweep(L, prm, b, x):
    """One Vanka step (Section 5.1): the Dirichlet dofs exactly, then the blocks
    color by color; the residual is recomputed before each color, which equals
    recomputing it before each block because blocks of one color do not interact."""
    V = L.vanka
    M = V["M"]
    omega = prm.vanka_omega
    x = np.array(x, dtype=np.float64, copy=True)
    D = V["dirichlet"]
    x[D] = b[D]
    colors = V["colors"]
    for c in range(int(colors.max()) + 1 if len(colors) else 0):
        r = b - M @ x
        for bi in np.flatnonzero(colors == c):
            T = V["blocks"][bi]
            x[T] += omega * (V["inv"][bi] @ r[T])
    return x


def vanka_sweep_sequential(L, prm, b, x):
    """The same step block by block in the order (color, index) with the residual
    recomputed before every block: the plain definition, for the tests."""
    V = L.vanka
    M = V["M"]
    x = np.array(x, dtype=np.float64, copy=True)
    D = V["dirichlet"]
    x[D] = b[D]
    order = sorted(range(len(V["blocks"])), key=lambda i: (V["colors"][i], i))
    for bi in order:
        T = V["blocks"][bi]
        r = b - M @ x
        x[T] += prm.vanka_omega * np.linalg.solve(M[T][:, T].toarray(), r[T])
    return x
