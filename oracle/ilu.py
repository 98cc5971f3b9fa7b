"""Oracle: ILU(1) relaxation (Section 5), FP64, CPU.  Test infrastructure only.

The paper's ILU(1) smoother factors the whole saddle-point matrix of a level
with one level of fill, treating the diagonal of the zero (2,2) block as a
nonzero so that fill can enter it, and relaxes with

    x <- x + (L U)^-1 (b - A x).

It orders the unknowns naturally (lexicographically) for the Stokes problems and
by reverse Cuthill-McKee for the Navier-Stokes ones (Section 6.1).

Readings (the paper is silent on them):
  * Level of fill.  The usual ILU(k) rule: entries of the matrix and of the
    diagonal have level 0, an entry reached through pivot row m has level
    lev(i,m) + lev(m,j) + 1 (the smallest over all pivots), and entries of
    level > 1 are dropped; the elimination then runs in IKJ order over the
    kept pattern.  No damping.
  * Zero pivots.  A row of the zero block that the ordering places before all
    of its neighbours receives no fill, so its pivot stays exactly zero (the
    paper reports such ILU(1) + RCM breakdowns on some Navier-Stokes meshes).
    A pivot that no elimination step reaches and whose matrix entry is zero
    takes the value -sum_j M_ij M_ji / M_jj: the Schur-complement diagonal that
    eliminating its neighbours would give with their block replaced by its
    diagonal.  Every other pivot is the elimination's own.
  * Natural order: the level's dof order [u_x | u_y (| u_z) | p] (the block order of
    the paper's IFISS matrices, each block lexicographic).  Params.ilu_order =
    "location" is an alternative for symmetric problems, not the paper's: every dof
    sorted by its node's coordinates (last coordinate slowest), the dofs of one node
    as u_x, u_y (, u_z), p, a pressure placed at its co-located velocity node.
  * Reverse Cuthill-McKee (non-symmetric problems): on the graph of A + A^T
    without self loops, start at the vertex of smallest degree (lowest index on
    ties), visit the unvisited neighbours of each vertex by increasing degree
    (then index), start again from the smallest-degree unvisited vertex for
    every new component, and reverse the visiting order.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def rcm_order(M) -> np.ndarray:
    """Reverse Cuthill-McKee permutation (new position -> old index) by the rule above."""
    G = sp.csr_matrix(abs(sp.csr_matrix(M)) + abs(sp.csr_matrix(M)).T)
    n = G.shape[0]
    nbrs = [[int(j) for j in G.indices[G.indptr[i]:G.indptr[i + 1]] if j != i] for i in range(n)]
    deg = np.array([len(v) for v in nbrs])
    seen = np.zeros(n, dtype=bool)
    order = []
    by_degree = sorted(range(n), key=lambda i: (deg[i], i))
    for start in by_degree:
        if seen[start]:
            continue
        seen[start] = True
        queue = [start]
        head = 0
        while head < len(queue):
            v = queue[head]
            head += 1
            for u in sorted((u for u in nbrs[v] if not seen[u]), key=lambda u: (deg[u], u)):
                seen[u] = True
                queue.append(u)
        order.extend(queue)
    return np.array(order[::-1], dtype=np.int64)


def ilu1(M):
    """ILU(1) of M (square, any order) with its diagonal in the pattern: returns rows as
    dicts {col: value} -- the strict lower part holds L (unit diagonal implied), the
    diagonal and upper part hold U -- and the fill levels.  Two phases: the levels of
    row i over all pivot rows m < i (in increasing order), keeping entries of level
    <= 1; then elimination over that fixed pattern, so (L U)_ij = M_ij on it."""
    M = sp.csr_matrix(M)
    n = M.shape[0]
    val, lev = [], []
    for i in range(n):
        lv = {i: 0}
        for t in range(M.indptr[i], M.indptr[i + 1]):
            lv[int(M.indices[t])] = 0
        pending = sorted(j for j in lv if j < i)
        k = 0
        while k < len(pending):
            m = pending[k]
            k += 1
            for j, lmj in lev[m].items():
                if j <= m:
                    continue
                nl = lv[m] + lmj + 1
                if j in lv:
                    lv[j] = min(lv[j], nl)
                elif nl <= 1:
                    lv[j] = nl
                    if j < i:
                        pending.append(j)
                        pending[k:] = sorted(pending[k:])
        lev.append(lv)
        v = {j: 0.0 for j in lv}
        for t in range(M.indptr[i], M.indptr[i + 1]):
            v[int(M.indices[t])] += M.data[t]
        reached = False
        for m in sorted(j for j in v if j < i):
            f = v[m] / val[m][m]
            v[m] = f
            for j, u in val[m].items():
                if j > m and j in v:
                    v[j] -= f * u
                    reached = reached or j == i
        if not reached and v[i] == 0.0:
            v[i] = _schur_pivot(M, i)
        val.append(v)
    return val, lev


def _schur_pivot(M, i):
    """Pivot of a zero-block row that no elimination step reaches: the Schur-complement
    diagonal -sum_j M_ij M_ji / M_jj its neighbours would give, with the (velocity) block
    they belong to replaced by its diagonal."""
    s = 0.0
    for t in range(M.indptr[i], M.indptr[i + 1]):
        j = int(M.indices[t])
        if j == i:
            continue
        mjj = M[j, j]
        if mjj != 0.0:
            s -= M.data[t] * M[j, i] / mjj
    return s


def location_order(L) -> np.ndarray:
    """Dofs by node location (see the module docstring): position -> dof."""
    nu = L.dim * L.n_v
    X = np.empty((nu + L.n_p, L.dim))
    for c in range(L.dim):
        X[c * L.n_v:(c + 1) * L.n_v] = L.vcoords
    for k in range(L.n_p):
        v = int(L.p2v[k])
        X[nu + k] = L.vcoords[v] if v >= 0 else L.pcoords[k]
    keys = [np.arange(nu + L.n_p)] + [X[:, c] for c in range(L.dim)]
    return np.lexsort(keys).astype(np.int64)


def form_ilu(L, symmetric: bool, order: str = "block"):
    """The level's block matrix in the smoother's order (natural for a symmetric
    problem, Stokes; reverse Cuthill-McKee otherwise), its ILU(1) factors and the order."""
    M = sp.csr_matrix(L.full_matrix())
    if not symmetric:
        perm = rcm_order(M)
    elif order == "location":
        perm = location_order(L)
    else:
        perm = np.arange(M.shape[0])
    Mp = M[perm][:, perm]
    rows, _ = ilu1(Mp)
    n = M.shape[0]
    Lm = sp.lil_matrix((n, n))
    Um = sp.lil_matrix((n, n))
    for i, r in enumerate(rows):
        for j, v in r.items():
            (Lm if j < i else Um)[i, j] = v
    L.ilu = dict(M=M, perm=perm, L=sp.csr_matrix(Lm), U=sp.csr_matrix(Um))


def ilu_sweep(L, prm, b, x):
    """One ILU(1) step x <- x + (L U)^-1 (b - A x) in the smoother's order."""
    from scipy.sparse.linalg import spsolve_triangular
    I = L.ilu
    r = b - I["M"] @ x
    rp = r[I["perm"]]
    n = rp.shape[0]
    Lunit = I["L"] + sp.identity(n, format="csr")
    y = spsolve_triangular(Lunit, rp, lower=True)
    d = spsolve_triangular(sp.csr_matrix(I["U"]), y, lower=False)
    out = np.array(x, dtype=np.float64, copy=True)
    out[I["perm"]] += d
    return out
