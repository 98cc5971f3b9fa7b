"""Oracle: Braess-Sarazin relaxation, V-cycle and flexible GMRES (FP64, CPU).

Test infrastructure only (see the package docstring).  Vectors are arrays of
shape (N, k): k right-hand sides, dofs ordered [u_x | u_y (| u_z) | p].
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _split(L, x):
    nu = L.dim * L.n_v
    return x[:nu], x[nu:]


def apply_A(L, x):
    """Block product [I_d (x) A, Bt; B, C] x (eq. stokes_block_system / ns_block_system)."""
    u, p = _split(L, x)
    U = u.reshape(L.dim, L.n_v, -1)
    yu = np.stack([L.A @ U[c] for c in range(L.dim)]).reshape(L.dim * L.n_v, -1) + L.Bt @ p
    yp = L.B @ u
    if L.pinned >= 0:
        yp[L.pinned] += p[L.pinned]
    return np.vstack([yu, yp])


def gauss_seidel(L, g, iters: int, order: str = "strips"):
    """`iters` forward Gauss-Seidel iterations on S dp = g from dp = 0 (Section 5.2
    solves the Schur system approximately by a few Gauss-Seidel iterations; Section 6
    uses five).  The paper gives no
    ordering.  Reading: rows ordered by (strip parity, color, index), where the
    strips are consecutive blocks of T rows, T the smallest length for which
    strips two apart share no entry of S (hierarchy.strip_length), and each strip
    is greedily colored on its own subgraph.
    Rows with the same parity and color share no entry of S (same strip: the
    coloring; different strips of one parity: the bandwidth), so updating them
    at once gives the same result as one after another.

    order = "natural" takes the rows in index order instead (lexicographic on the
    structured meshes): one iteration is the triangular solve
    (D + L) dp_new = g - U dp_old with S = L + D + U."""
    S = L.S
    diag = S.diagonal()
    off = S - sp.diags(diag)
    dp = np.zeros_like(g)
    if order == "natural":
        lower = sp.tril(S, format="csr")
        upper = sp.triu(S, k=1, format="csr")
        for _ in range(iters):
            dp = spla.spsolve_triangular(lower, g - upper @ dp, lower=True)
        return dp
    if order != "strips":
        raise ValueError(f"unknown Gauss-Seidel order {order!r}")
    parity = (np.arange(L.n_p) // L.gs_strip) % 2
    ncol = int(L.colors.max()) + 1 if len(L.colors) else 0
    groups = [np.flatnonzero((parity == b) & (L.colors == c)) for b in (0, 1) for c in range(ncol)]
    groups = [rows for rows in groups if len(rows)]
    for _ in range(iters):
        for rows in groups:
            dp[rows] = (g[rows] - off[rows] @ dp) / diag[rows][:, None]
    return dp


def bs_sweep(L, prm, b, x):
    """One Braess-Sarazin step x <- x + M^-1 (b - A x) (Section 5.2) with
    M = [c D, Bt; B, 0] and the Schur complement S = B D^-1 Bt solved by
    Gauss-Seidel.  c = omega is the placement of eq. bs2's factorisation, the
    reading that reproduces Table 1's BS column; eq. bs itself has c = 1/omega.
    The steps, from the block factorisation of M:
        r = b - A x
        S dp = B D^-1 r_u - c r_p           (pinned row: dp = r_p)
        du = (1/c) D^-1 (r_u - Bt dp)
    """
    c = prm.c
    r = b - apply_A(L, x)
    ru, rp = _split(L, r)
    Dinv = np.tile(1.0 / L.D, L.dim)[:, None]
    g = L.B @ (Dinv * ru) - c * rp
    if L.pinned >= 0:
        g[L.pinned] = rp[L.pinned]
    dp = gauss_seidel(L, g, prm.gs_iters, prm.gs_order)
    du = (1.0 / c) * Dinv * (ru - L.Bt @ dp)
    return x + np.vstack([du, dp])


def coarse_solve(L, b):
    """Coarsest level: x = A^+ b with the pseudo-inverse formed at setup (form_coarse_solve)."""
    return L.coarse_pinv @ b


def restrict(L, r):
    ru, rp = _split(L, r)
    U = ru.reshape(L.dim, L.n_v, -1)
    return np.vstack([np.vstack([L.R @ U[c] for c in range(L.dim)]), L.Rp @ rp])


def prolong(L, Lc, xc):
    uc, pc = _split(Lc, xc)
    U = uc.reshape(Lc.dim, Lc.n_v, -1)
    return np.vstack([np.vstack([L.P @ U[c] for c in range(L.dim)]), L.Pp @ pc])


def vcycle(H, b, level: int = 0):
    """V(pre, post) cycle for A_l x = b from x = 0 (Alg. 1's relaxation form
    u <- u + S_l (b - A_l u), restriction by R_l, prolongation by P_l)."""
    b = np.asarray(b, dtype=np.float64)
    if b.ndim == 1:
        return vcycle(H, b[:, None], level)[:, 0]
    prm = H.params
    L = H.levels[level]
    if level == len(H.levels) - 1:
        if prm.coarse == "vanka":
            # the paper's coarsest relaxation (Section 6.1): Vanka steps from zero, as
            # many as the pre- and post-smoothing of the other levels together
            from .vanka import vanka_sweep
            x = np.zeros_like(b)
            for _ in range(prm.pre + prm.post):
                x = vanka_sweep(L, prm, b, x)
            return x
        return coarse_solve(L, b)
    if prm.smoother == "vanka":
        from .vanka import vanka_sweep as sweep
    elif prm.smoother == "ilu":
        from .ilu import ilu_sweep as sweep
    else:
        sweep = bs_sweep
    x = np.zeros_like(b)
    for _ in range(prm.pre):
        x = sweep(L, prm, b, x)
    r = b - apply_A(L, x)
    xc = vcycle(H, restrict(L, r), level + 1)
    x = x + prolong(L, H.levels[level + 1], xc)
    for _ in range(prm.post):
        x = sweep(L, prm, b, x)
    return x


def fgmres(H, b, rtol=1e-8, restart=100, maxit=500, precond=None):
    """Right-preconditioned flexible GMRES (x0 = 0), one right-hand side at a time.

    Arnoldi by modified Gram-Schmidt, Givens rotations on the Hessenberg
    matrix, stop when the recurrence residual |g_{j+1}| <= rtol ||b||; the
    true residual ||b - A x|| / ||b|| is then recomputed and the cycle
    restarted from x if it is still above rtol.  Returns (x, iterations,
    true relative residuals, history of recurrence residuals).
    """
    L0 = H.levels[0]
    b = np.asarray(b, dtype=np.float64)
    if b.ndim == 1:
        b = b[:, None]
    M = precond or (lambda v: vcycle(H, v))
    k = b.shape[1]
    X = np.zeros_like(b)
    its = np.zeros(k, dtype=np.int64)
    relres = np.zeros(k)
    hist = []
    for col in range(k):
        bc = b[:, col]
        bnorm = np.linalg.norm(bc)
        x = np.zeros_like(bc)
        h_col = []
        if bnorm == 0.0:
            hist.append(h_col)
            continue
        total = 0
        r = bc.copy()
        beta = np.linalg.norm(r)
        while beta / bnorm > rtol and total < maxit:
            V = [r / beta]
            Z = []
            Hm = np.zeros((restart + 1, restart))
            cs = np.zeros(restart)
            sn = np.zeros(restart)
            g = np.zeros(restart + 1)
            g[0] = beta
            j_end = 0
            for j in range(restart):
                Z.append(M(V[j]))
                w = apply_A(L0, Z[j][:, None])[:, 0]
                for i in range(j + 1):
                    Hm[i, j] = np.dot(V[i], w)
                    w = w - Hm[i, j] * V[i]
                Hm[j + 1, j] = np.linalg.norm(w)
                for i in range(j):
                    t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                    Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                    Hm[i, j] = t
                a, bb = Hm[j, j], Hm[j + 1, j]
                rr = np.hypot(a, bb)
                cs[j], sn[j] = (1.0, 0.0) if rr == 0.0 else (a / rr, bb / rr)
                Hm[j, j] = rr
                Hm[j + 1, j] = 0.0
                g[j + 1] = -sn[j] * g[j]
                g[j] = cs[j] * g[j]
                total += 1
                j_end = j + 1
                h_col.append(abs(g[j + 1]) / bnorm)
                if abs(g[j + 1]) <= rtol * bnorm or bb == 0.0 or total >= maxit:
                    break
                V.append(w / bb)
            y = sla.solve_triangular(Hm[:j_end, :j_end], g[:j_end])
            for i in range(j_end):
                x = x + y[i] * Z[i]
            r = bc - apply_A(L0, x[:, None])[:, 0]
            beta = np.linalg.norm(r)
        X[:, col] = x
        its[col] = total
        relres[col] = beta / bnorm
        hist.append(h_col)
    return X, its, relres, hist
