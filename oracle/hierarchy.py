"""Oracle: hierarchy setup of Alg. 1 (setup_hierarchy) with Alg. 2-4 and EMIN.

Test infrastructure only (see the package docstring).  Every function follows
the paper's steps in order; Python loops over vertices are used on purpose.

Conventions shared with the problem generator:
  * a level holds the scalar velocity block A (n_v x n_v, shared by the d
    components), the (2,1) block B (n_p x d*n_v, component-major columns),
    the (1,2) block Bt (d*n_v x n_p; equal to B^T unless R != P^T),
    velocity / pressure coordinates, the pressure -> velocity co-location map
    p2v (-1 where the co-located velocity is not a dof of this level), the
    Dirichlet velocity mask and an optional pinned pressure.
  * coarse dofs are numbered in ascending order of their fine index.
"""
from __future__ import annotations

import dataclasses
from collections import deque

import numpy as np
import scipy.sparse as sp

UNMARKED, CPT, FPT, EXCL = 0, 1, 2, 3


@dataclasses.dataclass
class Params:
    """Section 6 defaults: tau1=0.06 (eq. e:filtering), tau2=sqrt(1.5e-3) (Alg. 4),
    BS relaxation 0.666 with 5 Gauss-Seidel iterations, BS(2,2), one EMIN step.

    tau1 = None takes the dimension's default: 0.06 in 2D (Section 6); in 3D,
    where the paper has no experiments, 0.015.  On a uniform 2D Q2 mesh the
    scaled couplings |a_ij| / sqrt(a_ii a_jj) are >= 0.09 between nearest nodes
    and <= 0.036 farther away, so 0.06 keeps exactly the nearest-neighbour
    graph; in 3D the two ranges overlap (nearest down to 0.016, farther up to
    0.06), 0.06 leaves most velocity nodes without an edge, and 0.015 is the
    threshold that keeps every nearest neighbour."""
    tau1: float | None = None
    tau2sq: float = 1.5e-3
    omega: float = 0.666
    omega_in_M: str = "direct"    # eq. bs2's factorisation: M = [omega D, B^T; B, 0]; "inverse": eq. bs
    gs_iters: int = 5
    pre: int = 2
    post: int = 2
    emin: str = "auto"            # "cg" (Stokes), "gmres" (Oseen); auto picks by symmetry
    smoother: str = "bs"          # "bs" Braess-Sarazin (Section 5.2), "vanka" (Section 5.1), "ilu" ILU(1) (Section 5)
    vanka_omega: float = 0.5      # Vanka under-relaxation (Section 6)
    ilu_order: str = "block"      # ILU(1) order of symmetric levels: "block" (the paper's) or "location"
    coarse: str = "exact"         # coarsest level: "exact" (pseudo-inverse) or "vanka" (pre + post Vanka
                                  # steps from zero, as the paper relaxes it, Section 6.1)
    gs_order: str = "strips"      # Gauss-Seidel order on S: "strips" (strip parity, color, index; the GPU's)
                                  # or "natural" (row index order, the textbook forward sweep)
    max_coarse: int = 200
    max_levels: int = 12

    def tau1_for(self, dim: int) -> float:
        if self.tau1 is not None:
            return self.tau1
        return 0.06 if dim == 2 else 0.015

    @property
    def c(self) -> float:
        """Scale of D in the (1,1) block of the Braess-Sarazin matrix M."""
        return 1.0 / self.omega if self.omega_in_M == "inverse" else self.omega


@dataclasses.dataclass
class Level:
    dim: int
    n_v: int
    n_p: int
    A: sp.csr_matrix
    B: sp.csr_matrix
    Bt: sp.csr_matrix
    vcoords: np.ndarray
    pcoords: np.ndarray
    p2v: np.ndarray
    dirichlet: np.ndarray
    pinned: int
    # smoother (Section 5.2)
    D: np.ndarray = None          # |A| row sums (Dirichlet rows: 1/c so that c*D = 1)
    S: sp.csr_matrix = None       # B D^-1 Bt, pinned row = identity
    colors: np.ndarray = None     # greedy coloring of each Gauss-Seidel strip of S's graph
    gs_strip: int = 1             # Gauss-Seidel strip length T = bandwidth of S
    # transfers to the next level (Alg. 2)
    P: sp.csr_matrix = None       # velocity, one component (n_v x n_v_coarse)
    Pp: sp.csr_matrix = None      # pressure (n_p x n_p_coarse)
    R: sp.csr_matrix = None
    Rp: sp.csr_matrix = None
    # coarsest-level solve
    coarse_pinv: np.ndarray = None
    # Vanka smoother data (oracle.vanka.form_vanka), when that smoother is chosen
    vanka: dict = None
    # ILU(1) smoother data (oracle.ilu.form_ilu), when that smoother is chosen
    ilu: dict = None
    # setup diagnostics (for the tests)
    info: dict = dataclasses.field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.dim * self.n_v + self.n_p

    def nnz(self) -> int:
        return self.dim * self.A.nnz + self.B.nnz + self.Bt.nnz + (1 if self.pinned >= 0 else 0)

    def full_matrix(self) -> sp.csr_matrix:
        Av = sp.kron(sp.identity(self.dim, format="csr"), self.A, format="csr")
        C = sp.csr_matrix((self.n_p, self.n_p))
        if self.pinned >= 0:
            C = sp.csr_matrix(([1.0], ([self.pinned], [self.pinned])), shape=(self.n_p, self.n_p))
        return sp.bmat([[Av, self.Bt], [self.B, C]], format="csr")


@dataclasses.dataclass
class Hierarchy:
    levels: list
    params: Params
    symmetric: bool

    def complexity(self) -> float:
        """Operator complexity: sum of nnz over levels / nnz of the finest (Section 6.1)."""
        return sum(L.nnz() for L in self.levels) / self.levels[0].nnz()


# ----------------------------------------------------------------------------
# sparse helpers (library primitives only)

def pattern(M) -> sp.csr_matrix:
    """Same structure as M, every stored entry (explicit zeros included) set to 1."""
    Q = sp.csr_matrix(M, copy=True)
    Q.data = np.ones_like(Q.data)
    return Q


def on_pattern(pat, V) -> sp.csr_matrix:
    """CSR with the structure of `pat` and the values of V on it (0 where V has none)."""
    pat = sp.csr_matrix(pat)
    pat.sort_indices()
    rows = np.repeat(np.arange(pat.shape[0]), np.diff(pat.indptr))
    vals = np.asarray(sp.csr_matrix(V)[rows, pat.indices]).ravel() if pat.nnz else np.zeros(0)
    return sp.csr_matrix((vals.astype(np.float64), pat.indices.copy(), pat.indptr.copy()), shape=pat.shape)


def spgemm(A, B) -> sp.csr_matrix:
    """A @ B on its structural pattern: the product of the patterns (all-positive, so
    nothing cancels) carries the values of A @ B; entries that cancel stay as zeros."""
    return on_pattern(pattern(A) @ pattern(B), sp.csr_matrix(A) @ sp.csr_matrix(B))


def kron_identity(d, M) -> sp.csr_matrix:
    return sp.kron(sp.identity(d, format="csr"), sp.csr_matrix(M), format="csr")


# ----------------------------------------------------------------------------
# form_aux_block_diagonal: eq. e:filtering

def filter_lump(Z, tau: float):
    """Drop |z_ij| <= tau*sqrt(|z_ii z_jj|) (i != j) and add the dropped values to the
    diagonal, so each row sum is kept (eq. e:filtering, Section 4.1; applied to
    B B^T for pressures and to the velocity block for velocities, Section 4.2).

    Returns the filtered matrix and the adjacency lists of its graph without
    self-loops.  Reading: a non-symmetric matrix (Oseen) gets the union of the
    kept pattern and its transpose as graph; the paper does not say.
    """
    Z = sp.coo_matrix(Z)
    n = Z.shape[0]
    d = np.zeros(n)
    on = Z.row == Z.col
    np.add.at(d, Z.row[on], Z.data[on])
    off = ~on
    r, c, v = Z.row[off], Z.col[off], Z.data[off]
    thr = tau * np.sqrt(np.abs(d[r] * d[c]))
    drop = np.abs(v) <= thr
    lump = np.zeros(n)
    # row sums of the dropped entries, in CSR order (row, then column)
    order = np.lexsort((c[drop], r[drop]))
    for i, val in zip(r[drop][order], v[drop][order]):
        lump[i] += val
    keep = ~drop
    F = sp.csr_matrix((np.concatenate([v[keep], d + lump]),
                       (np.concatenate([r[keep], np.arange(n)]), np.concatenate([c[keep], np.arange(n)]))),
                      shape=(n, n))
    adj = [set() for _ in range(n)]
    for i, j in zip(r[keep], c[keep]):
        adj[i].add(int(j))
        adj[int(j)].add(int(i))
    return F, [sorted(a) for a in adj]


def bfs(adj, src: int, maxd: int) -> dict:
    """Graph distances (edge counts) from src to every vertex within maxd."""
    dist = {src: 0}
    q = deque([src])
    while q:
        v = q.popleft()
        if dist[v] == maxd:
            continue
        for w in adj[v]:
            w = int(w)
            if w not in dist:
                dist[w] = dist[v] + 1
                q.append(w)
    return dist


def _sqdist(x, y) -> float:
    s = 0.0
    for k in range(len(x)):
        t = float(x[k]) - float(y[k])
        s = s + t * t
    return s


# ----------------------------------------------------------------------------
# Alg. 3: find_coarse_pressures, update_heuristics, find_extra_dist3_Cpoints

def find_coarse_pressures(adj, X, excluded):
    """Alg. 3 main loop: greedy distance-4 C/F split of the filtered pressure graph.

    Readings (the paper leaves them open):
      * the first vertex is the lowest-index unmarked one ("arbitrary");
      * update_heuristics: h1(j) is taken as the smallest Euclidean distance
        from j to the C-points within graph distance 4 of j, the term that
        the paper's harmonic average favours (Section 4.1).  The literal
        harmonic mean gives a staggered packing on uniform meshes and stalls
        GMRES on the 256x256 lid cavity; the minimum reproduces the perfect
        coarsening of Fig. 2 that the paper says its metrics encourage;
      * k = argmin over Cand of squared h1, where values within a relative
        1e-9 of the minimum tie and the lowest index wins; if Cand is empty,
        the lowest-index unmarked vertex;
      * excluded vertices (a pinned pressure) take no part and get no
        interpolation.
    Returns state per vertex, S_j as {C-point: graph distance} (C-points
    within distance 3 of j), and the C-points in selection order.
    """
    n = len(adj)
    state = np.full(n, UNMARKED, dtype=np.int8)
    for e in excluded:
        state[e] = EXCL
    S = [dict() for _ in range(n)]
    h1sq = np.full(n, np.inf)
    cand = set()
    order = []

    def lowest_unmarked(start):
        while start < n and state[start] != UNMARKED:
            start += 1
        return start

    next_unmarked = lowest_unmarked(0)
    k = next_unmarked if next_unmarked < n else None
    while k is not None:
        dist = bfs(adj, k, 4)
        for j, dj in dist.items():
            if dj <= 3:
                S[j][k] = dj
        state[k] = CPT
        order.append(k)
        for j, dj in dist.items():
            if dj <= 3 and j != k and state[j] == UNMARKED:
                state[j] = FPT
        for j, dj in dist.items():
            if dj == 4:
                cand.add(j)
        cand = {j for j in cand if state[j] == UNMARKED}
        # update_heuristics for the vertices within distance 4 of the new C-point
        for j, dj in dist.items():
            if j != k:
                h1sq[j] = min(h1sq[j], _sqdist(X[j], X[k]))
        if cand:
            m = min(h1sq[j] for j in cand)
            k = min(j for j in cand if h1sq[j] <= m * (1.0 + 1e-9))
        else:
            next_unmarked = lowest_unmarked(next_unmarked)
            k = next_unmarked if next_unmarked < n else None
    return state, S, order


def _seg_sqdist(x, a, b) -> float:
    """Squared Euclidean distance from x to the segment [a, b]."""
    ab = [float(b[k]) - float(a[k]) for k in range(len(x))]
    ax = [float(x[k]) - float(a[k]) for k in range(len(x))]
    L2 = 0.0
    dot = 0.0
    for k in range(len(x)):
        L2 = L2 + ab[k] * ab[k]
        dot = dot + ax[k] * ab[k]
    t = dot / L2 if L2 > 0.0 else 0.0
    t = min(max(t, 0.0), 1.0)
    s = 0.0
    for k in range(len(x)):
        e = ax[k] - t * ab[k]
        s = s + e * e
    return s


def find_extra_dist3_cpoints(adj, X, state, S):
    """Convert badly covered F-points to C-points (Alg. 3's last step, Section 4.1).

    The paper names the criteria without thresholds.  Reading, in index order:
      * |S_j| = 1 and j is at graph distance 3 from its only C-point;
      * |S_j| = 2, j is at graph distance 3 from both C-points, and its
        distance to the segment joining them exceeds 1/4 of the segment's
        length.
    Each conversion adds j to S_v of every v within graph distance 3 of j,
    before later vertices are examined.  Returns the converted vertices.
    """
    added = []
    n = len(adj)
    for j in range(n):
        if state[j] != FPT:
            continue
        s = sorted(S[j].keys())
        convert = False
        if len(s) == 1:
            convert = S[j][s[0]] == 3
        elif len(s) == 2:
            a, b = s
            if S[j][a] == 3 and S[j][b] == 3:
                L2 = _sqdist(X[a], X[b])
                convert = _seg_sqdist(X[j], X[a], X[b]) > 0.0625 * L2
        if convert:
            state[j] = CPT
            added.append(j)
            for v, dv in bfs(adj, j, 3).items():
                S[v][j] = dv
    return added


def pressure_pattern(state, S, C_sorted):
    """N^(p): row i holds the coarse indices of S_i (Section 4.1).  Readings: a
    C-point's row is its own coarse index (injection); excluded rows are empty."""
    cidx = {c: t for t, c in enumerate(C_sorted)}
    rows = []
    for i in range(len(state)):
        if state[i] == CPT:
            rows.append([cidx[i]])
        elif state[i] == FPT:
            rows.append(sorted(cidx[c] for c in S[i]))
        else:
            rows.append([])
    return rows


# ----------------------------------------------------------------------------
# Alg. 4: find_velocity_Cpoints

def find_velocity_cpoints(state, S, X, tau2sq: float):
    """Alg. 4: add pressure mid-points to C^(p), giving C-bar^(p).

    Loop over F-points by descending |S_i|, ties by index (Section 4.2).
    Readings of the garbled lines: t_i is the diagonal of the bounding box of
    B_i, t_i^2 = sum_k (max_k - min_k)^2, and ||.||_* is the Euclidean norm;
    the test is dist^2 >= tau2^2 t_i^2 with an empty minimum equal to +inf.
    X_i sums the coordinates of S_i in ascending index order, then divides.
    m = argmin over B_i of (squared distance to X_i, index).
    """
    n = len(state)
    F = [i for i in range(n) if state[i] == FPT]
    Fset = set(F)
    users = {}            # C-point -> F-points whose S contains it
    for j in F:
        for c in S[j]:
            users.setdefault(c, []).append(j)
    Cbar = set(i for i in range(n) if state[i] == CPT)
    order = sorted(F, key=lambda i: (-len(S[i]), i))
    dim = X.shape[1]
    visited_counts = []
    for i in order:
        s = sorted(S[i].keys())
        Xi = [0.0] * dim
        for k in range(dim):
            acc = 0.0
            for c in s:
                acc = acc + float(X[c, k])
            Xi[k] = acc / len(s)
        sset = set(s)
        cand = users[s[0]]
        visited_counts.append(len(cand))
        Bi = sorted(j for j in cand if j in Fset and sset.issubset(S[j].keys()))
        t2 = 0.0
        for k in range(dim):
            vals = [float(X[j, k]) for j in Bi]
            e = max(vals) - min(vals)
            t2 = t2 + e * e
        m = min(Bi, key=lambda j: (_sqdist(X[j], Xi), j))
        dmin = np.inf
        for j in Bi:
            if j in Cbar:
                dmin = min(dmin, _sqdist(X[j], X[m]))
        if dmin >= tau2sq * t2:
            Cbar.add(m)
    return Cbar, visited_counts


# ----------------------------------------------------------------------------
# velocity pattern (Section 4.2)

def velocity_pattern(adjv, Cv: set, dirichlet):
    """N^(v): non-Dirichlet row i holds the C^(v) nodes within graph distance 3 of i
    in the graph of the filtered velocity block; C-point rows are injection;
    Dirichlet rows are empty.  Extra C-points (Section 4.2, last paragraph),
    reading: in index order, a non-Dirichlet node whose row is still empty
    becomes a C-point and joins the rows of its distance-3 neighbours."""
    n = len(adjv)
    rows = [set() for _ in range(n)]
    Cv = set(int(c) for c in Cv)
    for c in sorted(Cv):
        for v in bfs(adjv, c, 3):
            rows[v].add(c)
    extra = []
    for i in range(n):
        if dirichlet[i] or i in Cv or rows[i]:
            continue
        Cv.add(i)
        extra.append(i)
        for v in bfs(adjv, i, 3):
            rows[v].add(i)
    C_sorted = sorted(Cv)
    cidx = {c: t for t, c in enumerate(C_sorted)}
    out = []
    for i in range(n):
        if dirichlet[i]:
            out.append([])
        elif i in Cv:
            out.append([cidx[i]])
        else:
            out.append(sorted(cidx[c] for c in rows[i]))
    return out, C_sorted, extra


# ----------------------------------------------------------------------------
# EMIN (Section 4.3, eq. min_problem)

def _pattern_matrix(rows, ncols) -> sp.csr_matrix:
    indptr = np.zeros(len(rows) + 1, dtype=np.int64)
    indptr[1:] = np.cumsum([len(r) for r in rows])
    indices = np.array([c for r in rows for c in r], dtype=np.int64)
    return sp.csr_matrix((np.ones(len(indices)), indices, indptr), shape=(len(rows), ncols))


def _project(G, Npat) -> sp.csr_matrix:
    """Orthogonal projection onto {pattern N, zero row sums}: take G on the pattern
    and subtract each row's mean over its pattern entries."""
    Gp = on_pattern(Npat, G)
    cnt = np.diff(Gp.indptr)
    rows = np.repeat(np.arange(Gp.shape[0]), cnt)
    sums = np.zeros(Gp.shape[0])
    for i, v in zip(rows, Gp.data):
        sums[i] += v
    mean = np.divide(sums, cnt, out=np.zeros_like(sums), where=cnt > 0)
    Gp.data = Gp.data - np.repeat(mean, cnt)
    return Gp


def emin_step(At, rows, ncols, method: str) -> sp.csr_matrix:
    """One EMIN-AMG step for min sum_j ||P_j||_chi^2 s.t. P in pattern, P 1 = 1 (eq. min_problem).

    Initial guess: the binary pattern divided by each row's count (Section 4.3).
    Reading of the step the paper takes from Olson et al. (its Alg. 2/3):
      R0 = -Proj(At P0);
      cg:    alpha = <R0,R0>_F / <R0, At R0>_F     (chi = At-norm, symmetric)
      gmres: Q = Proj(At R0), alpha = <R0,Q>_F / <Q,Q>_F  (chi = At^T At-norm)
      P = P0 + alpha R0, kept on the pattern (explicit zeros stay).
    """
    N = _pattern_matrix(rows, ncols)
    cnt = np.diff(N.indptr)
    P0 = N.copy()
    P0.data = np.repeat(np.divide(1.0, cnt, out=np.zeros(len(cnt)), where=cnt > 0), cnt)
    At = sp.csr_matrix(At)
    R0 = _project(At @ P0, N)
    R0.data = -R0.data
    if method == "cg":
        num = float(np.dot(R0.data, R0.data))
        den = float((R0.multiply(At @ R0)).sum())
    else:
        Q = _project(At @ R0, N)
        num = float(np.dot(R0.data, Q.data))
        den = float(np.dot(Q.data, Q.data))
    alpha = num / den if den != 0.0 else 0.0
    P = P0.copy()
    P.data = P0.data + alpha * R0.data
    return P


# ----------------------------------------------------------------------------
# smoother data (Section 5.2) and coarse solve

def strip_length(S) -> int:
    """Strip length T of the Gauss-Seidel ordering: the smallest T >= bandwidth/2 such
    that every entry of S couples rows of the same or of adjacent strips of T
    consecutive rows (so strips two apart never interact).  On a lexicographic
    grid this is a whole number of grid lines."""
    Sc = sp.coo_matrix(S)
    offd = Sc.row != Sc.col
    if not offd.any():
        return 1
    r, c = Sc.row[offd], Sc.col[offd]
    bw = int(np.abs(r - c).max())
    for T in range((bw + 1) // 2, bw + 1):
        if T > 0 and np.abs(r // T - c // T).max() <= 1:
            return T
    return bw


def greedy_coloring(S, strip: int) -> np.ndarray:
    """Colors for the Gauss-Seidel ordering: each strip of `strip` consecutive rows is
    colored on its own induced subgraph of S's graph (off-diagonal stored entries),
    vertices in index order, each taking the smallest color not used by an already
    colored neighbour in the same strip."""
    S = sp.csr_matrix(S)
    n = S.shape[0]
    colors = np.full(n, -1, dtype=np.int64)
    for i in range(n):
        used = set()
        for j in S.indices[S.indptr[i]:S.indptr[i + 1]]:
            if j != i and j // strip == i // strip and colors[j] >= 0:
                used.add(colors[j])
        c = 0
        while c in used:
            c += 1
        colors[i] = c
    return colors


def form_relaxation(L: Level, prm: Params):
    """Braess-Sarazin data: d_ii = sum_j |A_ij| (Section 5.2) and the explicit Schur
    complement S = B D^-1 B^T (Bt on levels where R != P^T), its greedy coloring and
    the strip length of the Gauss-Seidel ordering (see gauss_seidel).  Readings: a
    Dirichlet row of M is the identity row of A (D_ii = 1/c, so c*D_ii = 1);
    a pinned pressure row of S is the identity row (its update is exact)."""
    absA = abs(L.A)
    D = np.asarray(absA.sum(axis=1)).ravel()
    D[L.dirichlet] = 1.0 / prm.c
    Dinv_all = np.tile(1.0 / D, L.dim)
    # structural pattern of B Bt (nothing cancels in the product of patterns), values of B D^-1 Bt
    S = on_pattern(pattern(L.B) @ pattern(L.Bt), (L.B @ sp.diags(Dinv_all)) @ L.Bt)
    if L.pinned >= 0:
        S = sp.lil_matrix(S)
        S[L.pinned, L.pinned] = 1.0
        S = sp.csr_matrix(S)
    L.D = D
    L.S = S
    L.gs_strip = strip_length(S)
    L.colors = greedy_coloring(S, L.gs_strip)


def form_coarse_solve(L: Level, rcond: float = 1e-12):
    """Coarsest level: FP64 minimum-norm least-squares solve x = A^+ b through the
    SVD, singular values below rcond * sigma_max dropped.  Reading: the paper
    relaxes with Vanka on the coarsest grid because that problem is singular
    (Section 6.1); a direct solve of the singular system needs a choice of
    solution, and the pseudo-inverse takes the one orthogonal to the null
    space (the constant pressure, plus any spurious pressure mode of a very
    small, inf-sup unstable coarsest level).  A nonsingular coarsest level
    (a pinned fine pressure) gets its plain inverse.

    The SVD gives A^+ only to about cond(A) times the unit roundoff in the
    directions of small singular values (the pinned problem's levels have
    cond ~ 1e7).  On coarsest levels of at most 512 dofs (every hierarchy with
    the default max_coarse), two steps of X <- X + X (I - A X) with the residual
    I - A X formed in extended precision (numpy's longdouble) bring X to working
    accuracy; X R stays in X's row space, so dropped directions stay dropped."""
    A = L.full_matrix().toarray()
    X = np.linalg.pinv(A, rcond=rcond)
    Al = A.astype(np.longdouble)
    for _ in range(2 if A.shape[0] <= 512 else 0):
        R = (np.eye(A.shape[0], dtype=np.longdouble) - Al @ X.astype(np.longdouble)).astype(np.float64)
        X = X + X @ R
    L.coarse_pinv = X


# ----------------------------------------------------------------------------
# Alg. 2 and Alg. 1

def _make_level(prob_like) -> Level:
    return Level(dim=prob_like.dim, n_v=prob_like.n_v, n_p=prob_like.n_p, A=sp.csr_matrix(prob_like.A),
                 B=sp.csr_matrix(prob_like.B), Bt=sp.csr_matrix(prob_like.B.T),
                 vcoords=np.asarray(prob_like.vcoords), pcoords=np.asarray(prob_like.pcoords),
                 p2v=np.asarray(prob_like.p2v), dirichlet=np.asarray(prob_like.v_dirichlet, dtype=bool),
                 pinned=int(prob_like.pinned))


def form_interpolation(L: Level, prm: Params, method: str, reuse: Level = None):
    """Alg. 2 plus form_restriction and the Petrov-Galerkin product of Alg. 1.
    Returns the next level, or None when coarsening makes no progress.
    With `reuse` (the same level of a hierarchy built for a matrix of the same
    structure), its coarse points and transfer patterns are taken and only the
    filtering, EMIN, restriction and Galerkin products are redone: Section 6.1
    says the graph phase can be done once per nonlinear sequence."""
    # form_aux_block_diagonal
    Zp = spgemm(L.B, L.B.T)
    Ap, adjp = filter_lump(Zp, prm.tau1_for(L.dim))
    Av, adjv = filter_lump(L.A, prm.tau1_for(L.dim))
    if reuse is not None:
        Cp, Cv = list(reuse.info["Cp"]), list(reuse.info["Cv"])
        rows_of = lambda M: [list(M.indices[M.indptr[i]:M.indptr[i + 1]]) for i in range(M.shape[0])]  # noqa: E731
        rows_p, rows_v = rows_of(reuse.Pp), rows_of(reuse.P)
        L.info.update(dict(Cp=Cp, Cv=Cv, reused=True))
        return _finish_interpolation(L, method, Ap, Av, Cp, Cv, rows_p, rows_v)
    excluded = [L.pinned] if L.pinned >= 0 else []
    # find_coarse_pressure (Alg. 3)
    state, S, order = find_coarse_pressures(adjp, L.pcoords, excluded)
    extra = find_extra_dist3_cpoints(adjp, L.pcoords, state, S)
    Cp = sorted(int(i) for i in np.flatnonzero(state == CPT))
    if len(Cp) >= L.n_p:
        return None
    # pressure pattern
    rows_p = pressure_pattern(state, S, Cp)
    # coarse velocities (Alg. 4) and co-location
    Cbar, visited = find_velocity_cpoints(state, S, L.pcoords, prm.tau2sq)
    Cv0 = set()
    for k in Cbar:
        v = int(L.p2v[k])
        if v >= 0 and not L.dirichlet[v]:
            Cv0.add(v)
    rows_v, Cv, extra_v = velocity_pattern(adjv, Cv0, L.dirichlet)
    L.info.update(dict(n_cp=len(Cp), n_cbar=len(Cbar), n_cv=len(Cv), extra_p=extra, extra_v=extra_v,
                       selection_order=order, state=state.copy(), S=[dict(s) for s in S],
                       Cp=Cp, Cbar=sorted(Cbar), Cv=Cv, visited=visited,
                       adjp=adjp, adjv=adjv, Ap_filtered=Ap, Av_filtered=Av))
    return _finish_interpolation(L, method, Ap, Av, Cp, Cv, rows_p, rows_v)


def _finish_interpolation(L: Level, method: str, Ap, Av, Cp, Cv, rows_p, rows_v):
    """EMIN prolongators on the patterns, restriction and the Petrov-Galerkin product."""
    Pp = emin_step(Ap, rows_p, len(Cp), method)
    Pv = emin_step(Av, rows_v, len(Cv), method)
    # form_restriction (Section 4.3): R = P^T, or EMIN on A^T with the transposed pattern
    if method == "cg":
        Rv, Rp = sp.csr_matrix(Pv.T), sp.csr_matrix(Pp.T)
    else:
        Rv = sp.csr_matrix(emin_step(sp.csr_matrix(Av.T), rows_v, len(Cv), method).T)
        Rp = sp.csr_matrix(emin_step(sp.csr_matrix(Ap.T), rows_p, len(Cp), method).T)
    L.P, L.Pp, L.R, L.Rp = Pv, Pp, Rv, Rp
    d = L.dim
    Ac = spgemm(spgemm(Rv, L.A), Pv)
    Bc = spgemm(spgemm(Rp, L.B), kron_identity(d, Pv))
    Btc = spgemm(spgemm(kron_identity(d, Rv), L.Bt), Pp)
    # coarse co-location map: restriction of p2v to the coarse points
    vpos = {v: t for t, v in enumerate(Cv)}
    p2v_c = np.array([vpos.get(int(L.p2v[k]), -1) if L.p2v[k] >= 0 else -1 for k in Cp], dtype=np.int64)
    # project_coordinates (Alg. 1): reading = injection of the coarse points' coordinates
    return Level(dim=d, n_v=len(Cv), n_p=len(Cp), A=Ac, B=Bc, Bt=Btc,
                 vcoords=L.vcoords[Cv], pcoords=L.pcoords[Cp], p2v=p2v_c,
                 dirichlet=np.zeros(len(Cv), dtype=bool), pinned=-1)


def setup_hierarchy(prob, prm: Params = None, reuse: Hierarchy = None) -> Hierarchy:
    """Alg. 1 (setup_hierarchy), iterated: relaxation data, then transfers and the
    Galerkin product, until the level has <= max_coarse dofs (the paper reports
    coarsest levels below 205 dofs, Section 6.1), coarsening stalls, or
    max_levels is reached.  With `reuse` (a hierarchy for a matrix of the same
    structure, e.g. the previous Picard step), its levels, coarse points and
    transfer patterns are kept (see form_interpolation)."""
    prm = prm or Params()
    method = prm.emin if prm.emin != "auto" else ("cg" if prob.symmetric else "gmres")
    levels = [_make_level(prob)]
    while True:
        L = levels[-1]
        form_relaxation(L, prm)
        if reuse is not None:
            # the reused hierarchy decides the levels, coarse points and patterns
            if len(levels) >= len(reuse.levels):
                break
            levels.append(form_interpolation(L, prm, method, reuse.levels[len(levels) - 1]))
            continue
        if L.N <= prm.max_coarse or len(levels) == prm.max_levels:
            break
        Lc = form_interpolation(L, prm, method)
        if Lc is None or Lc.N >= L.N:
            L.P = L.Pp = L.R = L.Rp = None
            break
        if prm.coarse == "vanka" and Lc.n_p <= 1:
            # the coarsest level is relaxed with Vanka (Section 6.1): a level keeping only
            # one pressure (the constant, whose B vanishes) has no Vanka step, so the
            # current level stays the coarsest
            L.P = L.Pp = L.R = L.Rp = None
            break
        levels.append(Lc)
    form_coarse_solve(levels[-1])
    if prm.smoother == "vanka":
        from .vanka import form_vanka
        for L in levels[:-1]:
            form_vanka(L)
    if prm.coarse == "vanka":
        from .vanka import form_vanka
        form_vanka(levels[-1])
    if prm.smoother == "ilu":
        from .ilu import form_ilu
        for L in levels[:-1]:
            form_ilu(L, bool(prob.symmetric), prm.ilu_order)
    return Hierarchy(levels=levels, params=prm, symmetric=bool(prob.symmetric))
