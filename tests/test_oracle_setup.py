"""Pins for the oracle's hierarchy setup (Alg. 1-4, eq. e:filtering, eq. min_problem).

Each test checks the oracle against something other than itself: invariants
the paper states, special cases it works out, closed forms, dense products.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from synth import make_problem, stokes_lid_2d, stokes_pinned_2d, oseen_recirculating_2d
from oracle import setup_hierarchy, Params
from oracle.hierarchy import (CPT, FPT, EXCL, bfs, filter_lump, find_coarse_pressures,
                              find_velocity_cpoints, emin_step, pressure_pattern, kron_identity)


@pytest.fixture(scope="module")
def lid32():
    p = stokes_lid_2d(32, nrhs=1, body="none", lo=-1.0, hi=1.0)
    return p, setup_hierarchy(p)


def test_filter_keeps_row_sums_and_gives_9_point_pressure_graph(lid32):
    """eq. e:filtering lumps dropped entries, so row sums are kept; on a uniform
    mesh the filtered B B^T graph is the 9-point graph (footnote to Fig. 2)."""
    p, H = lid32
    L0 = H.levels[0]
    Z = (L0.B @ L0.B.T).tocsr()
    F, adj = filter_lump(Z, 0.06)
    assert np.allclose(np.asarray(F.sum(axis=1)).ravel(), np.asarray(Z.sum(axis=1)).ravel(), atol=1e-15)
    m = 33
    for (i, j) in [(10, 10), (16, 5), (1, 20)]:
        v = j * m + i
        nb = sorted(adj[v])
        expect = sorted((j + dy) * m + (i + dx) for dx in (-1, 0, 1) for dy in (-1, 0, 1) if dx or dy)
        assert nb == expect
    # filtered graphs have no self loops and are symmetric
    for v in range(len(adj)):
        assert v not in adj[v]
        for w in adj[v]:
            assert v in adj[w]


def test_alg3_distance4_packing_and_coverage(lid32):
    """After Alg. 3's main loop C-points are pairwise >= 4 apart and every F-point
    is within distance 3 of a C-point (Section 4.1)."""
    p, H = lid32
    L0 = H.levels[0]
    info = L0.info
    adj = info["adjp"]
    main = info["selection_order"]
    mainset = set(main)
    for c in main:
        d = bfs(adj, c, 3)
        assert not (set(d) - {c}) & mainset
    state = info["state"]
    for j in np.flatnonzero(state == FPT):
        assert any(bfs(adj, int(j), 3).get(c) is not None for c in info["S"][j])
        assert info["S"][j]


def test_alg3_perfect_coarsening_on_uniform_mesh(lid32):
    """Started at p_{0,0}, the packing heuristic picks every 4th node in each direction,
    the perfect coarsening of Fig. 2 (right) that the paper says its metrics encourage."""
    p, H = lid32
    L0 = H.levels[0]
    m = 33
    expect = sorted(j * m + i for i in range(0, m, 4) for j in range(0, m, 4))
    assert L0.info["Cp"] == expect
    assert L0.info["extra_p"] == []


def test_alg4_midpoints_on_perfect_coarsening(lid32):
    """Alg. 4 on a perfect distance-4 coarsening adds exactly the even-indexed pressure
    nodes (targets sit on pressure vertices, Fig. 4); visits 7^d-1 = 48 points and
    |B_i| <= 3^(d-1) 7^(d-1) = 21 (Section 4.2's cost bound)."""
    p, H = lid32
    L0 = H.levels[0]
    m = 33
    expect = sorted(j * m + i for i in range(0, m, 2) for j in range(0, m, 2))
    assert L0.info["Cbar"] == expect
    assert max(L0.info["visited"]) == 48
    # |B_i| bound, recomputed from the S sets
    S = L0.info["S"]
    state = L0.info["state"]
    F = [i for i in range(len(state)) if state[i] == FPT]
    sizes = [sum(1 for j in F if set(S[i]) <= set(S[j])) for i in F[::7]]
    assert max(sizes) == 21


def test_alg4_tau2_large_rejects_midpoints():
    """With tau2 very large no mid-point passes the distance test except where B_i
    holds no C-bar point yet; with tau2 = 0 every chosen m is added."""
    p = stokes_lid_2d(16, nrhs=1, body="none")
    H = setup_hierarchy(p)
    info = H.levels[0].info
    S, state, X = info["S"], info["state"].copy(), p.pcoords
    Cbar0, _ = find_velocity_cpoints(state, S, X, 0.0)
    Cbar_big, _ = find_velocity_cpoints(state, S, X, 1e6)
    C = set(np.flatnonzero(state == CPT))
    assert C < Cbar_big <= Cbar0
    assert len(Cbar_big) < len(Cbar0)


def test_pinned_pressure_is_excluded():
    p = stokes_pinned_2d(8)
    H = setup_hierarchy(p)
    L0 = H.levels[0]
    assert L0.info["state"][0] == EXCL
    assert L0.Pp[0].nnz == 0
    assert H.levels[1].pinned == -1


def test_velocity_pattern_rows(lid32):
    p, H = lid32
    L0, L1 = H.levels[0], H.levels[1]
    P = L0.P
    Cv = L0.info["Cv"]
    cnt = np.diff(P.indptr)
    assert np.all(cnt[L0.dirichlet] == 0)
    assert np.all(cnt[~L0.dirichlet] > 0)
    for t, c in enumerate(Cv):
        assert cnt[c] == 1 and P.indices[P.indptr[c]] == t and P.data[P.indptr[c]] == 1.0
    # coarse velocities are the interior nodes co-located with the even pressure nodes
    nv1 = 65
    expect = sorted(j * nv1 + i for i in range(4, nv1 - 1, 4) for j in range(4, nv1 - 1, 4))
    assert Cv == expect
    assert L1.n_v == len(Cv) and L1.n_p == 81


def test_emin_constraint_pattern_and_energy(lid32):
    """P 1 = 1 on every non-excluded row (W in range(P), Section 4.3), the pattern is
    respected, and one CG step does not raise the energy of the initial guess."""
    p, H = lid32
    for L in H.levels[:-1]:
        for P, rowsmask in ((L.P, ~L.dirichlet), (L.Pp, np.arange(L.n_p) != L.pinned)):
            s = np.asarray(P.sum(axis=1)).ravel()
            assert np.abs(s[rowsmask] - 1.0).max() < 1e-12
            assert np.all(s[~rowsmask] == 0.0)
    L0 = H.levels[0]
    info = L0.info
    rows = pressure_pattern(info["state"], info["S"], info["Cp"])
    At = info["Ap_filtered"]
    P1 = emin_step(At, rows, len(info["Cp"]), "cg")
    cnt = np.array([len(r) for r in rows])
    P0 = sp.csr_matrix((np.repeat(1.0 / np.maximum(cnt, 1), cnt), np.concatenate([np.array(r, int) for r in rows]),
                        np.concatenate([[0], np.cumsum(cnt)])), shape=P1.shape)
    e0 = (P0.multiply(At @ P0)).sum()
    e1 = (P1.multiply(At @ P1)).sum()
    assert e1 < e0
    assert np.array_equal(P1.indices, L0.Pp.indices)


def _dense_transfer(L, which):
    M = L.P if which == "P" else L.R
    Mp = L.Pp if which == "P" else L.Rp
    return sp.block_diag([kron_identity(L.dim, M), Mp]).toarray()


@pytest.mark.parametrize("case", ["lid", "pinned", "oseen"])
def test_galerkin_identity_and_block_structure(case):
    """A_{l+1} = R_l A_l P_l (Alg. 1) against a dense triple product; the coarse
    (2,2) block is zero, the velocity block is I_d (x) A_hat_{l+1}, and the
    constant pressure is a null vector on every coarse level."""
    if case == "lid":
        p = stokes_lid_2d(16, nrhs=1, body="none")
    elif case == "pinned":
        p = stokes_pinned_2d(16)
    else:
        p = oseen_recirculating_2d(16, Re=10.0, nrhs=1)
    H = setup_hierarchy(p)
    assert len(H.levels) >= 2
    for l in range(len(H.levels) - 1):
        L, Lc = H.levels[l], H.levels[l + 1]
        A = L.full_matrix().toarray()
        RAP = _dense_transfer(L, "R") @ A @ _dense_transfer(L, "P")
        Ac = Lc.full_matrix().toarray()
        assert np.abs(RAP - Ac).max() <= 1e-13 * np.abs(A).max()
        assert np.abs(Ac[Lc.dim * Lc.n_v:, Lc.dim * Lc.n_v:]).max() == 0.0
        if case == "pinned":
            # the pin removes the constant pressure from the null space on every level
            sv = np.linalg.svd(Ac, compute_uv=False)
            assert sv[-1] > 1e-8 * sv[0]
            continue
        z = np.zeros(Lc.N)
        z[Lc.dim * Lc.n_v:] = 1.0
        assert np.abs(Ac @ z).max() <= 1e-12 * np.abs(Ac).max()
        if case != "oseen":
            assert np.abs(z @ Ac).max() <= 1e-12 * np.abs(Ac).max()
            assert abs(Lc.Bt - Lc.B.T).max() <= 1e-14 * abs(Lc.B).max()


def test_oseen_restriction_is_petrov_galerkin():
    """NS case: R != P^T, R comes from EMIN with the transposed pattern (Section 4.3);
    R^T keeps the pattern of P and R^T 1 = 1."""
    p = oseen_recirculating_2d(16, Re=100.0, nrhs=1)
    H = setup_hierarchy(p)
    L0 = H.levels[0]
    Rt = L0.R.T.tocsr()
    Rt.sort_indices()
    P = L0.P.copy()
    P.sort_indices()
    assert np.array_equal(Rt.indptr, P.indptr) and np.array_equal(Rt.indices, P.indices)
    assert abs(Rt - P).max() > 1e-6
    s = np.asarray(Rt.sum(axis=1)).ravel()
    assert np.abs(s[~L0.dirichlet] - 1.0).max() < 1e-12


def test_coarsest_level_size_and_operator_complexity():
    """Table 1 hierarchy shape: coarsest level below 205 dofs and low complexity."""
    p = stokes_lid_2d(64, nrhs=1, body="none", lo=-1.0, hi=1.0)
    H = setup_hierarchy(p)
    assert H.levels[-1].N < 205
    assert 1.0 < H.complexity() < 1.12
    sizes = [L.N for L in H.levels]
    assert all(a > 8 * b for a, b in zip(sizes, sizes[1:-1]))


def test_3d_hierarchy_builds_with_null_vector():
    p = make_problem(4, 3, 0.0, 1.0, bc="lid", nrhs=1)
    H = setup_hierarchy(p, Params(max_coarse=200))
    assert len(H.levels) >= 2
    Lc = H.levels[1]
    z = np.zeros(Lc.N)
    z[Lc.dim * Lc.n_v:] = 1.0
    Ac = Lc.full_matrix()
    assert np.abs(Ac @ z).max() <= 1e-12 * abs(Ac).max()


def _scaled_couplings(p):
    """(nearest, farther) scaled couplings |a_ij| / sqrt(a_ii a_jj) between interior velocity nodes."""
    A = p.A.tocsr()
    X = np.asarray(p.vcoords)
    h = (X[:, 0].max() - X[:, 0].min()) / (2 * p.n)
    d = A.diagonal()
    inter = ~np.asarray(p.v_dirichlet)
    near, far = [], []
    for i in np.flatnonzero(inter):
        for t in range(A.indptr[i], A.indptr[i + 1]):
            j = A.indices[t]
            if j != i and inter[j]:
                s = abs(A.data[t]) / np.sqrt(abs(d[i] * d[j]))
                (near if np.abs(X[j] - X[i]).max() <= 1.5 * h else far).append(s)
    return np.array(near), np.array(far)


def test_default_tau1_keeps_nearest_neighbours_in_2d_and_3d():
    """Reading of eq. e:filtering's tau1 by dimension: in 2D, 0.06 separates the nearest-neighbour
    couplings of the Q2 velocity block from the farther ones exactly; in 3D the two ranges overlap
    and 0.06 would leave velocity nodes with no edge, while the 3D default 0.015 keeps every
    nearest neighbour."""
    from oracle.hierarchy import filter_lump
    p2 = stokes_lid_2d(12, nrhs=1)
    near, far = _scaled_couplings(p2)
    assert near.min() > 0.06 > far.max()
    assert Params().tau1_for(2) == 0.06 and Params().tau1_for(3) == 0.015 and Params(tau1=0.2).tau1_for(3) == 0.2
    p3 = make_problem(6, 3, 0.0, 1.0, bc="lid", nrhs=1)
    near, far = _scaled_couplings(p3)
    assert near.min() > 0.015 and far.max() > near.min()
    _, adj = filter_lump(p3.A, 0.06)
    inter = ~np.asarray(p3.v_dirichlet)
    assert any(len(adj[i]) == 0 for i in np.flatnonzero(inter))
    _, adj = filter_lump(p3.A, Params().tau1_for(3))
    X = np.asarray(p3.vcoords)
    h = 1.0 / (2 * p3.n)
    A = p3.A.tocsr()
    for i in np.flatnonzero(inter):
        nb = {int(j) for j in A.indices[A.indptr[i]:A.indptr[i + 1]]
              if j != i and inter[j] and np.abs(X[j] - X[i]).max() <= 1.5 * h}
        assert nb <= set(int(j) for j in adj[i]), i


def test_3d_velocities_coarsen_with_the_3d_tau1():
    """With the 3D tau1 the first coarse level keeps a small fraction of the velocity nodes, as in
    2D; with 0.06 most velocity nodes are isolated in the filtered graph and become coarse."""
    p = make_problem(8, 3, 0.0, 1.0, bc="lid", nrhs=1)
    H = setup_hierarchy(p)
    assert H.levels[1].n_v < 0.1 * H.levels[0].n_v
    assert H.levels[-1].N <= 200
    H06 = setup_hierarchy(p, Params(tau1=0.06, max_levels=2))
    assert H06.levels[1].n_v > 0.3 * H06.levels[0].n_v


def _infsup_estimates(n):
    """Table 3's estimate: the smallest non-zero singular value of
    lump(|M_l^p|)^-1/2 B_l lump(|M_l^v|)^-1/2 on every level, with the mass matrices
    carried to the coarse levels as M_l = R_l M_{l-1} P_l (Section 6.1)."""
    from synth.q2q1 import mass_matrices
    p = stokes_lid_2d(n, nrhs=1, body="none", lo=-1.0, hi=1.0)
    H = setup_hierarchy(p)
    Mv, Mp = mass_matrices(n, 2, -1.0, 1.0)
    scal = lambda M: sp.diags(1.0 / np.sqrt(np.asarray(abs(M).sum(axis=1)).ravel()))  # noqa: E731
    out = []
    for l, L in enumerate(H.levels):
        if l > 0:
            Lp = H.levels[l - 1]
            Mv, Mp = Lp.R @ Mv @ Lp.P, Lp.Rp @ Mp @ Lp.Pp
        Bs = scal(Mp) @ L.B @ sp.kron(sp.identity(L.dim), scal(Mv))
        ev = np.sort(np.linalg.eigvalsh((Bs @ Bs.T).toarray()))
        out.append(float(np.sqrt(ev[ev > 1e-10 * ev[-1]][0])))
    return out


def test_table3_infsup_estimates_of_the_coarse_operators():
    """Table 3 (256x256: 1.54, 1.56, 1.56, 1.07): the estimate does not depend on the mesh,
    the first coarse level matches the paper's 1.56, and no level approaches zero.  With the
    formula as written (lumping |M|) the finest level gives 1.42, 8% below the paper's 1.54;
    lumping M itself gives 1.56 there, so the paper's fine-level figure may come from that
    lumping.  A wrong B scale, transfer or Galerkin product moves these values."""
    s16, s32, s64 = _infsup_estimates(16), _infsup_estimates(32), _infsup_estimates(64)
    assert abs(s16[0] - s64[0]) < 0.02 and abs(s32[0] - s64[0]) < 0.01
    assert abs(s64[0] - 1.54) <= 0.10 * 1.54
    assert abs(s64[1] - 1.56) <= 0.03 * 1.56
    assert abs(s32[1] - s64[1]) < 0.03
    assert min(s64) > 0.2


# ----------------------------------------------------------------------------
# find_extra_dist3_Cpoints (Alg. 3's last step) on hand-built graphs whose
# coarse points and S sets are worked out by hand in the docstrings

def _path_graph(n):
    return [[j for j in (i - 1, i + 1) if 0 <= j < n] for i in range(n)]


def test_extra_cpoint_for_an_fpoint_covered_once_at_distance_three():
    """Path 0-1-...-7 on the x axis.  Alg. 3 starts at 0 (C); 1, 2, 3 become F and 4,
    at distance 4, the only candidate, becomes the next C; 5, 6, 7 become F.  Then
    S_7 = {4: 3}: one C-point at graph distance 3, so 7 is converted (|S_j| = 1 rule),
    while 1 (S = {0: 1, 4: 3}), 2, 3, 5, 6 are not.  The conversion adds 7 to the S
    sets of the vertices within distance 3 of it (4, 5, 6), and the pattern rows
    use the coarse numbering of C = {0, 4, 7}."""
    from oracle.hierarchy import find_extra_dist3_cpoints
    adj = _path_graph(8)
    X = np.array([[float(i), 0.0] for i in range(8)])
    state, S, order = find_coarse_pressures(adj, X, [])
    assert order == [0, 4]
    assert [int(s) for s in state] == [CPT, FPT, FPT, FPT, CPT, FPT, FPT, FPT]
    assert S[7] == {4: 3} and S[1] == {0: 1, 4: 3} and S[5] == {4: 1}
    added = find_extra_dist3_cpoints(adj, X, state, S)
    assert added == [7] and state[7] == CPT
    assert S[6] == {4: 2, 7: 1} and S[5] == {4: 1, 7: 2} and S[4] == {4: 0, 7: 3}
    rows = pressure_pattern(state, S, [0, 4, 7])
    assert rows[7] == [2] and rows[6] == [1, 2] and rows[1] == [0, 1]


def _two_cpoint_graph(jxy):
    """a = 0 at (0, 0) and b = 4 at (4, 0) joined by the path 0-1-2-3-4 on the x axis;
    j = 5 joined to a by 0-6-7-5 and to b by 4-8-9-5 (distance 3 from both).  The
    coordinates of 6-9 are placed far away so that b (h1 = 16), not 9 (also at graph
    distance 4 from a), is the closest candidate after a."""
    adj = [[1, 6], [0, 2], [1, 3], [2, 4], [3, 8], [7, 9], [0, 7], [6, 5], [4, 9], [8, 5]]
    X = np.array([[0, 0], [1, 0], [2, 0], [3, 0], [4, 0], list(jxy), [-5, 9], [-5, 10], [9, -9], [9, -10]],
                 dtype=float)
    return adj, X


@pytest.mark.parametrize("jxy, convert", [((2.0, 2.0), True), ((2.0, 0.5), False), ((2.0, 1.01), True),
                                          ((2.0, 0.99), False), ((5.0, 0.5), True)])
def test_extra_cpoint_for_an_fpoint_between_two_distant_cpoints(jxy, convert):
    """Alg. 3 gives C = {a, b} = {0, 4} and S_j = {0: 3, 4: 3}.  The reading converts j when
    its distance to the segment [a, b] exceeds a quarter of |ab| = 1: (2, 2), (2, 1.01)
    are converted, (2, 0.5) and (2, 0.99) are not; (5, 0.5) lies 0.5 from the line but
    1.118 from the segment's end b, so it is converted (segment, not line)."""
    from oracle.hierarchy import find_extra_dist3_cpoints
    adj, X = _two_cpoint_graph(jxy)
    state, S, order = find_coarse_pressures(adj, X, [])
    assert order == [0, 4]
    assert S[5] == {0: 3, 4: 3}
    assert all(len(S[v]) != 1 or 3 not in S[v].values() for v in range(10) if state[v] == FPT)
    added = find_extra_dist3_cpoints(adj, X, state, S)
    assert added == ([5] if convert else [])


def test_extra_cpoints_fire_on_perturbed_meshes_and_keep_the_coverage():
    """With perturbed node positions (synth.with_perturbed_coordinates) Alg. 3's packing is
    irregular and some F-points end up badly covered (one C-point at distance 3, or two
    far from the segment between them); they are converted, and every remaining F-point
    stays within graph distance 3 of a C-point (the coverage Section 4.1 states)."""
    from synth import with_perturbed_coordinates
    p = with_perturbed_coordinates(stokes_lid_2d(16, nrhs=1), 0.35, 100)
    H = setup_hierarchy(p, Params(max_levels=2))
    L0 = H.levels[0]
    extra = L0.info["extra_p"]
    assert len(extra) >= 2
    state, S = L0.info["state"], L0.info["S"]
    for j in extra:
        assert state[j] == CPT
    for v in range(L0.n_p):
        if state[v] == FPT:
            assert any(d <= 3 for c, d in S[v].items() if state[c] == CPT)


# ----------------------------------------------------------------------------
# EMIN step (eq. min_problem, Section 4.3): optimality along its search direction,
# checked with a projection built here from a null-space basis of each row's
# constraint (not the oracle's mean subtraction)

def _test_projection(G, rows, ncols):
    """Orthogonal projection of G onto {X : X_ij = 0 off the pattern, X 1 = 0}, row by
    row through an orthonormal basis of the null space of the row's all-ones vector."""
    import scipy.linalg as sla
    G = sp.csr_matrix(G)
    out = np.zeros((len(rows), ncols))
    for i, cols in enumerate(rows):
        if len(cols) < 2:
            continue
        g = np.asarray(G[i, cols].todense()).ravel()
        Q = sla.null_space(np.ones((1, len(cols))))
        out[i, cols] = Q @ (Q.T @ g)
    return out


def _emin_case(kind):
    if kind == "stokes_pressure":
        p = stokes_lid_2d(16, nrhs=1)
        H = setup_hierarchy(p, Params(max_levels=2))
        info = H.levels[0].info
        return info["Ap_filtered"], pressure_pattern(info["state"], info["S"], info["Cp"]), len(info["Cp"])
    if kind == "stokes_velocity":
        p = stokes_lid_2d(16, nrhs=1)
        H = setup_hierarchy(p, Params(max_levels=2))
        L = H.levels[0]
        P = L.P
        rows = [list(P.indices[P.indptr[i]:P.indptr[i + 1]]) for i in range(P.shape[0])]
        return L.info["Av_filtered"], rows, P.shape[1]
    p = oseen_recirculating_2d(16, Re=100.0, nrhs=1)
    H = setup_hierarchy(p, Params(max_levels=2))
    L = H.levels[0]
    P = L.P
    rows = [list(P.indices[P.indptr[i]:P.indptr[i + 1]]) for i in range(P.shape[0])]
    return L.info["Av_filtered"], rows, P.shape[1]


@pytest.mark.parametrize("kind", ["stokes_pressure", "stokes_velocity"])
def test_emin_cg_step_is_the_exact_line_minimum(kind):
    """One CG step of min tr(P^T A P) over {pattern, P 1 = 1} from P0 = pattern / row
    count: P1 - P0 is a multiple of the projected negative gradient R0 = -Proj(A P0), and
    P1 minimises the energy on that line, i.e. <R0, A P1>_F = 0 (the directional
    derivative vanishes), which fixes the step length; the energy is larger a little
    before and after P1 on the line."""
    A, rows, nc = _emin_case(kind)
    A = sp.csr_matrix(A)
    n = len(rows)
    P0 = np.zeros((n, nc))
    for i, cols in enumerate(rows):
        if cols:
            P0[i, cols] = 1.0 / len(cols)
    R0 = -_test_projection(A @ sp.csr_matrix(P0), rows, nc)
    P1 = emin_step(A, rows, nc, "cg").toarray()
    D = P1 - P0
    a = np.sum(D * R0) / np.sum(R0 * R0)
    assert a > 0 and np.linalg.norm(D - a * R0) <= 1e-12 * np.linalg.norm(D)
    g0 = np.sum(R0 * (A @ P0))
    g1 = np.sum(R0 * (A @ P1))
    assert abs(g1) <= 1e-10 * abs(g0)
    energy = lambda P: np.sum(P * (A @ P))  # noqa: E731
    e1 = energy(P1)
    assert energy(P1 + 0.05 * a * R0) > e1 and energy(P1 - 0.05 * a * R0) > e1


def test_emin_gmres_step_minimises_the_projected_residual():
    """One GMRES step (Oseen, Section 4.3): P1 = P0 + alpha R0 minimises the Frobenius
    norm of the projected residual Proj(A P) on the line P0 + t R0, so the residual at P1
    is orthogonal to Q = Proj(A R0)."""
    A, rows, nc = _emin_case("oseen_velocity")
    A = sp.csr_matrix(A)
    n = len(rows)
    P0 = np.zeros((n, nc))
    for i, cols in enumerate(rows):
        if cols:
            P0[i, cols] = 1.0 / len(cols)
    R0 = -_test_projection(A @ sp.csr_matrix(P0), rows, nc)
    Q = _test_projection(A @ sp.csr_matrix(R0), rows, nc)
    P1 = emin_step(A, rows, nc, "gmres").toarray()
    D = P1 - P0
    a = np.sum(D * R0) / np.sum(R0 * R0)
    assert np.linalg.norm(D - a * R0) <= 1e-12 * np.linalg.norm(D)
    res1 = _test_projection(A @ sp.csr_matrix(P1), rows, nc)
    res0 = _test_projection(A @ sp.csr_matrix(P0), rows, nc)
    assert abs(np.sum(Q * res1)) <= 1e-10 * abs(np.sum(Q * res0))
    nrm = lambda t: np.linalg.norm(_test_projection(A @ sp.csr_matrix(P0 + t * R0), rows, nc))  # noqa: E731
    assert nrm(1.05 * a) > np.linalg.norm(res1) and nrm(0.95 * a) > np.linalg.norm(res1)


# ----------------------------------------------------------------------------
# Hierarchy shape at 592,387 dofs (Section 6.1, Tables 2 and 3)

@pytest.fixture(scope="module")
def lid256():
    p = stokes_lid_2d(256, nrhs=1, body="none", lo=-1.0, hi=1.0)
    return setup_hierarchy(p, Params(max_levels=4))


def test_first_coarse_level_in_the_papers_tau1_band(lid256):
    """Section 6.1 (Table 2 discussion): the first coarse matrix of the 592,387-dof lid
    cavity has between 28,088 rows (tau1 = 0) and 74,428 rows (tau1 = 0.25); tau1 = 0.06
    lies between.  The perfect distance-4 coarsening gives 65^2 pressures and 127^2
    interior velocities per component: 36,483 rows."""
    assert lid256.levels[0].N == 592387
    assert 28088 <= lid256.levels[1].N <= 74428
    assert lid256.levels[1].N == 36483


@pytest.mark.xfail(strict=True, reason="reading 5's coarsening misses the paper's coarse levels below level 1: "
                   "level 2 has 4,629 rows (paper 2,199-2,739) and level 3 15 pressures (paper 150); on level 1 "
                   "tau1 = 0.06 keeps only the diagonal couplings of B B^T (axis neighbours scale to 0.009)")
def test_second_and_third_levels_match_tables_2_and_3(lid256):
    """Section 6.1: the level-2 matrix of the 592,387-dof problem has 2,199 (tau2 = 0.4) to
    2,739 rows; Table 3's coarsest operator shown (level 3) has 150 pressure dofs."""
    assert 2199 <= lid256.levels[2].N <= 2739
    assert abs(lid256.levels[3].n_p - 150) <= 30


def test_level_one_pressure_graph_keeps_only_diagonal_neighbours(lid256):
    """Why the coarser levels miss Tables 2-3 (measured, reading 5 of the design notes): on the
    Galerkin level 1 the scaled couplings |z_ij| / sqrt(z_ii z_jj) of Z = B_1 B_1^T are
    ~0.14 to the diagonal neighbours but ~0.009 to the axis neighbours and ~0.056 two
    apart, so tau1 = 0.06 leaves an interior node only its four diagonal neighbours (the
    graph splits into the two checkerboard classes) and Alg. 3 keeps 497 of the 4,225
    pressures where a perfect coarsening keeps 17^2 = 289."""
    from oracle.hierarchy import spgemm
    L1 = lid256.levels[1]
    adj = L1.info["adjp"]
    m = 65
    X = L1.pcoords
    h = X[1, 0] - X[0, 0]
    for c in (32 * m + 32, 20 * m + 40):
        offs = sorted(tuple(np.round((X[j] - X[c]) / h).astype(int)) for j in adj[c])
        assert offs == [(-1, -1), (-1, 1), (1, -1), (1, 1)]
    assert L1.info["n_cp"] == 497
