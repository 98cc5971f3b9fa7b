"""Pins of the oracle's Vanka relaxation (Section 5.1) against what the paper and
the mathematics fix: the block definition, the exact local solve, the
equivalence of the colored sweep with the block-by-block Gauss-Seidel sweep,
the Dirichlet reading, dense solves on tiny meshes and Table 1's Vanka(1,1)
iteration counts."""
import numpy as np
import pytest
import scipy.sparse as sp

from synth import make_problem, oseen_recirculating_2d, stokes_lid_2d, stokes_pinned_2d, uniform_pm1
from oracle import Params, fgmres, setup_hierarchy, vcycle
from oracle.vanka import vanka_sweep, vanka_sweep_sequential

VANKA = dict(smoother="vanka", pre=1, post=1)


def _hier(p, **kw):
    return setup_hierarchy(p, Params(**{**VANKA, **kw}))


CASES = {
    "lid8": lambda: stokes_lid_2d(8, nrhs=1),
    "pinned8": lambda: stokes_pinned_2d(8, nrhs=1),
    "oseen8": lambda: oseen_recirculating_2d(8, Re=100.0, nrhs=1),
    "lid3d": lambda: make_problem(3, 3, 0.0, 1.0, bc="lid", nrhs=1),
}


@pytest.mark.parametrize("case", list(CASES))
def test_blocks_follow_the_rows_of_B(case):
    """T_i = the columns of row i of B plus pressure dof i; Dirichlet velocity dofs are
    in no block; every other dof is in some block."""
    p = CASES[case]()
    L = _hier(p).levels[0]
    V = L.vanka
    nu = L.dim * L.n_v
    B = sp.csr_matrix(L.B)
    for i in range(L.n_p):
        T = V["blocks"][i]
        assert T[-1] == nu + i
        assert np.array_equal(T[:-1], np.sort(B.indices[B.indptr[i]:B.indptr[i + 1]]))
    inblock = np.zeros(L.N, dtype=bool)
    for T in V["blocks"]:
        inblock[T] = True
    D = np.tile(np.asarray(L.dirichlet, dtype=bool), L.dim)
    assert not np.any(inblock[:nu][D])
    assert np.all(inblock[:nu][~D]) and np.all(inblock[nu:])
    assert len(V["blocks"]) == L.n_p  # no singleton blocks on these meshes


def test_block_support_is_the_element_patch_of_its_pressure():
    """On a uniform 2D mesh a pressure node's block holds only velocity nodes of the
    elements around it (within one element width in each direction)."""
    p = stokes_lid_2d(8, nrhs=1)
    L = _hier(p).levels[0]
    h = 1.0 / 8
    for i in range(L.n_p):
        T = L.vanka["blocks"][i][:-1]
        nodes = T % L.n_v
        d = np.abs(np.asarray(L.vcoords)[nodes] - np.asarray(L.pcoords)[i]).max(axis=1)
        assert np.all(d <= h + 1e-12)


@pytest.mark.parametrize("case", list(CASES))
def test_same_color_blocks_neither_overlap_nor_couple(case):
    p = CASES[case]()
    L = _hier(p).levels[0]
    V = L.vanka
    M = abs(sp.csr_matrix(L.full_matrix()))
    for c in range(int(V["colors"].max()) + 1):
        idx = np.flatnonzero(V["colors"] == c)
        owner = np.full(L.N, -1)
        for b in idx:
            assert np.all(owner[V["blocks"][b]] == -1)   # no overlap
            owner[V["blocks"][b]] = b
        for b in idx:
            T = V["blocks"][b]
            touched = np.unique(M[T].indices)
            others = owner[touched]
            assert np.all((others == -1) | (others == b))   # no coupling through A


@pytest.mark.parametrize("case", list(CASES))
def test_colored_sweep_equals_block_by_block_sweep(case):
    p = CASES[case]()
    H = _hier(p)
    L = H.levels[0]
    b = uniform_pm1(3, L.N * 2).reshape(L.N, 2)
    x = uniform_pm1(4, L.N * 2).reshape(L.N, 2)
    y1 = vanka_sweep(L, H.params, b, x)
    y2 = np.column_stack([vanka_sweep_sequential(L, H.params, b[:, k], x[:, k]) for k in range(2)])
    assert np.abs(y1 - y2).max() <= 1e-12 * np.abs(y2).max()


def test_a_block_with_omega_one_solves_its_local_system_exactly():
    """x <- x + R^T (R A R^T)^-1 R (f - A x) makes R (f - A x) = 0."""
    p = oseen_recirculating_2d(8, Re=10.0, nrhs=1)
    L = _hier(p).levels[0]
    V = L.vanka
    M = V["M"]
    f = uniform_pm1(5, L.N)
    x = uniform_pm1(6, L.N)
    for bi in (0, 17, L.n_p // 2, L.n_p - 1):
        T = V["blocks"][bi]
        y = x.copy()
        y[T] += V["inv"][bi] @ (f - M @ x)[T]
        assert np.abs((f - M @ y)[T]).max() <= 1e-12 * np.abs(f).max() * 10


def test_dirichlet_dofs_are_exact_after_a_sweep():
    p = stokes_lid_2d(8, nrhs=1)
    H = _hier(p)
    L = H.levels[0]
    b = uniform_pm1(7, L.N)
    y = vanka_sweep(L, H.params, b, np.zeros(L.N))
    D = L.vanka["dirichlet"]
    assert np.array_equal(y[D], b[D])


@pytest.mark.parametrize("case", ["pinned", "lid", "oseen"])
@pytest.mark.parametrize("n", [2, 4, 8])
def test_vanka_fgmres_equals_dense_solve(case, n):
    p = {"pinned": lambda: stokes_pinned_2d(n, nrhs=2),
         "lid": lambda: stokes_lid_2d(n, nrhs=2),
         "oseen": lambda: oseen_recirculating_2d(n, Re=10.0, nrhs=2)}[case]()
    H = _hier(p)
    x, its, rel, _ = fgmres(H, p.b, rtol=1e-12, maxit=400)
    A = p.full_matrix().toarray()
    xd = np.linalg.lstsq(A, p.b, rcond=None)[0]
    nu = p.dim * p.n_v
    if p.pinned < 0:   # pressure up to a constant
        x = x.copy()
        x[nu:] -= x[nu:].mean(axis=0)
        xd[nu:] -= xd[nu:].mean(axis=0)
    assert np.all(np.linalg.norm(x - xd, axis=0) <= 1e-9 * np.linalg.norm(xd, axis=0))


@pytest.mark.parametrize("n,paper_its", [(8, 11), (16, 12), (32, 14), (64, 15)])
def test_table1_vanka_iterations(n, paper_its):
    """Table 1, Vanka(1,1), GMRES to 1e-6 on the leaky lid cavity of (-1,1)^2 with zero
    body force: at most 1.25x the paper's count (the coarsest solve here is the
    pseudo-inverse, the paper relaxes there with Vanka)."""
    p = stokes_lid_2d(n, nrhs=1, body="none", lo=-1.0, hi=1.0)
    H = _hier(p)
    x, its, rel, _ = fgmres(H, p.b, rtol=1e-6)
    assert its[0] <= 1.25 * paper_its, (its, paper_its)
    assert its[0] >= 0.6 * paper_its, (its, paper_its)


@pytest.mark.parametrize("case", ["pinned", "lid", "oseen"])
@pytest.mark.parametrize("smoother", ["bs", "vanka"])
def test_coarsest_vanka_relaxation_fgmres_equals_dense_solve(case, smoother):
    """The paper's coarsest treatment (Section 6.1: Vanka relaxation instead of a direct
    solve), Params.coarse = "vanka": FGMRES with that preconditioner still reaches the
    dense solution (it is a fixed linear preconditioner)."""
    n = 4
    p = {"pinned": lambda: stokes_pinned_2d(n, nrhs=2), "lid": lambda: stokes_lid_2d(n, nrhs=2),
         "oseen": lambda: oseen_recirculating_2d(n, Re=10.0, nrhs=2)}[case]()
    prm = Params(smoother=smoother, pre=1, post=1, coarse="vanka") if smoother == "vanka" else Params(coarse="vanka")
    H = setup_hierarchy(p, prm)
    x, its, rel, _ = fgmres(H, p.b, rtol=1e-12, maxit=400)
    A = p.full_matrix().toarray()
    xd = np.linalg.lstsq(A, p.b, rcond=None)[0]
    nu = p.dim * p.n_v
    if p.pinned < 0:
        x = x.copy()
        x[nu:] -= x[nu:].mean(axis=0)
        xd[nu:] -= xd[nu:].mean(axis=0)
    assert np.all(np.linalg.norm(x - xd, axis=0) <= 1e-9 * np.linalg.norm(xd, axis=0))


def test_coarsest_vanka_relaxation_is_pre_plus_post_steps_from_zero():
    """On a one-level hierarchy the cycle is the coarsest treatment alone: pre + post
    Vanka steps from x = 0, which contract the error of the coarsest system."""
    p = stokes_pinned_2d(2, nrhs=1)
    H = setup_hierarchy(p, Params(smoother="vanka", pre=1, post=2, coarse="vanka"))
    assert len(H.levels) == 1
    L = H.levels[0]
    b = p.b
    x = np.zeros_like(b)
    for _ in range(3):
        x = vanka_sweep(L, H.params, b, x)
    assert np.array_equal(vcycle(H, b), x)
    xd = np.linalg.solve(p.full_matrix().toarray(), b)
    assert np.linalg.norm(x - xd) < 0.9 * np.linalg.norm(xd)
