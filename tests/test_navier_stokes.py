"""Steady Navier-Stokes lid cavity (Section 6.2): the Picard generator of the test
systems (synth.navier_stokes) and the oracle's AMG on them against Table 5.

Pins: the discrete-wind assembly equals the analytic-wind assembly for a wind
the Q2 space holds exactly; the Picard sequence reaches the paper's 1e-8
nonlinear residual; on the last Picard system the oracle's GMRES (to a relative
1e-6, the paper's tolerance) with Vanka(1,1), BS(2,2) and ILU(1)(1,1) needs at
most 1.25 x the iteration counts of Table 5; with BS(2,2) at least as many as
Table 1 shows for the Stokes problem on the same mesh (the paper's Navier-Stokes
counts exceed its Stokes counts everywhere); and it keeps Table 5's trends (more
iterations at the smaller viscosity; Vanka no worse than Braess-Sarazin; ILU(1)
no worse than Braess-Sarazin).

There is no lower band tied to Table 5: the oracle's counts sit at 45-75% of the
paper's (its Vanka counts at nu = 0.01, 13-14, do not even rise above its Stokes
ones as the paper's do), and none of the explanations at hand closes
that gap.  The
coarsest level (exact here, Vanka in the paper) moves them by at most 3.  The
stopping test matters more: the paper names a residual tolerance of 1e-6 without
saying relative; read as an absolute ||r|| <= 1e-6 (||b|| is 4-8 on these
systems) the counts rise by 15-25% (Vanka 16/16/16/31 and BS 18/19/18/47 on
8x8-32x32 at nu = 0.01 and 16x16 at nu = 0.002, against 20/26/22/49 and
19/22/26/55), still below the paper's.  The Gauss-Seidel order is not it either:
relaxing S's rows in index order (oracle Params(gs_order="natural")) leaves the
BS(2,2) counts of all five systems unchanged."""
import numpy as np
import pytest

from synth import make_problem, picard_lid_cavity
from synth.q2q1 import assemble
from oracle import Params, fgmres, setup_hierarchy

# Table 1 (Stokes lid cavity): (Vanka(1,1), BS(2,2)) iterations per mesh (BS used)
TABLE1 = {8: (11, 9), 16: (12, 10), 32: (14, 14)}
# Table 5 (Navier-Stokes lid cavity): (Vanka(1,1), BS(2,2)) iterations
TABLE5 = {(8, 0.01): (20, 19), (16, 0.01): (26, 22), (32, 0.01): (22, 26),
          (16, 0.002): (49, 55), (32, 0.002): (53, 60)}
# its ILU(1)(1,1) column (reverse Cuthill-McKee order)
TABLE5_ILU = {(8, 0.01): 6, (16, 0.01): 7, (32, 0.01): 9, (16, 0.002): 9, (32, 0.002): 13}


def test_discrete_wind_assembly_equals_analytic_for_a_q2_wind():
    """w = (x y, x^2 - y) lies in Q2: its nodal interpolant gives the same convection matrix."""
    n = 6
    wind = lambda X: np.stack([X[..., 0] * X[..., 1], X[..., 0] ** 2 - X[..., 1]], axis=-1)  # noqa: E731
    A1, _, vX, _, _, _, _ = assemble(n, 2, -1.0, 1.0, nu=0.3, wind=wind)
    wn = wind(np.asarray(vX)).T
    A2, _, _, _, _, _, _ = assemble(n, 2, -1.0, 1.0, nu=0.3, wind_nodal=wn)
    assert abs(A1 - A2).max() <= 1e-13 * abs(A1).max()


@pytest.fixture(scope="module")
def picard_systems():
    return {key: picard_lid_cavity(*key) for key in TABLE5}


def test_picard_reaches_the_nonlinear_tolerance(picard_systems):
    for key, (last, x, hist) in picard_systems.items():
        assert hist[-1] < 1e-8, (key, hist[-5:])
        assert hist[0] > 1e-4, key          # the Stokes start is not a Navier-Stokes solution
        # the final iterate solves the nonlinear equations: its own Oseen system has a small residual
        q = make_problem(key[0], 2, -1.0, 1.0, bc="lid", nu=key[1], body="none",
                         wind_nodal=x[:2 * last.n_v].reshape(2, last.n_v))
        assert np.linalg.norm(q.b[:, 0] - q.full_matrix() @ x) < 1e-8


def _its(last, prm):
    H = setup_hierarchy(last, prm)
    _, its, rel, _ = fgmres(H, last.b, rtol=1e-6, maxit=300)
    assert rel[0] <= 1e-6
    return int(its[0])


def test_table5_iterations_and_trends(picard_systems):
    vk = Params(smoother="vanka", pre=1, post=1)
    bs = Params()
    ours = {}
    for key, (last, _, _) in picard_systems.items():
        assert not last.symmetric   # Oseen systems: EMIN GMRES for P and R
        v, b = _its(last, vk), _its(last, bs)
        ours[key] = (v, b)
        pv, pb = TABLE5[key]
        sb = TABLE1[key[0]][1]
        assert v <= 1.25 * pv, (key, v, pv)
        assert sb <= b <= 1.25 * pb, (key, b, pb, sb)
        assert v <= b, (key, v, b)
    for n in (16, 32):
        assert ours[(n, 0.002)][0] > ours[(n, 0.01)][0] and ours[(n, 0.002)][1] > ours[(n, 0.01)][1]


def test_table5_ilu_iterations(picard_systems):
    """ILU(1)(1,1) with reverse Cuthill-McKee order on the last Picard systems: at most
    1.25 x Table 5's ILU column and no more iterations than Braess-Sarazin(2,2) on the
    same system (the paper's ILU column is the smallest of Table 5's rows)."""
    il = Params(smoother="ilu", pre=1, post=1)
    for key, (last, _, _) in picard_systems.items():
        i = _its(last, il)
        assert 1 <= i <= 1.25 * TABLE5_ILU[key], (key, i, TABLE5_ILU[key])
        assert i <= _its(last, Params()), key


def test_reused_coarsening_gives_the_fresh_hierarchy_on_the_same_matrix(picard_systems):
    """Reusing a hierarchy on its own matrix reproduces it: same transfers and coarse operators."""
    last = picard_systems[(16, 0.01)][0]
    H = setup_hierarchy(last)
    R = setup_hierarchy(last, reuse=H)
    assert len(R.levels) == len(H.levels)
    for L1, L2 in zip(H.levels[:-1], R.levels[:-1]):
        for nm in ("P", "Pp", "R", "Rp"):
            assert abs(getattr(L1, nm) - getattr(L2, nm)).max() == 0.0
    assert abs(H.levels[-1].full_matrix() - R.levels[-1].full_matrix()).max() == 0.0


def test_picard_with_reused_coarsening_keeps_its_iterations(picard_systems):
    """The coarsening of the first Oseen step reused for the last Picard system: the
    patterns stay valid (P 1 = 1 on every level) and GMRES needs at most two more
    iterations than with a fresh setup."""
    last = picard_systems[(32, 0.01)][0]
    first = make_problem(32, 2, -1.0, 1.0, bc="lid", nu=0.01, body="none",
                         wind_nodal=np.zeros((2, last.n_v)) + 1e-3)
    H0 = setup_hierarchy(first)
    Hr = setup_hierarchy(last, reuse=H0)
    Hf = setup_hierarchy(last)
    for L in Hr.levels[:-1]:
        ones = np.ones(L.P.shape[1])
        rows = ~np.asarray(L.dirichlet, dtype=bool)
        assert np.abs((L.P @ ones)[rows] - 1.0).max() <= 1e-12
    _, its_r, rel_r, _ = fgmres(Hr, last.b, rtol=1e-6)
    _, its_f, _, _ = fgmres(Hf, last.b, rtol=1e-6)
    assert rel_r[0] <= 1e-6 and its_r[0] <= its_f[0] + 2, (its_r, its_f)
