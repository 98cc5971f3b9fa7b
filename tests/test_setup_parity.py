"""Host-side parity of the library's C++ hierarchy setup with the oracle (no GPU).

The library is built with host_only=1, so nothing is uploaded; the C/F
splits, patterns and colors must be identical (integer work: bit-exact) and
the matrices equal to rounding.
"""
import os
import re
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from synth import stokes_lid_2d, stokes_pinned_2d, oseen_recirculating_2d, make_problem, with_perturbed_coordinates
from oracle import setup_hierarchy, Params

g = pytest.importorskip("paper_1607_02489_gb300")
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module", autouse=True)
def built():
    g._build.build()
    g.load()


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "emin_amg.h")).read()
    declared = sorted(set(re.findall(r"\b(amg_[a-z_]+)\s*\(", hdr)))
    assert len(declared) >= 12
    lib = g.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(g.EXPORTED) == declared
    out = subprocess.run(["nm", "-D", "--defined-only", g.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (amg_[a-z_]+)", out))
    assert set(declared) <= exported


def _csr(t):
    rp, col, val, shape = t
    return sp.csr_matrix((val, col, rp), shape=shape)


def _compare(prob, prm=None, reuse=None, **kw):
    """Library setup (host only) against the oracle's; reuse = (library hierarchy,
    oracle hierarchy) whose coarsening both reuse."""
    if reuse is None:
        Hg = g.Hierarchy(prob, host_only=1, **kw)
        Ho = setup_hierarchy(prob, prm or Params())
    else:
        Hg = g.Hierarchy(prob, host_only=1, reuse=reuse[0], **kw)
        Ho = setup_hierarchy(prob, prm or Params(), reuse=reuse[1])
    assert Hg.num_levels() == len(Ho.levels)
    for l, L in enumerate(Ho.levels):
        info = Hg.level_info(l)
        pts = Hg.level_points(l)
        assert (info["n_v"], info["n_p"], info["pinned"]) == (L.n_v, L.n_p, L.pinned)
        assert np.array_equal(pts["colors"], L.colors)
        assert info["n_colors"] == int(L.colors.max()) + 1
        assert info["gs_strip"] == L.gs_strip
        assert np.abs(pts["D"] - L.D).max() <= 1e-12 * np.abs(L.D).max()
        last = l + 1 == len(Ho.levels)
        if not last:
            assert np.array_equal(pts["Cp"], L.info["Cp"])
            assert np.array_equal(pts["Cv"], L.info["Cv"])
        # tolerances relative to the level's operator scale (a coarsest level with a single
        # pressure has B and S at rounding level, where a relative comparison means nothing)
        scale = abs(L.full_matrix()).max()
        s_scale = max(abs(L.S).max(), abs(Ho.levels[0].S).max())
        for nm in ["A", "B", "Bt", "S"] + ([] if last else ["P", "Pp", "R", "Rp"]):
            M = _csr(Hg.level_matrix(l, nm))
            O = sp.csr_matrix(getattr(L, nm))
            O.sort_indices()
            assert np.array_equal(M.indptr, O.indptr) and np.array_equal(M.indices, O.indices), (l, nm)
            ref = {"A": scale, "B": scale, "Bt": scale, "S": s_scale}.get(nm, abs(O).max())
            assert abs(M - O).max() <= 1e-11 * ref, (l, nm, abs(M - O).max(), ref)
    # the coarsest pseudo-inverse: both sides refine their SVD's result (Newton-Schulz with
    # residuals in extended precision), so they agree well below cond * u, which reaches
    # 1e-9 on the pinned problems.  On singular levels what refinement cannot reach is the
    # SVD's tilt of the kept singular vectors towards the null space (u ||A|| / gap).
    X, Xo = Hg.coarse_inverse(), Ho.levels[-1].coarse_pinv
    assert np.linalg.norm(X - Xo) <= 1e-11 * np.linalg.norm(Xo), np.linalg.norm(X - Xo) / np.linalg.norm(Xo)


@pytest.mark.parametrize("n", [8, 16, 32, 64])
def test_stokes_lid_setup_matches_oracle(n):
    _compare(stokes_lid_2d(n, nrhs=1))


@pytest.mark.parametrize("n", [8, 16, 32])
def test_stokes_pinned_setup_matches_oracle(n):
    _compare(stokes_pinned_2d(n))


@pytest.mark.parametrize("Re", [1.0, 10.0, 100.0])
def test_oseen_setup_matches_oracle(Re):
    _compare(oseen_recirculating_2d(32, Re=Re, nrhs=1))


def test_ragged_mesh_and_parameters_match_oracle():
    """A mesh size not divisible by 4 (ragged coarsening at the far edges), and non-default
    tau1 / tau2 / omega placement."""
    p = make_problem(18, 2, 0.0, 1.0, bc="lid", nrhs=1)
    _compare(p)
    _compare(p, Params(tau1=0.1, tau2sq=0.04, omega_in_M="inverse"), tau1=0.1, tau2sq=0.04, omega_on_D=1)


def test_3d_setup_matches_oracle():
    _compare(make_problem(4, 3, 0.0, 1.0, bc="lid", nrhs=1))


def test_invalid_problem_is_rejected():
    p = stokes_lid_2d(4, nrhs=1)
    bad = stokes_lid_2d(4, nrhs=1)
    bad.A = bad.A.copy()
    bad.A.indices = bad.A.indices.copy()
    r = int(np.flatnonzero(np.diff(bad.A.indptr) >= 2)[0])
    t = bad.A.indptr[r]
    bad.A.indices[t], bad.A.indices[t + 1] = bad.A.indices[t + 1], bad.A.indices[t]   # columns out of order
    with pytest.raises(g.AmgError) as e:
        g.Hierarchy(bad, host_only=1)
    assert e.value.status == -1
    with pytest.raises(g.AmgError):
        g.Hierarchy(p, host_only=1, max_nrhs=64)
    H = g.Hierarchy(p, host_only=1)
    assert H.num_levels() >= 1


def test_3d_setup_matches_oracle_at_8():
    _compare(make_problem(8, 3, 0.0, 1.0, bc="lid", nrhs=1))


@pytest.mark.parametrize("case", ["lid32", "pinned16", "oseen32", "lid18", "lid3d"])
def test_vanka_blocks_and_colors_match_oracle(case):
    """The library's Vanka setup (smoother = 1) against the oracle's: the same blocks
    (dofs in the same order) and the same greedy colors on every smoothed level."""
    from synth import stokes_pinned_2d, oseen_recirculating_2d
    prob = {"lid32": lambda: stokes_lid_2d(32, nrhs=1), "pinned16": lambda: stokes_pinned_2d(16, nrhs=1),
            "oseen32": lambda: oseen_recirculating_2d(32, Re=100.0, nrhs=1),
            "lid18": lambda: make_problem(18, 2, 0.0, 1.0, bc="lid", nrhs=1),
            "lid3d": lambda: make_problem(4, 3, 0.0, 1.0, bc="lid", nrhs=1)}[case]()
    Ho = setup_hierarchy(prob, Params(smoother="vanka", pre=1, post=1))
    Hg = g.Hierarchy(prob, host_only=1, smoother=1, pre=1, post=1)
    assert Hg.num_levels() == len(Ho.levels)
    for l, L in enumerate(Ho.levels[:-1]):
        V = Hg.level_vanka(l)
        blocks = L.vanka["blocks"]
        assert len(V["ptr"]) - 1 == len(blocks)
        for b, T in enumerate(blocks):
            assert np.array_equal(V["dofs"][V["ptr"][b]:V["ptr"][b + 1]], T), (l, b)
        assert np.array_equal(V["colors"], L.vanka["colors"]), l
        assert V["ncolors"] == int(L.vanka["colors"].max()) + 1
    with pytest.raises(g.AmgError):
        Hg.level_vanka(len(Ho.levels) - 1)


def test_gs_variant_calls_need_a_device_hierarchy():
    """amg_set_gs_variant on a host-only hierarchy is an argument error; amg_gs_variant
    reports -1 there (no cycle was built)."""
    H = g.Hierarchy(stokes_lid_2d(8, nrhs=1), host_only=1)
    with pytest.raises(g.AmgError) as exc:
        H.set_gs_variant(0, 1, "pipelined", 0)
    assert exc.value.status == -1 and "host-only" in str(exc.value)
    assert all(v == "not chosen" for v, _, _ in H.gs_variants(1))


def test_vanka_inverses_over_the_limit_fail_setup():
    """Setup refuses a level whose FP64 Vanka block inverses exceed amg_params.vanka_max_mib
    (large 3D blocks) with AMG_ERR_SETUP and a message naming the size; the same problem
    builds under the default limit, and a non-positive limit is an argument error."""
    prob = make_problem(4, 3, 0.0, 1.0, bc="lid", nrhs=1)
    g.Hierarchy(prob, host_only=1, smoother=1, pre=1, post=1)  # a few MiB: within 16 GiB
    with pytest.raises(g.AmgError) as exc:
        g.Hierarchy(prob, host_only=1, smoother=1, pre=1, post=1, vanka_max_mib=0.01)
    assert exc.value.status == -4 and "MiB, more than the limit" in str(exc.value)
    with pytest.raises(g.AmgError) as exc:
        g.Hierarchy(prob, host_only=1, smoother=1, vanka_max_mib=0.0)
    assert exc.value.status == -1


@pytest.mark.parametrize("case", ["lid32", "pinned16", "oseen32"])
def test_coarsest_vanka_blocks_match_oracle(case):
    """coarse = 1 (the paper's Vanka relaxation of the coarsest level): the coarsest level
    carries the same blocks and colors as the oracle's, with either smoother."""
    from synth import stokes_pinned_2d, oseen_recirculating_2d
    prob = {"lid32": lambda: stokes_lid_2d(32, nrhs=1), "pinned16": lambda: stokes_pinned_2d(16, nrhs=1),
            "oseen32": lambda: oseen_recirculating_2d(32, Re=100.0, nrhs=1)}[case]()
    Ho = setup_hierarchy(prob, Params(coarse="vanka"))
    Hg = g.Hierarchy(prob, host_only=1, coarse=1)
    c = len(Ho.levels) - 1
    assert Hg.num_levels() == c + 1
    V = Hg.level_vanka(c)
    blocks = Ho.levels[c].vanka["blocks"]
    assert len(V["ptr"]) - 1 == len(blocks)
    for b, T in enumerate(blocks):
        assert np.array_equal(V["dofs"][V["ptr"][b]:V["ptr"][b + 1]], T), b
    assert np.array_equal(V["colors"], Ho.levels[c].vanka["colors"])
    with pytest.raises(g.AmgError):
        Hg.level_vanka(0)   # Braess-Sarazin levels carry no blocks



def test_reused_coarsening_matches_oracle():
    """amg_hierarchy_create_reuse against the oracle's reuse: the coarsening of one Oseen
    matrix kept for another of the same structure (another wind), EMIN / RAP redone."""
    from synth import make_problem as mk
    n = 16
    nv = (2 * n + 1) ** 2
    X = np.linspace(-1, 1, 2 * n + 1)
    xx, yy = np.meshgrid(X, X)
    w1 = np.stack([yy.ravel() * (1 - xx.ravel() ** 2), -xx.ravel() * (1 - yy.ravel() ** 2)])
    first = mk(n, 2, -1.0, 1.0, bc="lid", nu=0.05, body="none", wind_nodal=w1)
    second = mk(n, 2, -1.0, 1.0, bc="lid", nu=0.02, body="none", wind_nodal=3.0 * w1 + 0.2)
    Hg0 = g.Hierarchy(first, host_only=1)
    Ho0 = setup_hierarchy(first)
    _compare(second, reuse=(Hg0, Ho0))
    # a matrix of another structure is refused
    other = mk(n + 2, 2, -1.0, 1.0, bc="lid", nu=0.02, body="none", wind_nodal=np.zeros((2, (2 * n + 5) ** 2)))
    with pytest.raises(g.AmgError):
        g.Hierarchy(other, host_only=1, reuse=Hg0)
    assert nv == first.n_v


@pytest.mark.parametrize("case", ["lid32", "pinned16", "oseen32", "lid18", "lid3d", "lid32_loc", "lid3d_loc"])
def test_ilu_factors_match_oracle(case):
    """The library's ILU(1) setup (smoother = 2) against the oracle's on every smoothed
    level: the same order (natural for Stokes, reverse Cuthill-McKee for Oseen; integer
    work, bit-exact), the same factor patterns and the factors and pivots to rounding.
    oseen32's coarse level has zero-block pivots that no elimination step reaches; the
    _loc cases take the location order (ilu_order = 1)."""
    loc = case.endswith("_loc")
    case = case.replace("_loc", "")
    prob = {"lid32": lambda: stokes_lid_2d(32, nrhs=1), "pinned16": lambda: stokes_pinned_2d(16, nrhs=1),
            "oseen32": lambda: oseen_recirculating_2d(32, Re=100.0, nrhs=1),
            "lid18": lambda: make_problem(18, 2, 0.0, 1.0, bc="lid", nrhs=1),
            "lid3d": lambda: make_problem(4, 3, 0.0, 1.0, bc="lid", nrhs=1)}[case]()
    Ho = setup_hierarchy(prob, Params(smoother="ilu", pre=1, post=1, ilu_order="location" if loc else "block"))
    Hg = g.Hierarchy(prob, host_only=1, smoother=2, pre=1, post=1, ilu_order=1 if loc else 0)
    assert Hg.num_levels() == len(Ho.levels)
    for l, L in enumerate(Ho.levels[:-1]):
        F = Hg.level_ilu(l)
        I = L.ilu
        n = L.N
        assert np.array_equal(F["perm"], I["perm"]), l
        Lo = sp.csr_matrix(I["L"])
        Uo = sp.csr_matrix(I["U"])
        piv_o = Uo.diagonal()
        Uo = sp.triu(Uo, k=1, format="csr")
        Lg = sp.csr_matrix((F["lower"][2], F["lower"][1], F["lower"][0]), shape=(n, n))
        Ug = sp.csr_matrix((F["upper"][2], F["upper"][1], F["upper"][0]), shape=(n, n))
        for Mg, Mo, nm in ((Lg, Lo, "L"), (Ug, Uo, "U")):
            Mg = Mg.copy()
            Mg.eliminate_zeros()
            Mo.eliminate_zeros()
            Mo.sort_indices()
            assert np.array_equal(Mg.indptr, Mo.indptr) and np.array_equal(Mg.indices, Mo.indices), (l, nm)
            scale = max(abs(Mo).max(), 1e-300)
            assert abs(Mg - Mo).max() <= 1e-11 * scale, (l, nm, abs(Mg - Mo).max(), scale)
        assert np.abs(F["pivots"] - piv_o).max() <= 1e-11 * np.abs(piv_o).max(), l
        assert F["depth_lower"] >= 1 and F["depth_upper"] >= 1
    with pytest.raises(g.AmgError):
        Hg.level_ilu(len(Ho.levels) - 1)


@pytest.mark.parametrize("case", ["lid16", "oseen16"])
def test_ilu_substitution_depths_are_the_longest_dependency_chains(case):
    """The substitutions hand out rows by (dependency level, position); their depths are
    the longest chains of the factors' dependencies (row i after every column j of its
    row in L, or in U for the backward pass), recomputed here from the exported factors."""
    prob = stokes_lid_2d(16, nrhs=1) if case == "lid16" else oseen_recirculating_2d(16, Re=50.0, nrhs=1)
    Hg = g.Hierarchy(prob, host_only=1, smoother=2, pre=1, post=1)
    for l in range(Hg.num_levels() - 1):
        F = Hg.level_ilu(l)
        n = len(F["perm"])
        for (ptr, col, _), lower, depth in ((F["lower"], True, F["depth_lower"]),
                                            (F["upper"], False, F["depth_upper"])):
            lev = np.zeros(n, dtype=np.int64)
            for i in (range(n) if lower else range(n - 1, -1, -1)):
                c = col[ptr[i]:ptr[i + 1]]
                assert np.all(c < i) if lower else np.all(c > i)
                lev[i] = lev[c].max() + 1 if len(c) else 0
            assert depth == lev.max() + 1, (l, lower, depth, lev.max() + 1)


def test_coarsest_vanka_stops_before_a_level_without_pressure_coupling():
    """A level keeping only the constant pressure (the 8^3 lid cube's third level) has B = 0 to
    rounding and a singular Vanka block.  With coarse = 1, coarsening stops before it (library
    and oracle alike); a hierarchy that still ends on such a level (here: coarsening reused from
    one built without the rule) is refused at setup (AMG_ERR_SETUP; the oracle raises)."""
    p = make_problem(8, 3, 0.0, 1.0, bc="lid", nrhs=1)
    H0 = g.Hierarchy(p, host_only=1)
    Ho0 = setup_hierarchy(p)
    assert H0.level_info(H0.num_levels() - 1)["n_p"] == 1 and Ho0.levels[-1].n_p == 1
    Hg = g.Hierarchy(p, host_only=1, coarse=1)
    Ho = setup_hierarchy(p, Params(coarse="vanka"))
    assert Hg.num_levels() == len(Ho.levels) == H0.num_levels() - 1
    assert Hg.level_info(Hg.num_levels() - 1)["n_p"] == Ho.levels[-1].n_p > 1
    V = Hg.level_vanka(Hg.num_levels() - 1)
    assert np.array_equal(V["colors"], Ho.levels[-1].vanka["colors"])
    with pytest.raises(g.AmgError) as e:
        g.Hierarchy(p, host_only=1, coarse=1, reuse=H0)
    assert e.value.status == -4 and "singular" in str(e.value)
    with pytest.raises(ValueError):
        setup_hierarchy(p, Params(coarse="vanka"), reuse=Ho0)


def test_coarsest_vanka_hierarchy_at_256_matches_oracle():
    """The 256x256 lid cavity with coarse = 1: coarsening stops at the 301-dof level (15
    pressures) instead of the 23-dof one-pressure level, in the library as in the oracle."""
    p = stokes_lid_2d(256, nrhs=1)
    Hg = g.Hierarchy(p, host_only=1, coarse=1)
    Ho = setup_hierarchy(p, Params(coarse="vanka"))
    assert Hg.num_levels() == len(Ho.levels) == 4
    c = Hg.level_info(3)
    assert (c["n_v"], c["n_p"]) == (Ho.levels[3].n_v, Ho.levels[3].n_p) == (143, 15)


def test_pinned_coarse_inverse_is_refined_beyond_cond_u():
    """The 16x16 pinned problem's coarsest level is nonsingular but ill-conditioned
    (cond ~ 7.5e6): an SVD alone gives its inverse only to cond * u ~ 1e-9, and two
    SVDs of the same matrix differ by ~1e-10.  After refinement the library's and the
    oracle's inverses agree to ~1e-14."""
    p = stokes_pinned_2d(16)
    Hg = g.Hierarchy(p, host_only=1)
    Ho = setup_hierarchy(p)
    A = Ho.levels[-1].full_matrix().toarray()
    s = np.linalg.svd(A, compute_uv=False)
    assert s[0] / s[-1] > 1e6
    X, Xo = Hg.coarse_inverse(), Ho.levels[-1].coarse_pinv
    raw = np.linalg.pinv(A, rcond=1e-12)
    assert np.linalg.norm(raw - Xo) > 1e-11 * np.linalg.norm(Xo)  # the SVD alone is cond * u away
    assert np.linalg.norm(X - Xo) <= 1e-13 * np.linalg.norm(Xo)


@pytest.mark.parametrize("n, amp, seed", [(16, 0.35, 100), (16, 0.35, 102), (20, 0.2, 100), (20, 0.35, 101)])
def test_perturbed_coordinates_setup_matches_oracle(n, amp, seed):
    """Perturbed node positions make Alg. 3 leave badly covered F-points, which
    find_extra_dist3_Cpoints converts (the oracle reports them): the library's C/F
    splits, with those extra C-points, patterns and values match the oracle's."""
    p = with_perturbed_coordinates(stokes_lid_2d(n, nrhs=1), amp, seed)
    Ho = setup_hierarchy(p)
    assert sum(len(L.info.get("extra_p", [])) for L in Ho.levels[:-1]) >= 2
    _compare(p)
