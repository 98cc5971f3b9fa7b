"""Numeric setup on the GPU (amg_params.device_setup = 1, the default).

  * amg_hierarchy_create_reuse with the device path forms the filtered matrices,
    EMIN steps, restrictions, Galerkin products and Braess-Sarazin data on the
    GPU: every pattern equals the host reuse's exactly and every value agrees
    to 1e-11 of the operator's scale (Stokes with R = P^T, the pinned problem,
    Oseen with Petrov-Galerkin restriction), and FGMRES runs the same solve.
  * The dense Gauss-Seidel maps of small levels, formed on the GPU by the same
    ordered sweep, equal the host's to 1e-12.
The host setup is itself pinned to the oracle (test_setup_parity.py).
"""
import time

import numpy as np
import pytest
import scipy.sparse as sp

from synth import make_problem, stokes_lid_2d, oseen_recirculating_2d

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1607_02489_gb300")

MATS = ["A", "B", "Bt", "S", "P", "Pp", "R", "Rp"]


@pytest.fixture(scope="module", autouse=True)
def gpu_and_lib():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    g._build.build()
    g.load()


def _csr(t):
    rp, col, val, shape = t
    return sp.csr_matrix((val, col, rp), shape=shape)


PAIRS = {
    # (problem the coarsening is built for, problem of the same structure it is reused on)
    "stokes_lid48": (lambda: stokes_lid_2d(48, nrhs=2), lambda: make_problem(48, 2, 0.0, 1.0, bc="lid", nu=0.37,
                                                                           nrhs=2, seed=3)),
    "stokes_pinned16": (lambda: make_problem(16, 2, 0.0, 1.0, pin=True, nrhs=1),
                        lambda: make_problem(16, 2, 0.0, 1.0, pin=True, nu=2.5, nrhs=1, seed=4)),
    "oseen32": (lambda: oseen_recirculating_2d(32, Re=10.0, nrhs=2), lambda: oseen_recirculating_2d(32, Re=100.0,
                                                                                                     nrhs=2)),
}


def _compare_levels(Hd, Hh):
    assert Hd.num_levels() == Hh.num_levels()
    for l in range(Hh.num_levels()):
        last = l + 1 == Hh.num_levels()
        ref = max(abs(_csr(Hh.level_matrix(l, nm))).max() for nm in ("A", "B"))
        for nm in MATS[:4] + ([] if last else MATS[4:]):
            D, H = _csr(Hd.level_matrix(l, nm)), _csr(Hh.level_matrix(l, nm))
            assert np.array_equal(D.indptr, H.indptr) and np.array_equal(D.indices, H.indices), (l, nm)
            scale = ref if nm in ("A", "B", "Bt") else max(abs(H).max(), 1e-300)
            if nm == "S":
                scale = max(abs(H).max(), abs(_csr(Hh.level_matrix(0, "S"))).max())
            assert abs(D - H).max() <= 1e-11 * scale, (l, nm, abs(D - H).max(), scale)
        pd, ph = Hd.level_points(l), Hh.level_points(l)
        assert np.array_equal(pd["colors"], ph["colors"]) and np.array_equal(pd["Cp"], ph["Cp"])
        assert np.abs(pd["D"] - ph["D"]).max() <= 1e-12 * np.abs(ph["D"]).max()
    X, Xh = Hd.coarse_inverse(), Hh.coarse_inverse()
    assert np.linalg.norm(X - Xh) <= 1e-10 * np.linalg.norm(Xh)


@pytest.mark.parametrize("case", list(PAIRS))
def test_device_reuse_matches_host_reuse(case):
    p0, p1 = PAIRS[case][0](), PAIRS[case][1]()
    k = p1.b.shape[1]
    H0d = g.Hierarchy(p0, max_nrhs=k)
    H0h = g.Hierarchy(p0, host_only=1)
    Hd = g.Hierarchy(p1, reuse=H0d, max_nrhs=k)
    Hh = g.Hierarchy(p1, reuse=H0h, host_only=1)
    _compare_levels(Hd, Hh)
    # a second reuse along the sequence shares the device plan and stays exact
    Hd2 = g.Hierarchy(p1, reuse=Hd, max_nrhs=k)
    _compare_levels(Hd2, Hh)
    # the same solve as with the host-built reuse
    Hhs = g.Hierarchy(p1, reuse=g.Hierarchy(p0, max_nrhs=k, device_setup=0), max_nrhs=k, device_setup=0)
    b = torch.tensor(p1.b, device="cuda")
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    st1, its1, rel1 = Hd.fgmres(b, x1, rtol=1e-9)
    st2, its2, rel2 = Hhs.fgmres(b, x2, rtol=1e-9)
    assert st1 == g.AMG_OK and st2 == g.AMG_OK
    assert np.all(np.abs(its1 - its2) <= 1), (its1, its2)
    assert ((x1 - x2).norm() / x2.norm()).item() <= 1e-7


@pytest.mark.parametrize("n", [32, 64])
def test_device_dense_gauss_seidel_maps_equal_the_hosts(n):
    p = stokes_lid_2d(n, nrhs=1)
    Hd = g.Hierarchy(p, max_nrhs=1)
    Hh = g.Hierarchy(p, host_only=1)
    checked = 0
    for l in range(Hh.num_levels() - 1):
        if Hh.level_info(l)["n_p"] > 4608:
            continue
        Md, Mh = Hd.level_gs_map(l), Hh.level_gs_map(l)
        assert Md.shape == Mh.shape
        assert np.linalg.norm(Md - Mh) <= 1e-12 * np.linalg.norm(Mh), (l, np.linalg.norm(Md - Mh))
        checked += 1
    assert checked >= 2


def test_setup_times_at_256():
    """Not a pass/fail check of speed: prints the host and device setup times of the
    592,387-dof lid cavity (fresh, and reused for the next matrix of a sequence)."""
    p = stokes_lid_2d(256, nrhs=1)
    q = make_problem(256, 2, 0.0, 1.0, bc="lid", nu=0.5, nrhs=1, seed=1)
    out = {}
    for dev in (0, 1):
        t = time.perf_counter()
        H = g.Hierarchy(p, max_nrhs=1, device_setup=dev)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        H2 = g.Hierarchy(q, reuse=H, max_nrhs=1, device_setup=dev)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out[dev] = (t1 - t, t2 - t1)
        del H2, H
    print(f"\nsetup at 256x256: host fresh {out[0][0]:.3f} s reuse {out[0][1]:.3f} s; "
          f"device fresh {out[1][0]:.3f} s reuse {out[1][1]:.3f} s")
