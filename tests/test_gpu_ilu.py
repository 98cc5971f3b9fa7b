"""GPU parity of the ILU(1) smoother (Section 5, amg_params.smoother = 2) through the
C ABI against the oracle's ILU V-cycle and FGMRES.

Tolerances as for the other smoothers (test_gpu_parity.py): FP64 V-cycle relative
2-norm error <= 1e-11 per column; FP32 V-cycle <= 1e-4; FGMRES
iterations within +-1 (FP64 cycle), true residual re-checked on the host.  The
substitutions are sync-free (rows wait on the values they need), but each row's
sum runs in a fixed lane order, so a cycle is deterministic."""
import numpy as np
import pytest

from synth import make_problem, oseen_recirculating_2d, picard_lid_cavity, stokes_lid_2d, stokes_pinned_2d, uniform_pm1
from oracle import Params, fgmres, setup_hierarchy, vcycle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1607_02489_gb300")

IL = dict(smoother=2, pre=1, post=1)
ILO = Params(smoother="ilu", pre=1, post=1)

CASES = {
    "pinned16": lambda: stokes_pinned_2d(16, nrhs=1),
    "lid32": lambda: stokes_lid_2d(32, nrhs=2),
    # reverse Cuthill-McKee order; its coarse level has zero-block pivots no elimination reaches
    "oseen32": lambda: oseen_recirculating_2d(32, Re=100.0, nrhs=4),
    "lid18_ragged3": lambda: make_problem(18, 2, 0.0, 1.0, bc="lid", nrhs=3, seed=5),
    "lid3d": lambda: make_problem(4, 3, 0.0, 1.0, bc="lid", nrhs=1),
}


@pytest.fixture(scope="module", autouse=True)
def gpu_and_lib():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    g._build.build()
    g.load()


def _relerr(a, b):
    return np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300)


@pytest.mark.parametrize("case", list(CASES))
def test_ilu_vcycle_fp64_matches_oracle(case):
    p = CASES[case]()
    Ho = setup_hierarchy(p, ILO)
    Hg = g.Hierarchy(p, max_nrhs=p.b.shape[1], **IL)
    r = uniform_pm1(41, p.N * p.b.shape[1]).reshape(p.N, -1)
    zo = vcycle(Ho, r)
    rt = torch.tensor(r, device="cuda")
    zt = torch.empty_like(rt)
    Hg.vcycle(rt, zt)
    torch.cuda.synchronize()
    err = _relerr(zt.cpu().numpy(), zo)
    print(f"\nFP64 ILU(1) V-cycle vs oracle, {case}: max relative error {err.max():.2e}")
    assert np.all(err <= 1e-11), err
    z2 = torch.empty_like(rt)
    Hg.vcycle(rt, z2)
    torch.cuda.synchronize()
    assert torch.equal(zt, z2)


@pytest.mark.parametrize("case", ["lid32", "lid3d"])
def test_ilu_location_order_vcycle_matches_oracle(case):
    """The alternative order (amg_params.ilu_order = 1) against the oracle's."""
    p = CASES[case]()
    Ho = setup_hierarchy(p, Params(smoother="ilu", pre=1, post=1, ilu_order="location"))
    Hg = g.Hierarchy(p, max_nrhs=p.b.shape[1], ilu_order=1, **IL)
    r = uniform_pm1(44, p.N * p.b.shape[1]).reshape(p.N, -1)
    zo = vcycle(Ho, r)
    rt = torch.tensor(r, device="cuda")
    zt = torch.empty_like(rt)
    Hg.vcycle(rt, zt)
    torch.cuda.synchronize()
    err = _relerr(zt.cpu().numpy(), zo)
    assert np.all(err <= 1e-11), err


@pytest.mark.parametrize("K", [1, 8, 32])
def test_ilu_vcycle_lane_groups(K):
    """Every lane split of a row (32 / K groups of K lanes): K = 1, 8 and 32 columns."""
    p = stokes_lid_2d(16, nrhs=1)
    Ho = setup_hierarchy(p, ILO)
    Hg = g.Hierarchy(p, max_nrhs=K, **IL)
    r = uniform_pm1(42, p.N * K).reshape(p.N, K)
    zo = vcycle(Ho, r)
    rt = torch.tensor(r, device="cuda")
    zt = torch.empty_like(rt)
    Hg.vcycle(rt, zt)
    torch.cuda.synchronize()
    err = _relerr(zt.cpu().numpy(), zo)
    assert np.all(err <= 1e-11), err


@pytest.mark.parametrize("case", ["lid32", "oseen32"])
def test_ilu_vcycle_fp32_close_to_oracle(case):
    p = CASES[case]()
    Ho = setup_hierarchy(p, ILO)
    Hg = g.Hierarchy(p, max_nrhs=p.b.shape[1], vcycle_fp32=1, **IL)
    r = uniform_pm1(43, p.N * p.b.shape[1]).reshape(p.N, -1)
    zo = vcycle(Ho, r)
    rt = torch.tensor(r, device="cuda")
    zt = torch.empty_like(rt)
    Hg.vcycle(rt, zt)
    torch.cuda.synchronize()
    err = _relerr(zt.cpu().numpy(), zo)
    assert np.all(err <= 1e-4) and np.all(err > 0), err


@pytest.mark.parametrize("case", ["pinned16", "lid32", "oseen32"])
@pytest.mark.parametrize("fp32", [0, 1])
def test_ilu_fgmres_matches_oracle(case, fp32):
    p = CASES[case]()
    Ho = setup_hierarchy(p, ILO)
    xo, its_o, rel_o, _ = fgmres(Ho, p.b, rtol=1e-8)
    Hg = g.Hierarchy(p, max_nrhs=p.b.shape[1], vcycle_fp32=fp32, **IL)
    bt = torch.tensor(p.b, device="cuda")
    xt = torch.zeros_like(bt)
    st, its, rel = Hg.fgmres(bt, xt, rtol=1e-8, restart=100, maxit=300)
    assert st == g.AMG_OK and np.all(rel <= 1e-8)
    if not fp32:
        assert np.all(np.abs(its - its_o) <= 1), (its, its_o)
    else:
        assert np.all(its <= its_o + 2), (its, its_o)
    A = p.full_matrix()
    x = xt.cpu().numpy()
    assert np.all(np.linalg.norm(p.b - A @ x, axis=0) <= 1.01e-8 * np.linalg.norm(p.b, axis=0))


def test_ilu_on_a_navier_stokes_picard_system():
    """The last Picard system of the lid cavity at nu = 0.01 on 16x16 (Table 5's second
    row): reverse Cuthill-McKee order on a non-symmetric matrix, FGMRES to the paper's
    1e-6 in the oracle's iterations +-1."""
    last, _, _ = picard_lid_cavity(16, 0.01)
    Ho = setup_hierarchy(last, ILO)
    _, its_o, _, _ = fgmres(Ho, last.b, rtol=1e-6)
    Hg = g.Hierarchy(last, max_nrhs=1, **IL)
    bt = torch.tensor(last.b, device="cuda")
    xt = torch.zeros_like(bt)
    st, its, rel = Hg.fgmres(bt, xt, rtol=1e-6, restart=100, maxit=300)
    assert st == g.AMG_OK and np.all(np.abs(its - its_o) <= 1), (its, its_o)
    x = xt.cpu().numpy()
    assert np.linalg.norm(last.b - last.full_matrix() @ x) <= 1.01e-6 * np.linalg.norm(last.b)


def test_ilu_profile_counts_its_launches():
    p = stokes_lid_2d(32, nrhs=1)
    Hg = g.Hierarchy(p, max_nrhs=1, **IL)
    b = torch.tensor(p.b, device="cuda")
    z = torch.empty_like(b)
    Hg.vcycle(b, z)
    ms, cnt = Hg.profile_vcycle(1, reps=2)
    il = g.KERNEL_CLASSES.index("ilu")
    gs = g.KERNEL_CLASSES.index("gs_color")
    # two substitutions per step, pre 1 + post 1 steps per cycle, 2 cycles
    assert cnt[0, il] == 2 * 2 * 2 and cnt[:, gs].sum() == 0
