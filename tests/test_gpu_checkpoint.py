"""GPU side of hierarchy checkpoints (amg_hierarchy_export / amg_hierarchy_import).

  * An exported and re-imported hierarchy runs the same V-cycle bit for bit
    (fixed kernel choices, autotune = 0, on both handles).
  * The oracle's own hierarchy, written in the file format and imported, gives a
    V-cycle that matches the oracle's to 1e-11 and FGMRES iterations within +-1:
    V-cycle parity that does not depend on setup parity.
"""
import numpy as np
import pytest

from synth import stokes_lid_2d, stokes_pinned_2d, oseen_recirculating_2d, uniform_pm1
from oracle import setup_hierarchy, vcycle, fgmres

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1607_02489_gb300")
from hierarchy_file import write_oracle_hierarchy  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def gpu_and_lib():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    g._build.build()
    g.load()


CASES = {
    "lid32": lambda: stokes_lid_2d(32, nrhs=2),
    "pinned16": lambda: stokes_pinned_2d(16, nrhs=1),
    "oseen32": lambda: oseen_recirculating_2d(32, Re=10.0, nrhs=4),
}


def _relerr(a, b):
    return np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300)


@pytest.mark.parametrize("fp32", [0, 1])
def test_reimported_hierarchy_runs_the_same_cycle(fp32, tmp_path):
    p = stokes_lid_2d(64, nrhs=4)
    H = g.Hierarchy(p, max_nrhs=4, autotune=0, vcycle_fp32=fp32)
    path = str(tmp_path / "h.bin")
    H.export(path)
    H2 = g.Hierarchy.from_file(path, max_nrhs=4, autotune=0, vcycle_fp32=fp32)
    r = torch.tensor(uniform_pm1(51, p.N * 4).reshape(p.N, 4), device="cuda")
    z1, z2 = torch.empty_like(r), torch.empty_like(r)
    H.vcycle(r, z1)
    H2.vcycle(r, z2)
    torch.cuda.synchronize()
    assert torch.equal(z1, z2)


@pytest.mark.parametrize("case", list(CASES))
def test_imported_oracle_hierarchy_matches_the_oracle_cycle(case, tmp_path):
    p = CASES[case]()
    Ho = setup_hierarchy(p)
    path = str(tmp_path / "oracle.bin")
    write_oracle_hierarchy(Ho, path)
    k = p.b.shape[1]
    H = g.Hierarchy.from_file(path, max_nrhs=k)
    r = uniform_pm1(52, p.N * k).reshape(p.N, k)
    zo = vcycle(Ho, r)
    rt = torch.tensor(r, device="cuda")
    zt = torch.empty_like(rt)
    H.vcycle(rt, zt)
    torch.cuda.synchronize()
    err = _relerr(zt.cpu().numpy(), zo)
    print(f"\nimported oracle hierarchy, {case}: V-cycle max relative error {err.max():.2e}")
    assert np.all(err <= 1e-11), err
    _, its_o, _, _ = fgmres(Ho, p.b, rtol=1e-8)
    bt = torch.tensor(p.b, device="cuda")
    xt = torch.zeros_like(bt)
    st, its, rel = H.fgmres(bt, xt, rtol=1e-8)
    assert st == g.AMG_OK and np.all(np.abs(its - its_o) <= 1), (its, its_o)
