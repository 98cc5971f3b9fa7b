"""GPU checks at the full sizes of the Oseen and 3D Stokes workloads, where the
oracle is too slow to run: properties that hold at any size, and outputs the
definition computes one by one.

* 2D Oseen, 512x512 mesh (2,364,419 dofs), Re in {1, 10, 100}, 32 right-hand
  sides in one launch, FP32 V-cycle inside FP64 FGMRES to 1e-8:
  every column converges, its true residual recomputed on the host is <= 1e-8,
  the block product A x equals the host product, and the FP32-V-cycle solutions
  of two columns equal the FP64-V-cycle ones to 1e-7 (relative 2-norm, pressure
  compared up to its constant).
* 3D Stokes, 48^3 hex mesh (2,855,668 dofs), lid-driven, one right-hand side,
  FP32 V-cycle: the same checks.

The FP64 path itself is checked against the oracle element by element at the
sizes the oracle finishes in seconds (test_gpu_parity.py).
"""
import numpy as np
import pytest

from synth import oseen_recirculating_2d, stokes_lid_3d

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1607_02489_gb300")

RTOL = 1e-8
RESTART, MAXIT = 60, 400


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    g._build.build()
    g.load()


def _relerr_up_to_pressure_constant(p, x, ref):
    nu = p.dim * p.n_v
    d = x - ref
    d[nu:] -= d[nu:].mean(axis=0)
    r = ref.copy()
    r[nu:] -= r[nu:].mean(axis=0)
    return np.linalg.norm(d, axis=0) / np.linalg.norm(r, axis=0)


def _check_full(p, nrhs, fp64_cols):
    H32 = g.Hierarchy(p, max_nrhs=nrhs, vcycle_fp32=1)
    b = torch.tensor(p.b, device="cuda")
    x = torch.zeros_like(b)
    st, its, rel = H32.fgmres(b, x, rtol=RTOL, restart=RESTART, maxit=MAXIT)
    assert st == g.AMG_OK and np.all(rel <= RTOL), (st, its, rel)
    A = p.full_matrix()
    xh = x.cpu().numpy()
    true = np.linalg.norm(p.b - A @ xh, axis=0) / np.linalg.norm(p.b, axis=0)
    assert np.all(true <= 1.01 * RTOL), true
    # the block product, against the host product on every row
    y = torch.empty_like(b)
    H32.apply(x, y)
    yh = y.cpu().numpy()
    ref = A @ xh
    assert np.all(np.linalg.norm(yh - ref, axis=0) <= 1e-13 * np.linalg.norm(ref, axis=0))
    # FP32-V-cycle solutions against the FP64-V-cycle ones
    del H32
    k = len(fp64_cols)
    H64 = g.Hierarchy(p, max_nrhs=k, vcycle_fp32=0)
    b64 = torch.tensor(np.ascontiguousarray(p.b[:, fp64_cols]), device="cuda")
    x64 = torch.zeros_like(b64)
    st64, its64, rel64 = H64.fgmres(b64, x64, rtol=RTOL, restart=RESTART, maxit=MAXIT)
    assert st64 == g.AMG_OK
    err = _relerr_up_to_pressure_constant(p, xh[:, fp64_cols], x64.cpu().numpy())
    assert np.all(err <= 1e-7), err
    assert np.all(np.abs(its[fp64_cols] - its64) <= 2), (its[fp64_cols], its64)
    return its


@pytest.mark.parametrize("Re", [1.0, 10.0, 100.0])
def test_oseen_512_thirty_two_rhs(Re):
    p = oseen_recirculating_2d(512, Re=Re, nrhs=32)
    assert p.N == 2364419
    its = _check_full(p, 32, [0, 31])
    assert its.max() <= MAXIT


def test_stokes_3d_48():
    p = stokes_lid_3d(48, nrhs=1)
    assert p.N == 2855668
    _check_full(p, 1, [0])
