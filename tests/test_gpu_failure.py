"""Failure path of the bounded device waits, run to its error status on a GPU.

The pipelined Gauss-Seidel kernel waits on neighbouring strips and the ILU(1)
substitutions wait on earlier rows; every such wait gives up after a poll
limit, sets the cycle's error word and returns, so the kernel always ends
and the solve reports AMG_ERR_CUDA.  amg_set_wait_limit lowers the limit to
one poll, which makes waits run out (a neighbour is still working when the
first poll finds its counter short), and then restores the default: the next
solve on the same hierarchy is correct and equal to a fresh hierarchy's.
Nothing here faults or hangs the GPU: the waits end by their own limit.
"""
import numpy as np
import pytest

from synth import stokes_lid_2d

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1607_02489_gb300")


@pytest.fixture(scope="module", autouse=True)
def gpu_and_lib():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    g._build.build()
    g.load()


def _solve(H, b):
    x = torch.zeros_like(b)
    st, its, rel = H.fgmres(b, x, rtol=1e-8)
    return st, its, rel, x


@pytest.mark.parametrize("kind", ["gauss_seidel_strips", "ilu_substitution"])
def test_a_wait_that_runs_out_returns_the_cuda_error_status(kind):
    # autotune = 0: the 128x128 finest level (65 strips of two grid lines) keeps the
    # pipelined strip kernel, whose odd strips wait on their even neighbours
    kw = dict(autotune=0) if kind == "gauss_seidel_strips" else dict(smoother=2, pre=1, post=1)
    p = stokes_lid_2d(128 if kind == "gauss_seidel_strips" else 32, nrhs=1)
    H = g.Hierarchy(p, max_nrhs=1, **kw)
    b = torch.tensor(p.b, device="cuda")
    H.set_wait_limit(1)
    with pytest.raises(g.AmgError) as exc:
        _solve(H, b)
    assert exc.value.status == -3 and "timed out" in str(exc.value)
    H.set_wait_limit(0)  # the default limit again
    st, its, rel, x = _solve(H, b)
    assert st == g.AMG_OK and np.all(rel <= 1e-8)
    H2 = g.Hierarchy(p, max_nrhs=1, **kw)
    st2, its2, rel2, x2 = _solve(H2, b)
    assert np.array_equal(its, its2)
    if kind == "gauss_seidel_strips":  # fixed kernel choices: the same bits
        assert torch.equal(x, x2)
    else:
        assert ((x - x2).norm() / x2.norm()).item() <= 1e-12


def test_a_device_allocation_failure_returns_oom_and_the_handle_stays_usable():
    """A Krylov workspace far beyond the device's memory (restart 10^8: basis vectors of
    2,467 x 2 doubles, about 4 TB) makes its first cudaMalloc fail; the solve returns
    AMG_ERR_OOM before any launch, and the same hierarchy then solves normally."""
    p = stokes_lid_2d(16, nrhs=2)
    H = g.Hierarchy(p, max_nrhs=2)
    b = torch.tensor(p.b, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(g.AmgError) as exc:
        H.fgmres(b, x, rtol=1e-8, restart=100_000_000, maxit=10)
    assert exc.value.status == -2 and "cudaMalloc" in str(exc.value)
    st, its, rel = H.fgmres(b, x, rtol=1e-8)
    assert st == g.AMG_OK and np.all(rel <= 1e-8)
