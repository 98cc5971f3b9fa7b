"""amg_apply_noalloc against amg_apply (GPU).

amg_apply_noalloc serves callers that cannot allocate device memory during a call
(a memory budget owned by another allocator, or a loop that cannot take the
device synchronisation of cudaMalloc/cudaFree).  Its scratch is a static array
in the library; this checks that two calls in a row give amg_apply's result, and
that sizes beyond the array are refused.  Collected last on purpose.
"""
import numpy as np
import pytest

from synth import stokes_lid_2d, uniform_pm1

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1607_02489_gb300")


def test_apply_noalloc_matches_apply_on_two_calls_in_a_row():
    assert torch.cuda.is_available(), "needs a CUDA device"
    g._build.build()
    p = stokes_lid_2d(32, nrhs=3)
    H = g.Hierarchy(p, max_nrhs=4)
    for seed in (31, 32):
        x = torch.tensor(uniform_pm1(seed, p.N * 3).reshape(p.N, 3), device="cuda")
        y_ref = torch.empty_like(x)
        y = torch.full_like(x, float("nan"))
        H.apply(x, y_ref)
        H.apply_noalloc(x, y)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(y - y_ref, dim=0) / torch.linalg.norm(y_ref, dim=0)).cpu().numpy()
        assert np.all(err <= 1e-13), err


def test_apply_noalloc_refuses_sizes_beyond_its_scratch():
    g._build.build()
    p = stokes_lid_2d(128, nrhs=1)   # N = 148,739; with 8 columns N * K > 1,048,576
    H = g.Hierarchy(p, max_nrhs=8)
    x = torch.zeros((p.N, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(g.AmgError) as e:
        H.apply_noalloc(x, torch.empty_like(x))
    assert e.value.status == -1 and "exceeds the static scratch" in str(e.value)
