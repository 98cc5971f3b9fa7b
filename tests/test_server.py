"""GPU tests of the request server (amg_server_*): continuous batching of FGMRES
solves over several resident hierarchies.

Without batching (merge_k = 1) the server runs a request with the kernels, K
and workspace of a blocking solve of the same right-hand sides, and every
reduction has a fixed order, so the tolerance for "the same alone and in the
mix" is zero: bitwise equal solutions, iteration counts and residuals.  With
batching a request's columns run inside a wider cohort, whose kernels sum in a
different order: the stated tolerance is then iterations within +-1, relative
residual <= rtol (re-checked on the host) and solutions within 1e-6 of the
solve alone; a batched run is still bitwise reproducible.
"""
import numpy as np
import pytest

from synth import oseen_recirculating_2d, stokes_lid_2d, stokes_pinned_2d

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
g = pytest.importorskip("paper_1607_02489_gb300")

RESTART, MAXIT = 60, 300


@pytest.fixture(scope="module")
def hierarchies():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    g._build.build()
    g.load()
    probs = {
        "lid32": stokes_lid_2d(32, nrhs=8, seed=3),
        "oseen32_re10": oseen_recirculating_2d(32, Re=10.0, nrhs=8),
        "oseen48_re100": oseen_recirculating_2d(48, Re=100.0, nrhs=8),
        "pinned16": stokes_pinned_2d(16, nrhs=8),
    }
    hs = {}
    for name, p in probs.items():
        hs[name] = (p, g.Hierarchy(p, max_nrhs=8, vcycle_fp32=1))
    hs["lid32_fp64"] = (probs["lid32"], g.Hierarchy(probs["lid32"], max_nrhs=8, vcycle_fp32=0))
    return hs


def _requests():
    """(hierarchy name, first column, nrhs) of a mix of shapes and sizes."""
    return [("lid32", 0, 3), ("oseen32_re10", 1, 1), ("oseen48_re100", 0, 8), ("pinned16", 2, 2),
            ("lid32_fp64", 4, 4), ("oseen32_re10", 0, 5), ("lid32", 5, 1), ("oseen48_re100", 3, 2),
            ("pinned16", 0, 8), ("lid32", 0, 3)]


def _b(p, c0, k):
    return torch.tensor(np.ascontiguousarray(p.b[:, c0:c0 + k])).pin_memory()


def _alone(hs, name, c0, k, rtol):
    p, H = hs[name]
    b = _b(p, c0, k)
    x = torch.zeros_like(b).pin_memory()
    st, its, rel = H.fgmres_host(b, x, rtol=rtol, restart=RESTART, maxit=MAXIT)
    return st, its, rel, x


def test_mix_matches_solves_alone(hierarchies):
    hs = hierarchies
    rtol = 1e-8
    reqs = _requests()
    alone = [_alone(hs, n, c0, k, rtol) for n, c0, k in reqs]
    sv = g.Server(max_active=6, restart=RESTART, maxit=MAXIT, merge_k=1)
    bufs, tickets, results = [], [], {}
    max_running = 0
    # staggered arrivals: a few requests, some progress, then the rest
    for i, (n, c0, k) in enumerate(reqs):
        b = _b(hs[n][0], c0, k)
        x = torch.full_like(b, float("nan")).pin_memory()
        bufs.append((b, x))
        tickets.append(sv.submit(hs[n][1], b, x, rtol=rtol))
        for _ in range(3 if i % 3 == 0 else 0):
            for t in sv.progress():
                results[t] = sv.result(t)
            max_running = max(max_running, sv.stats()["running"])
    while len(results) < len(reqs):
        for t in sv.progress():
            results[t] = sv.result(t)
        max_running = max(max_running, sv.stats()["running"])
    stats = sv.stats()
    assert stats["errors"] == 0 and stats["queued"] == 0 and stats["running"] == 0
    assert max_running >= 2, "requests never overlapped"
    assert stats["kernel_launches"] > 0
    for i, t in enumerate(tickets):
        st, its, rel, sec = results[t]
        st0, its0, rel0, x0 = alone[i]
        assert st == st0 == g.AMG_OK, (i, st, st0)
        assert np.array_equal(its, its0), (i, its, its0)
        assert np.array_equal(rel, rel0), (i, rel, rel0)
        assert torch.equal(bufs[i][1], x0), i
        assert np.all(rel <= rtol)
        assert 0.0 <= sec[0] <= sec[1]
    sv.close()


def test_true_residuals_of_served_solves(hierarchies):
    hs = hierarchies
    sv = g.Server(max_active=4, restart=RESTART, maxit=MAXIT)
    todo = {}
    for n, c0, k in [("oseen48_re100", 0, 4), ("lid32", 2, 2), ("pinned16", 0, 1)]:
        p = hs[n][0]
        b = _b(p, c0, k)
        x = torch.zeros_like(b).pin_memory()
        todo[sv.submit(hs[n][1], b, x, rtol=1e-8)] = (p, b, x)
    done = {}
    while len(done) < len(todo):
        for t in sv.progress():
            done[t] = sv.result(t)
    for t, (p, b, x) in todo.items():
        st, its, rel, _ = done[t]
        assert st == g.AMG_OK
        A = p.full_matrix()
        bb, xx = b.numpy(), x.numpy()
        true = np.linalg.norm(bb - A @ xx, axis=0) / np.linalg.norm(bb, axis=0)
        assert np.all(true <= 1.01e-8), true
    sv.close()


def test_admission_by_memory_runs_one_at_a_time(hierarchies):
    """A budget that holds one slot of the largest request: requests still all
    complete, the slots never hold more than the budget (so a large request never
    runs beside another), and idle slots are released to make room for other shapes."""
    hs = hierarchies
    reqs = [("oseen48_re100", 0, 8), ("lid32", 0, 2), ("oseen48_re100", 0, 8), ("pinned16", 1, 1)]
    alone = [_alone(hs, n, c0, k, 1e-8) for n, c0, k in reqs]
    probe = g.Server(max_active=1, restart=RESTART, maxit=MAXIT, merge_k=1)
    b0 = _b(hs["oseen48_re100"][0], 0, 8)
    x0 = torch.zeros_like(b0).pin_memory()
    t0 = probe.submit(hs["oseen48_re100"][1], b0, x0)
    while not probe.progress():
        pass
    one_slot = probe.stats()["bytes_in_use"]
    probe.result(t0)
    probe.close()
    sv = g.Server(max_active=4, device_bytes=one_slot, restart=RESTART, maxit=MAXIT, merge_k=1)
    bufs, tickets, res = [], [], {}
    for n, c0, k in reqs:
        b = _b(hs[n][0], c0, k)
        x = torch.zeros_like(b).pin_memory()
        bufs.append(x)
        tickets.append(sv.submit(hs[n][1], b, x))
    while len(res) < len(reqs):
        for t in sv.progress():
            res[t] = sv.result(t)
        s = sv.stats()
        assert s["bytes_in_use"] <= one_slot
        running = [i for i, t in enumerate(tickets) if t not in res and sv.state(t) == 1]
        if 0 in running or 2 in running:  # a large request never runs beside another
            assert len(running) == 1, running
    s = sv.stats()
    assert s["slots_released"] >= 2 and s["errors"] == 0
    for i, t in enumerate(tickets):
        assert res[t][0] == g.AMG_OK
        assert torch.equal(bufs[i], alone[i][3])
    sv.close()


def test_request_larger_than_budget_fails_cleanly(hierarchies):
    hs = hierarchies
    p, H = hs["lid32"]
    sv = g.Server(max_active=2, device_bytes=1 << 20, restart=RESTART, maxit=MAXIT)
    b = _b(p, 0, 2)
    x = torch.zeros_like(b).pin_memory()
    t = sv.submit(H, b, x)
    done = []
    while not done:
        done = sv.progress()
    st, its, rel, _ = sv.result(t)
    assert st == -2  # AMG_ERR_OOM
    assert sv.stats()["errors"] == 1
    sv.close()


def test_server_argument_errors(hierarchies):
    p, H = hierarchies["pinned16"]
    sv = g.Server(max_active=1, restart=RESTART, maxit=MAXIT)
    b = torch.zeros((p.N, 33), dtype=torch.float64)
    with pytest.raises(g.AmgError):
        sv.submit(H, b, torch.zeros_like(b))
    with pytest.raises(g.AmgError):
        sv.submit(H, b[:, :1].contiguous(), torch.zeros((p.N, 1), dtype=torch.float64), rtol=0.0)
    with pytest.raises(KeyError):
        sv.result(12345)
    # a zero right-hand side completes at once with x = 0
    bz = torch.zeros((p.N, 1), dtype=torch.float64).pin_memory()
    xz = torch.full_like(bz, 3.0).pin_memory()
    t = sv.submit(H, bz, xz)
    done = []
    while not done:
        done = sv.progress()
    st, its, rel, _ = sv.result(t)
    assert st == g.AMG_OK and its[0] == 0 and rel[0] == 0.0 and torch.all(xz == 0)
    sv.close()


def test_reserved_slots_are_reused(hierarchies):
    p, H = hierarchies["oseen32_re10"]
    sv = g.Server(max_active=4, restart=RESTART, maxit=MAXIT, merge_k=1)
    sv.reserve(H, 3, 2)   # K = 4
    sv.reserve(H, 4, 2)   # same shape: nothing new
    s = sv.stats()
    assert s["slots"] == 2 and s["slots_created"] == 2 and s["running"] == 0 and s["bytes_in_use"] > 0
    outs = []
    for c0 in (0, 4):
        b = _b(p, c0, 3)
        x = torch.zeros_like(b).pin_memory()
        outs.append((sv.submit(H, b, x), x, _alone(hierarchies, "oseen32_re10", c0, 3, 1e-8)[3]))
    done = 0
    while done < 2:
        done += len(sv.progress())
    assert sv.stats()["slots_created"] == 2
    for t, x, x0 in outs:
        assert sv.result(t)[0] == g.AMG_OK and torch.equal(x, x0)
    small = g.Server(max_active=1, device_bytes=1 << 20, restart=RESTART, maxit=MAXIT)
    with pytest.raises(g.AmgError):
        small.reserve(H, 1, 1)
    small.close()
    sv.close()


def _run_batch(hs, reqs, rtol, merge_k):
    sv = g.Server(max_active=4, restart=RESTART, maxit=MAXIT, merge_k=merge_k)
    xs, tickets = [], []
    for n, c0, k in reqs:       # all queued before the first progress(): cohorts form
        b = _b(hs[n][0], c0, k)
        x = torch.full_like(b, float("nan")).pin_memory()
        xs.append((b, x))
        tickets.append(sv.submit(hs[n][1], b, x, rtol=rtol))
    res = {}
    while len(res) < len(reqs):
        for t in sv.progress():
            res[t] = sv.result(t)
    st = sv.stats()
    sv.close()
    return [res[t] for t in tickets], xs, st


def test_batched_cohorts_match_solves_alone_within_tolerance(hierarchies):
    hs = hierarchies
    rtol = 1e-8
    reqs = [("lid32", 0, 3), ("oseen32_re10", 1, 1), ("lid32", 3, 2), ("oseen32_re10", 0, 5), ("lid32", 5, 1),
            ("pinned16", 0, 2), ("oseen32_re10", 6, 2), ("pinned16", 2, 6), ("lid32", 6, 2)]
    alone = [_alone(hs, n, c0, k, rtol) for n, c0, k in reqs]
    res, xs, st = _run_batch(hs, reqs, rtol, merge_k=8)
    assert st["errors"] == 0
    assert st["cohorts"] < len(reqs), "no requests were batched"
    for i, (n, c0, k) in enumerate(reqs):
        status, its, rel, _ = res[i]
        st0, its0, rel0, x0 = alone[i]
        assert status == g.AMG_OK and np.all(rel <= rtol), (i, status, rel)
        assert np.all(np.abs(its - its0) <= 1), (i, its, its0)
        p = hs[n][0]
        b, x = xs[i]
        bb, xx = b.numpy(), x.numpy()
        true = np.linalg.norm(bb - p.full_matrix() @ xx, axis=0) / np.linalg.norm(bb, axis=0)
        assert np.all(true <= 1.01 * rtol), (i, true)
        nu = p.dim * p.n_v
        d = xx - x0.numpy()
        ref = x0.numpy().copy()
        if p.pinned < 0:
            d[nu:] -= d[nu:].mean(axis=0)
            ref[nu:] -= ref[nu:].mean(axis=0)
        err = np.linalg.norm(d, axis=0) / np.linalg.norm(ref, axis=0)
        assert np.all(err <= 1e-6), (i, err)
    # the same batched run again: bitwise the same
    res2, xs2, _ = _run_batch(hs, reqs, rtol, merge_k=8)
    for i in range(len(reqs)):
        assert np.array_equal(res[i][1], res2[i][1]) and torch.equal(xs[i][1], xs2[i][1])


def test_smallest_work_first_admits_the_small_request_first(hierarchies):
    """With policy 1 and one slot, a small request queued behind a large one starts first."""
    hs = hierarchies
    sv = g.Server(max_active=1, restart=RESTART, maxit=MAXIT, merge_k=1, policy=1)
    order = []
    big_b = _b(hs["oseen48_re100"][0], 0, 8)
    small_b = _b(hs["pinned16"][0], 0, 1)
    big = sv.submit(hs["oseen48_re100"][1], big_b, torch.zeros_like(big_b).pin_memory())
    small = sv.submit(hs["pinned16"][1], small_b, torch.zeros_like(small_b).pin_memory())
    while len(order) < 2:
        for t in sv.progress():
            order.append(t)
            assert sv.result(t)[0] == g.AMG_OK
    assert order == [small, big]
    sv.close()
