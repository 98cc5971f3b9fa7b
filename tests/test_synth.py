"""Pins for the synthetic Q2-Q1 problem generator (Section 2) and the splitmix64 draws."""
import os

import numpy as np
import pytest

from synth import make_problem, splitmix64, uniform_pm1, element_matrices, recirculating_wind
from synth.q2q1 import assemble

HERE = os.path.dirname(os.path.abspath(__file__))


def test_splitmix64_published_outputs():
    # first outputs of splitmix64 started from state 0 (Vigna's public-domain reference)
    z = splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # counter-based: a window equals the tail of a longer stream
    assert np.array_equal(splitmix64(7, 5, start=3), splitmix64(7, 8)[3:])


def test_uniform_range_and_moments():
    u = uniform_pm1(1, 200000)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1.0 / 3.0) < 0.01


def test_dof_counts_match_table1():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "table1_bs22.txt")) if l[0] != "#"]
    for r in rows:
        n, dofs = int(r[0]), int(r[1])
        assert 2 * (2 * n + 1) ** 2 + (n + 1) ** 2 == dofs
    p = make_problem(8, 2, -1.0, 1.0, bc="lid")
    assert p.N == 659


@pytest.mark.parametrize("h", [1.0, 0.3, 1.0 / 64])
def test_q2_element_stiffness_closed_form(h):
    K1 = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / (3 * h)
    M1 = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) * h / 30
    Ae, Be = element_matrices(2, h)
    assert np.allclose(Ae, np.kron(M1, K1) + np.kron(K1, M1), rtol=0, atol=1e-14 * np.abs(Ae).max())
    Ae3, _ = element_matrices(3, h)
    ref3 = np.kron(M1, np.kron(M1, K1)) + np.kron(M1, np.kron(K1, M1)) + np.kron(K1, np.kron(M1, M1))
    assert np.allclose(Ae3, ref3, rtol=0, atol=1e-13 * np.abs(ref3).max())


def test_divergence_sign_and_scale():
    """B u_h = -int psi_k div(u) for u = (x, 0): minus the pressure-node areas."""
    n = 8
    A, B, vX, pX, p2v, bnd, top = assemble(n, 2, 0.0, 1.0)
    h = 1.0 / n
    u = np.concatenate([vX[:, 0], np.zeros(len(vX))])
    area = np.full(len(pX), h * h)
    edge_x = (np.isclose(pX[:, 0], 0) | np.isclose(pX[:, 0], 1))
    edge_y = (np.isclose(pX[:, 1], 0) | np.isclose(pX[:, 1], 1))
    area[edge_x] /= 2
    area[edge_y] /= 2
    assert np.allclose(B @ u, -area, atol=1e-14)


def test_divergence_free_quadratic_field():
    """u = (x^2, -2xy) lies in Q2 and is divergence free, so B u_h = 0 on every row."""
    A, B, vX, pX, *_ = assemble(6, 2, -1.0, 1.0)
    u = np.concatenate([vX[:, 0] ** 2, -2 * vX[:, 0] * vX[:, 1]])
    assert np.abs(B @ u).max() < 1e-14


def test_stiffness_on_polynomials():
    """Interior rows: A_hat (linear) = 0 and A_hat (x^2+y^2) = -4 int phi_i."""
    n = 6
    A, B, vX, pX, p2v, bnd, top = assemble(n, 2, 0.0, 1.0)
    h = 1.0 / n
    inner = ~bnd
    lin = 3.0 * vX[:, 0] - 2.0 * vX[:, 1] + 0.5
    assert np.abs((A @ lin)[inner]).max() < 1e-13
    q = vX[:, 0] ** 2 + vX[:, 1] ** 2
    idx = np.arange(len(vX))
    ix, iy = idx % (2 * n + 1), idx // (2 * n + 1)
    w1 = lambda i: np.where(i % 2 == 0, h / 3, 2 * h / 3)  # noqa: E731
    assert np.allclose((A @ q)[inner], (-4 * w1(ix) * w1(iy))[inner], atol=1e-14)


def test_convection_skew_and_constant_kernel():
    """K_hat 1 = 0, and K_hat + K_hat^T = 0 for the divergence-free tangential wind."""
    A0, *_ = assemble(8, 2, -1.0, 1.0, nu=1.0)
    A1, *_ = assemble(8, 2, -1.0, 1.0, nu=1.0, wind=recirculating_wind)
    K = (A1 - A0).tocsr()
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-13
    assert abs(K + K.T).max() < 1e-13
    assert abs(K).max() > 1e-2


def test_boundary_conditions_and_colocation():
    p = make_problem(4, 2, 0.0, 1.0, bc="lid", nrhs=2, seed=3)
    assert np.array_equal(p.vcoords[p.p2v], p.pcoords)
    D = np.flatnonzero(p.v_dirichlet)
    Ad = p.A.toarray()
    assert np.array_equal(Ad[D][:, D], np.eye(len(D)))
    assert np.abs(Ad[D][:, ~p.v_dirichlet]).max() == 0
    assert np.abs(p.B.toarray()[:, np.concatenate([D, D + p.n_v])]).max() == 0
    top = np.isclose(p.vcoords[:, 1], 1.0)
    assert np.all(p.b[D[top[D]], :] == 1.0) and np.all(p.b[p.n_v + D, :] == 0.0)
    # the two right-hand sides differ only by their seeded body loads
    assert not np.allclose(p.b[:, 0], p.b[:, 1])
    assert abs(p.b[2 * p.n_v:].sum(axis=0)).max() < 1e-14


def test_serving_stream_is_a_seeded_poisson_mix():
    """Exponential gaps with the stated mean rate, every (n, Re, nrhs) choice from its set
    with roughly uniform frequencies, and the same stream for the same seed."""
    from synth import serving_stream, MESHES, REYNOLDS
    s = serving_stream(4000, rate=200.0, seed=0)
    assert s == serving_stream(4000, rate=200.0, seed=0)
    t = np.array([r["t"] for r in s])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 200.0) < 0.05 / 200.0        # 4000 draws: sd of the mean ~1.6%
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.06       # exponential: cv = 1
    for key, choices in (("n", MESHES), ("Re", REYNOLDS), ("nrhs", range(1, 9))):
        vals = [r[key] for r in s]
        assert set(vals) == set(choices)
        counts = np.array([vals.count(c) for c in choices])
        assert counts.min() > 0.8 * len(s) / len(choices)


def test_homogeneous_rhs_equals_make_problem_draws():
    from synth import homogeneous_rhs, oseen_recirculating_2d
    p = oseen_recirculating_2d(12, Re=100.0, nrhs=4, seed=9)
    assert np.array_equal(homogeneous_rhs(p, 4, 9), p.b)
