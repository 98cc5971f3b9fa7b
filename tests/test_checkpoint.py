"""Hierarchy checkpoints (amg_hierarchy_export / amg_hierarchy_import) on the host.

Round trip: a hierarchy written and read back has the same operators,
transfers, coarse points, smoother data and coarsest inverse (bit for bit:
import forms the smoother data with the same host code).  Oracle import: the
oracle's hierarchy written in the file format (tests/hierarchy_file.py) and
imported gives the oracle's Schur complements, Gauss-Seidel order and
coarsest inverse.  Malformed files are refused with AMG_ERR_ARG."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from synth import stokes_lid_2d, stokes_pinned_2d, oseen_recirculating_2d
from oracle import setup_hierarchy

g = pytest.importorskip("paper_1607_02489_gb300")
from hierarchy_file import write_oracle_hierarchy  # noqa: E402

MATS = ["A", "B", "Bt", "S", "P", "Pp", "R", "Rp"]


@pytest.fixture(scope="module", autouse=True)
def built():
    g._build.build()
    g.load()


def _csr(t):
    rp, col, val, shape = t
    return sp.csr_matrix((val, col, rp), shape=shape)


CASES = {
    "lid32": lambda: stokes_lid_2d(32, nrhs=1),
    "pinned16": lambda: stokes_pinned_2d(16),
    "oseen32": lambda: oseen_recirculating_2d(32, Re=10.0, nrhs=1),
}


@pytest.mark.parametrize("case", list(CASES))
def test_export_import_round_trip_is_exact(case, tmp_path):
    p = CASES[case]()
    H = g.Hierarchy(p, host_only=1)
    path = str(tmp_path / "h.bin")
    H.export(path)
    H2 = g.Hierarchy.from_file(path, host_only=1)
    assert H2.num_levels() == H.num_levels()
    for l in range(H.num_levels()):
        assert H2.level_info(l) == H.level_info(l)
        last = l + 1 == H.num_levels()
        for nm in MATS[:4] + ([] if last else MATS[4:]):
            a, b = H.level_matrix(l, nm), H2.level_matrix(l, nm)
            assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3])), (l, nm)
        pa, pb = H.level_points(l), H2.level_points(l)
        for k in pa:
            assert np.array_equal(pa[k], pb[k]), (l, k)
    assert np.array_equal(H.coarse_inverse(), H2.coarse_inverse())


@pytest.mark.parametrize("case", list(CASES))
def test_imported_oracle_hierarchy_has_the_oracles_smoother_data(case, tmp_path):
    p = CASES[case]()
    Ho = setup_hierarchy(p)
    path = str(tmp_path / "oracle.bin")
    write_oracle_hierarchy(Ho, path)
    H = g.Hierarchy.from_file(path, host_only=1)
    assert H.num_levels() == len(Ho.levels)
    for l, L in enumerate(Ho.levels):
        info, pts = H.level_info(l), H.level_points(l)
        assert (info["n_v"], info["n_p"], info["pinned"]) == (L.n_v, L.n_p, L.pinned)
        assert info["gs_strip"] == L.gs_strip
        assert np.array_equal(pts["colors"], L.colors)
        assert np.abs(pts["D"] - L.D).max() <= 1e-13 * np.abs(L.D).max()
        S = _csr(H.level_matrix(l, "S"))
        assert np.array_equal(S.indptr, L.S.indptr) and np.array_equal(S.indices, L.S.indices)
        assert abs(S - L.S).max() <= 1e-12 * max(abs(L.S).max(), abs(Ho.levels[0].S).max())
        # the operators and transfers are the file's, unchanged
        for nm in ("A", "B", "Bt") + (() if l + 1 == len(Ho.levels) else ("P", "Pp", "R", "Rp")):
            M = _csr(H.level_matrix(l, nm))
            O = sp.csr_matrix(getattr(L, nm))
            assert abs(M - O).max() == 0.0, (l, nm)
    X, Xo = H.coarse_inverse(), Ho.levels[-1].coarse_pinv
    assert np.linalg.norm(X - Xo) <= 1e-11 * np.linalg.norm(Xo)


def test_reuse_from_an_imported_hierarchy(tmp_path):
    """An imported hierarchy carries coarse points and patterns, so it can seed
    amg_hierarchy_create_reuse; on its own matrix that reproduces the original."""
    p = oseen_recirculating_2d(16, Re=10.0, nrhs=1)
    H = g.Hierarchy(p, host_only=1)
    path = str(tmp_path / "h.bin")
    H.export(path)
    Hi = g.Hierarchy.from_file(path, host_only=1)
    Hr = g.Hierarchy(p, host_only=1, reuse=Hi)
    for l in range(H.num_levels() - 1):
        for nm in ("P", "Pp", "R", "Rp"):
            a, b = H.level_matrix(l, nm), Hr.level_matrix(l, nm)
            assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3])), (l, nm)


def test_malformed_files_are_refused(tmp_path):
    p = stokes_lid_2d(8, nrhs=1)
    H = g.Hierarchy(p, host_only=1)
    path = str(tmp_path / "h.bin")
    H.export(path)
    data = open(path, "rb").read()
    bad = {
        "magic": b"XXXXXXXX" + data[8:],
        "truncated": data[: len(data) // 2],
        "version": data[:8] + np.array([7], dtype="<i4").tobytes() + data[12:],
    }
    # a column index of A out of range: A's first column entry sits after the level
    # header (4 ints), A's shape (2 ints), nnz (1 int64) and n_v + 1 row pointers
    n_v = H.level_info(0)["n_v"]
    off = 8 + 12 + 16 + 8 + 8 + 8 * (n_v + 1)
    bad["column"] = data[:off] + np.array([n_v + 5], dtype="<i4").tobytes() + data[off + 4:]
    for name, blob in bad.items():
        q = str(tmp_path / f"{name}.bin")
        open(q, "wb").write(blob)
        with pytest.raises(g.AmgError) as e:
            g.Hierarchy.from_file(q, host_only=1)
        assert e.value.status == -1, name
    with pytest.raises(g.AmgError):
        g.Hierarchy.from_file(str(tmp_path / "missing.bin"), host_only=1)
    with pytest.raises(g.AmgError):
        H.export(str(tmp_path / "no_such_dir" / "h.bin"))
