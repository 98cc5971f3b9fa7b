"""Writer of the hierarchy checkpoint format (include/emin_amg.h, amg_hierarchy_export)
for an oracle hierarchy, so the library can import the oracle's operators and
transfers and its V-cycle can be compared with the oracle's independently of
the setup.  Test infrastructure: numpy only, written from the format's
description, sharing no code with the library's reader."""
import numpy as np
import scipy.sparse as sp


def _csr(f, M):
    M = sp.csr_matrix(M)
    M.sort_indices()
    f.write(np.array([M.shape[0], M.shape[1]], dtype="<i4").tobytes())
    f.write(np.array([M.nnz], dtype="<i8").tobytes())
    f.write(np.asarray(M.indptr, dtype="<i8").tobytes())
    f.write(np.asarray(M.indices, dtype="<i4").tobytes())
    f.write(np.asarray(M.data, dtype="<f8").tobytes())


def write_oracle_hierarchy(H, path):
    """H: oracle.Hierarchy built without coarsening reuse (its levels carry Cp and Cv)."""
    with open(path, "wb") as f:
        f.write(b"EMINAMG1")
        f.write(np.array([1, len(H.levels), 1 if H.symmetric else 0], dtype="<i4").tobytes())
        for l, L in enumerate(H.levels):
            f.write(np.array([L.dim, L.n_v, L.n_p, L.pinned], dtype="<i4").tobytes())
            for M in (L.A, L.B, L.Bt):
                _csr(f, M)
            f.write(np.ascontiguousarray(L.vcoords, dtype="<f8").tobytes())
            f.write(np.ascontiguousarray(L.pcoords, dtype="<f8").tobytes())
            f.write(np.asarray(L.p2v, dtype="<i4").tobytes())
            f.write(np.asarray(L.dirichlet, dtype=np.uint8).tobytes())
            if l + 1 < len(H.levels):
                for M in (L.P, L.Pp, L.R, L.Rp):
                    _csr(f, M)
                for pts in (L.info["Cp"], L.info["Cv"]):
                    f.write(np.array([len(pts)], dtype="<i4").tobytes())
                    f.write(np.asarray(pts, dtype="<i4").tobytes())
