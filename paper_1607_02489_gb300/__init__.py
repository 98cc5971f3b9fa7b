"""Python binding of libemin_amg.so (include/emin_amg.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module only
converts arrays and tensors to the C ABI's pointers and sizes.  There is no
fallback: if the library is missing or no GPU is present, the calls raise.

Vectors are torch CUDA tensors of shape (N,) or (N, nrhs), float64,
contiguous, dofs ordered [u_x | u_y (| u_z) | p].
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

LIB_PATH = _build.LIB

AMG_OK, AMG_NOT_CONVERGED, AMG_BREAKDOWN = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", 2: "BREAKDOWN", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA",
                -4: "ERR_SETUP"}
EXPORTED = ["amg_params_default", "amg_hierarchy_create", "amg_hierarchy_create_reuse", "amg_hierarchy_export",
            "amg_hierarchy_import", "amg_vcycle_apply", "amg_apply", "amg_fgmres_solve",
            "amg_fgmres_solve_host", "amg_num_levels", "amg_level_get_info", "amg_level_get_matrix",
            "amg_level_get_points", "amg_hierarchy_destroy", "amg_last_error", "amg_profile_vcycle", "amg_kernel_launches", "amg_apply_noalloc", "amg_gs_variant", "amg_set_gs_variant", "amg_row_shape", "amg_profile_arnoldi", "amg_level_get_vanka", "amg_level_get_ilu",
            "amg_coarse_inverse", "amg_set_wait_limit", "amg_level_get_gs_map",
            "amg_server_params_default", "amg_server_create", "amg_server_reserve", "amg_server_submit", "amg_server_progress",
            "amg_server_result", "amg_server_state", "amg_server_get_stats", "amg_server_destroy", "amg_server_last_error"]
KERNEL_CLASSES = ["velocity", "schur_rhs", "gs_color", "update", "residual", "restrict", "prolong", "coarse", "vanka",
                  "ilu"]
MATRICES = {"A": 0, "B": 1, "Bt": 2, "S": 3, "P": 4, "Pp": 5, "R": 6, "Rp": 7}

_i32p = ctypes.POINTER(ctypes.c_int)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_ubyte)
_i64p = ctypes.POINTER(ctypes.c_longlong)


class AmgProblem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_vnodes", ctypes.c_int), ("n_pnodes", ctypes.c_int),
                ("A_rowptr", _i32p), ("A_col", _i32p), ("A_val", _f64p),
                ("B_rowptr", _i32p), ("B_col", _i32p), ("B_val", _f64p),
                ("vcoords", _f64p), ("pcoords", _f64p), ("p2v", _i32p), ("v_dirichlet", _u8p),
                ("pinned_p", ctypes.c_int), ("symmetric", ctypes.c_int)]


class AmgParams(ctypes.Structure):
    _fields_ = [("tau1", ctypes.c_double), ("tau2sq", ctypes.c_double), ("omega", ctypes.c_double),
                ("omega_on_D", ctypes.c_int), ("gs_iters", ctypes.c_int), ("pre", ctypes.c_int),
                ("post", ctypes.c_int), ("max_coarse", ctypes.c_int), ("max_levels", ctypes.c_int),
                ("vcycle_fp32", ctypes.c_int), ("max_nrhs", ctypes.c_int), ("host_only", ctypes.c_int),
                ("autotune", ctypes.c_int), ("smoother", ctypes.c_int), ("vanka_omega", ctypes.c_double),
                ("ilu_order", ctypes.c_int), ("coarse", ctypes.c_int), ("device_setup", ctypes.c_int),
                ("vanka_max_mib", ctypes.c_double)]


class AmgLevelInfo(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_v", ctypes.c_int), ("n_p", ctypes.c_int), ("pinned", ctypes.c_int),
                ("nnz_A", ctypes.c_longlong), ("nnz_B", ctypes.c_longlong), ("nnz_Bt", ctypes.c_longlong),
                ("nnz_S", ctypes.c_longlong), ("n_colors", ctypes.c_int),
                ("nnz_P", ctypes.c_longlong), ("nnz_Pp", ctypes.c_longlong), ("nnz_R", ctypes.c_longlong),
                ("nnz_Rp", ctypes.c_longlong), ("n_cp", ctypes.c_int), ("n_cv", ctypes.c_int),
                ("gs_strip", ctypes.c_int)]


class AmgServerParams(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int), ("device_bytes", ctypes.c_size_t), ("restart", ctypes.c_int),
                ("maxit", ctypes.c_int), ("merge_k", ctypes.c_int), ("policy", ctypes.c_int)]


class AmgServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int), ("running", ctypes.c_int), ("slots", ctypes.c_int),
                ("busy_slots", ctypes.c_int), ("bytes_in_use", ctypes.c_size_t), ("budget", ctypes.c_size_t),
                ("kernel_launches", ctypes.c_longlong), ("slots_created", ctypes.c_longlong),
                ("slots_released", ctypes.c_longlong), ("errors", ctypes.c_longlong), ("cohorts", ctypes.c_longlong)]


_lib = None


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libemin_amg.so (raise if it is absent; build it first on request)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() or "
                              "python -m paper_1607_02489_gb300._build")
        _build.build()
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    lib.amg_params_default.argtypes = [ctypes.POINTER(AmgParams)]
    lib.amg_params_default.restype = None
    lib.amg_hierarchy_create.argtypes = [ctypes.POINTER(AmgProblem), ctypes.POINTER(AmgParams), vp,
                                         ctypes.POINTER(vp)]
    lib.amg_hierarchy_create.restype = ctypes.c_int
    lib.amg_hierarchy_create_reuse.argtypes = [vp, ctypes.POINTER(AmgProblem), ctypes.POINTER(AmgParams), vp,
                                               ctypes.POINTER(vp)]
    lib.amg_hierarchy_create_reuse.restype = ctypes.c_int
    lib.amg_hierarchy_export.argtypes = [vp, ctypes.c_char_p]
    lib.amg_hierarchy_export.restype = ctypes.c_int
    lib.amg_hierarchy_import.argtypes = [ctypes.c_char_p, ctypes.POINTER(AmgParams), vp, ctypes.POINTER(vp)]
    lib.amg_hierarchy_import.restype = ctypes.c_int
    lib.amg_vcycle_apply.argtypes = [vp, vp, vp, ctypes.c_int, vp]
    lib.amg_vcycle_apply.restype = ctypes.c_int
    lib.amg_apply.argtypes = [vp, vp, vp, ctypes.c_int, vp]
    lib.amg_apply.restype = ctypes.c_int
    lib.amg_apply_noalloc.argtypes = [vp, vp, vp, ctypes.c_int, vp]
    lib.amg_apply_noalloc.restype = ctypes.c_int
    for name in ("amg_fgmres_solve", "amg_fgmres_solve_host"):
        f = getattr(lib, name)
        f.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, _i32p, _f64p, vp]
        f.restype = ctypes.c_int
    lib.amg_profile_vcycle.argtypes = [vp, ctypes.c_int, ctypes.c_int, _f64p, _i64p, vp]
    lib.amg_profile_vcycle.restype = ctypes.c_int
    lib.amg_profile_arnoldi.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p, _f64p, vp]
    lib.amg_profile_arnoldi.restype = ctypes.c_int
    lib.amg_gs_variant.argtypes = [vp, ctypes.c_int, ctypes.c_int, _i32p, ctypes.POINTER(ctypes.c_float)]
    lib.amg_gs_variant.restype = ctypes.c_int
    lib.amg_set_gs_variant.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.amg_set_gs_variant.restype = ctypes.c_int
    lib.amg_row_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.amg_row_shape.restype = ctypes.c_int
    lib.amg_kernel_launches.argtypes = [vp]
    lib.amg_kernel_launches.restype = ctypes.c_longlong
    lib.amg_num_levels.argtypes = [vp]
    lib.amg_num_levels.restype = ctypes.c_int
    lib.amg_level_get_info.argtypes = [vp, ctypes.c_int, ctypes.POINTER(AmgLevelInfo)]
    lib.amg_level_get_info.restype = ctypes.c_int
    lib.amg_level_get_matrix.argtypes = [vp, ctypes.c_int, ctypes.c_int, _i64p, _i32p, _f64p]
    lib.amg_level_get_matrix.restype = ctypes.c_int
    lib.amg_level_get_points.argtypes = [vp, ctypes.c_int, _i32p, _i32p, _i32p, _f64p]
    lib.amg_level_get_points.restype = ctypes.c_int
    lib.amg_level_get_vanka.argtypes = [vp, ctypes.c_int, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p]
    lib.amg_level_get_vanka.restype = ctypes.c_int
    lib.amg_level_get_ilu.argtypes = [vp, ctypes.c_int, _i32p, _i64p, _i64p, _i32p, _i32p, _i32p, _i32p, _i32p, _f64p,
                                      _i32p, _i32p, _f64p, _f64p]
    lib.amg_level_get_ilu.restype = ctypes.c_int
    lib.amg_level_get_gs_map.argtypes = [vp, ctypes.c_int, _i32p, _f64p]
    lib.amg_level_get_gs_map.restype = ctypes.c_int
    lib.amg_coarse_inverse.argtypes = [vp, _i32p, _f64p]
    lib.amg_coarse_inverse.restype = ctypes.c_int
    lib.amg_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    lib.amg_set_wait_limit.restype = ctypes.c_int
    lib.amg_hierarchy_destroy.argtypes = [vp]
    lib.amg_hierarchy_destroy.restype = None
    lib.amg_last_error.argtypes = []
    lib.amg_last_error.restype = ctypes.c_char_p
    lib.amg_server_params_default.argtypes = [ctypes.POINTER(AmgServerParams)]
    lib.amg_server_params_default.restype = None
    lib.amg_server_create.argtypes = [ctypes.POINTER(AmgServerParams), ctypes.POINTER(vp)]
    lib.amg_server_create.restype = ctypes.c_int
    lib.amg_server_submit.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_double, _i64p]
    lib.amg_server_submit.restype = ctypes.c_int
    lib.amg_server_reserve.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
    lib.amg_server_reserve.restype = ctypes.c_int
    lib.amg_server_progress.argtypes = [vp, _i64p, ctypes.c_int, _i32p]
    lib.amg_server_progress.restype = ctypes.c_int
    lib.amg_server_result.argtypes = [vp, ctypes.c_longlong, _i32p, _i32p, _f64p, _f64p, _i32p]
    lib.amg_server_result.restype = ctypes.c_int
    lib.amg_server_state.argtypes = [vp, ctypes.c_longlong, _i32p]
    lib.amg_server_state.restype = ctypes.c_int
    lib.amg_server_get_stats.argtypes = [vp, ctypes.POINTER(AmgServerStats)]
    lib.amg_server_get_stats.restype = ctypes.c_int
    lib.amg_server_destroy.argtypes = [vp]
    lib.amg_server_destroy.restype = None
    lib.amg_server_last_error.argtypes = [vp]
    lib.amg_server_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


class AmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status):
    if status < 0:
        raise AmgError(status, load().amg_last_error().decode())
    return status


def default_params(**kw) -> AmgParams:
    prm = AmgParams()
    load().amg_params_default(ctypes.byref(prm))
    for k, v in kw.items():
        if not hasattr(prm, k):
            raise KeyError(k)
        setattr(prm, k, v)
    return prm


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_ptr(t, what):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{what} must be a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Hierarchy:
    """amg_hierarchy_create over a problem with the fields of synth.Problem
    (A, B as scipy CSR, vcoords, pcoords, p2v, v_dirichlet, pinned, symmetric, dim)."""

    def __init__(self, prob, stream=None, reuse: "Hierarchy" = None, **params):
        lib = load()
        self.dim = int(prob.dim)
        self.n_v, self.n_p = int(prob.n_v), int(prob.n_p)
        self.N = self.dim * self.n_v + self.n_p
        A, B = prob.A, prob.B
        keep = dict(
            Ar=np.ascontiguousarray(A.indptr, dtype=np.int32), Ac=np.ascontiguousarray(A.indices, dtype=np.int32),
            Av=np.ascontiguousarray(A.data, dtype=np.float64),
            Br=np.ascontiguousarray(B.indptr, dtype=np.int32), Bc=np.ascontiguousarray(B.indices, dtype=np.int32),
            Bv=np.ascontiguousarray(B.data, dtype=np.float64),
            vX=np.ascontiguousarray(prob.vcoords, dtype=np.float64),
            pX=np.ascontiguousarray(prob.pcoords, dtype=np.float64),
            p2v=np.ascontiguousarray(prob.p2v, dtype=np.int32),
            dir=np.ascontiguousarray(prob.v_dirichlet, dtype=np.uint8))
        pb = AmgProblem(self.dim, self.n_v, self.n_p,
                        _ptr(keep["Ar"], ctypes.c_int), _ptr(keep["Ac"], ctypes.c_int), _ptr(keep["Av"], ctypes.c_double),
                        _ptr(keep["Br"], ctypes.c_int), _ptr(keep["Bc"], ctypes.c_int), _ptr(keep["Bv"], ctypes.c_double),
                        _ptr(keep["vX"], ctypes.c_double), _ptr(keep["pX"], ctypes.c_double),
                        _ptr(keep["p2v"], ctypes.c_int), _ptr(keep["dir"], ctypes.c_ubyte),
                        int(prob.pinned), 1 if prob.symmetric else 0)
        self.params = default_params(**params)
        handle = ctypes.c_void_p()
        sptr = ctypes.c_void_p(0) if self.params.host_only else _stream_ptr(stream)
        if reuse is not None:
            # coarsening and patterns of `reuse` (same structure), EMIN / RAP / smoother redone
            _check(lib.amg_hierarchy_create_reuse(reuse._h, ctypes.byref(pb), ctypes.byref(self.params), sptr,
                                                  ctypes.byref(handle)))
        else:
            _check(lib.amg_hierarchy_create(ctypes.byref(pb), ctypes.byref(self.params), sptr,
                                            ctypes.byref(handle)))
        self._h = handle

    @classmethod
    def from_file(cls, path, stream=None, **params) -> "Hierarchy":
        """amg_hierarchy_import: a hierarchy from a checkpoint file (operators and transfers
        of every level; the smoother data and the coarsest solve are formed)."""
        lib = load()
        self = cls.__new__(cls)
        self.params = default_params(**params)
        handle = ctypes.c_void_p()
        sptr = ctypes.c_void_p(0) if self.params.host_only else _stream_ptr(stream)
        _check(lib.amg_hierarchy_import(os.fsencode(path), ctypes.byref(self.params), sptr, ctypes.byref(handle)))
        self._h = handle
        info = self.level_info(0)
        self.dim, self.n_v, self.n_p = info["dim"], info["n_v"], info["n_p"]
        self.N = self.dim * self.n_v + self.n_p
        return self

    def export(self, path):
        """amg_hierarchy_export: write the hierarchy's checkpoint file."""
        _check(load().amg_hierarchy_export(self._h, os.fsencode(path)))

    def close(self):
        if getattr(self, "_h", None):
            load().amg_hierarchy_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _nrhs(t):
        return 1 if t.dim() == 1 else int(t.shape[1])

    def vcycle(self, r, z, stream=None):
        """z = M^-1 r (amg_vcycle_apply)."""
        _check(load().amg_vcycle_apply(self._h, _dev_ptr(r, "r"), _dev_ptr(z, "z"), self._nrhs(r), _stream_ptr(stream)))
        return z

    def apply(self, x, y, stream=None):
        """y = A x on the finest level (amg_apply)."""
        _check(load().amg_apply(self._h, _dev_ptr(x, "x"), _dev_ptr(y, "y"), self._nrhs(x), _stream_ptr(stream)))
        return y

    def apply_noalloc(self, x, y, stream=None):
        """y = A x through amg_apply_noalloc: no device allocation in the call; its
        scratch is the library's static 16 MiB array (N * K <= 1,048,576)."""
        _check(load().amg_apply_noalloc(self._h, _dev_ptr(x, "x"), _dev_ptr(y, "y"), self._nrhs(x),
                                        _stream_ptr(stream)))
        return y

    def fgmres(self, b, x, rtol=1e-8, restart=100, maxit=500, stream=None):
        """amg_fgmres_solve on device tensors; returns (status, iters, relres)."""
        k = self._nrhs(b)
        its = np.zeros(k, dtype=np.int32)
        rel = np.zeros(k, dtype=np.float64)
        st = _check(load().amg_fgmres_solve(self._h, _dev_ptr(b, "b"), _dev_ptr(x, "x"), k, float(rtol), int(restart),
                                            int(maxit), _ptr(its, ctypes.c_int), _ptr(rel, ctypes.c_double),
                                            _stream_ptr(stream)))
        return st, its, rel

    def fgmres_host(self, b_host, x_host, rtol=1e-8, restart=100, maxit=500, stream=None):
        """amg_fgmres_solve_host on host (pinned or pageable) float64 tensors or arrays."""
        import torch
        k = 1 if b_host.ndim == 1 else int(b_host.shape[1])
        for t, nm in ((b_host, "b"), (x_host, "x")):
            if isinstance(t, torch.Tensor):
                if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
                    raise TypeError(f"{nm} must be a contiguous float64 host tensor")
        bp = ctypes.c_void_p(b_host.data_ptr() if isinstance(b_host, torch.Tensor) else b_host.ctypes.data)
        xp = ctypes.c_void_p(x_host.data_ptr() if isinstance(x_host, torch.Tensor) else x_host.ctypes.data)
        its = np.zeros(k, dtype=np.int32)
        rel = np.zeros(k, dtype=np.float64)
        st = _check(load().amg_fgmres_solve_host(self._h, bp, xp, k, float(rtol), int(restart), int(maxit),
                                                 _ptr(its, ctypes.c_int), _ptr(rel, ctypes.c_double),
                                                 _stream_ptr(stream)))
        return st, its, rel

    def profile_arnoldi(self, nrhs, nv, reps=10, stream=None):
        """amg_profile_arnoldi: average ms of the inner-product and the update kernel of one
        Gram-Schmidt pass with nv basis vectors (overwrites the solver workspace)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(load().amg_profile_arnoldi(self._h, int(nrhs), int(nv), int(reps), ctypes.byref(a), ctypes.byref(b),
                                          _stream_ptr(stream)))
        return a.value, b.value

    def profile_vcycle(self, nrhs, reps=10, stream=None):
        """Per (level, kernel class) summed ms and launch counts over `reps` cycles
        (amg_profile_vcycle); arrays of shape (levels, len(KERNEL_CLASSES))."""
        L = self.num_levels()
        ms = np.zeros(L * len(KERNEL_CLASSES))
        cnt = np.zeros(L * len(KERNEL_CLASSES), dtype=np.int64)
        _check(load().amg_profile_vcycle(self._h, int(nrhs), int(reps), _ptr(ms, ctypes.c_double),
                                         _ptr(cnt, ctypes.c_longlong), _stream_ptr(stream)))
        return ms.reshape(L, -1), cnt.reshape(L, -1)

    GS_VARIANTS = {-1: "not chosen", 0: "one block", 1: "cluster", 2: "pipelined", 3: "phase launches", 4: "dense map"}

    def gs_variants(self, nrhs) -> list:
        """Per level: (variant name, cluster size, measured ms) of the Gauss-Seidel kernel
        the autotuner chose for nrhs right-hand sides (amg_gs_variant)."""
        out = []
        for l in range(self.num_levels()):
            c = ctypes.c_int()
            ms = ctypes.c_float()
            v = load().amg_gs_variant(self._h, l, int(nrhs), ctypes.byref(c), ctypes.byref(ms))
            out.append((self.GS_VARIANTS.get(v, str(v)), c.value, ms.value))
        return out

    def set_gs_variant(self, level, nrhs, variant, cluster=0):
        """amg_set_gs_variant: fix the Gauss-Seidel variant of a level (a name of
        GS_VARIANTS or its number) for nrhs right-hand sides."""
        if isinstance(variant, str):
            variant = {v: k for k, v in self.GS_VARIANTS.items()}[variant]
        _check(load().amg_set_gs_variant(self._h, int(level), int(nrhs), int(variant), int(cluster)))

    def row_shapes(self, nrhs) -> dict:
        """{level: {kernel class: row mapping 0-3}} of the sparse kernels (amg_row_shape)."""
        out = {}
        for l in range(self.num_levels() - 1):
            out[l] = {c: load().amg_row_shape(self._h, l, int(nrhs), k) for k, c in enumerate(KERNEL_CLASSES)
                      if c not in ("gs_color", "coarse", "vanka", "ilu")}
        return out

    def kernel_launches(self) -> int:
        """Kernels launched by this hierarchy so far (amg_kernel_launches)."""
        return int(load().amg_kernel_launches(self._h))

    # -- inspection (host copies of the setup) --
    def num_levels(self) -> int:
        return load().amg_num_levels(self._h)

    def level_info(self, level: int) -> dict:
        info = AmgLevelInfo()
        _check(load().amg_level_get_info(self._h, level, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in AmgLevelInfo._fields_}

    def level_matrix(self, level: int, which: str):
        """(rowptr int64, col int32, val float64, shape) of one matrix of a level."""
        info = self.level_info(level)
        d, nv, np_ = info["dim"], info["n_v"], info["n_p"]
        nvc = npc = 0
        if level + 1 < self.num_levels():
            ci = self.level_info(level + 1)
            nvc, npc = ci["n_v"], ci["n_p"]
        shapes = {"A": (nv, nv), "B": (np_, d * nv), "Bt": (d * nv, np_), "S": (np_, np_), "P": (nv, nvc),
                  "Pp": (np_, npc), "R": (nvc, nv), "Rp": (npc, np_)}
        nnz = {"A": "nnz_A", "B": "nnz_B", "Bt": "nnz_Bt", "S": "nnz_S", "P": "nnz_P", "Pp": "nnz_Pp",
               "R": "nnz_R", "Rp": "nnz_Rp"}[which]
        shape = shapes[which]
        rp = np.zeros(shape[0] + 1, dtype=np.int64)
        col = np.zeros(max(info[nnz], 1), dtype=np.int32)
        val = np.zeros(max(info[nnz], 1), dtype=np.float64)
        _check(load().amg_level_get_matrix(self._h, level, MATRICES[which], _ptr(rp, ctypes.c_longlong),
                                           _ptr(col, ctypes.c_int), _ptr(val, ctypes.c_double)))
        return rp, col[:info[nnz]], val[:info[nnz]], shape

    def level_vanka(self, level: int) -> dict:
        """Vanka blocks of a level (amg_level_get_vanka): ptr, dofs, colors, ncolors."""
        nb, nd, nc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().amg_level_get_vanka(self._h, level, ctypes.byref(nb), ctypes.byref(nd), ctypes.byref(nc),
                                          None, None, None))
        ptr = np.zeros(nb.value + 1, dtype=np.int32)
        dofs = np.zeros(max(nd.value, 1), dtype=np.int32)
        colors = np.zeros(max(nb.value, 1), dtype=np.int32)
        _check(load().amg_level_get_vanka(self._h, level, None, None, None, _ptr(ptr, ctypes.c_int),
                                          _ptr(dofs, ctypes.c_int), _ptr(colors, ctypes.c_int)))
        return dict(ptr=ptr, dofs=dofs[:nd.value], colors=colors[:nb.value], ncolors=nc.value)

    def level_ilu(self, level: int) -> dict:
        """ILU(1) factors of a level (amg_level_get_ilu): perm (position -> dof), the strict
        lower and upper factors as (ptr, col, val), the pivots and both substitutions' depths."""
        n, nl, nu = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
        dl, du = ctypes.c_int(), ctypes.c_int()
        _check(load().amg_level_get_ilu(self._h, level, ctypes.byref(n), ctypes.byref(nl), ctypes.byref(nu),
                                        ctypes.byref(dl), ctypes.byref(du), None, None, None, None, None, None,
                                        None, None))
        N = n.value
        perm = np.zeros(N, dtype=np.int32)
        lp, up = np.zeros(N + 1, dtype=np.int32), np.zeros(N + 1, dtype=np.int32)
        lc, uc = np.zeros(max(nl.value, 1), dtype=np.int32), np.zeros(max(nu.value, 1), dtype=np.int32)
        lv, uv = np.zeros(max(nl.value, 1)), np.zeros(max(nu.value, 1))
        piv = np.zeros(N)
        _check(load().amg_level_get_ilu(self._h, level, None, None, None, None, None, _ptr(perm, ctypes.c_int),
                                        _ptr(lp, ctypes.c_int), _ptr(lc, ctypes.c_int), _ptr(lv, ctypes.c_double),
                                        _ptr(up, ctypes.c_int), _ptr(uc, ctypes.c_int), _ptr(uv, ctypes.c_double),
                                        _ptr(piv, ctypes.c_double)))
        return dict(perm=perm, lower=(lp, lc[:nl.value], lv[:nl.value]), upper=(up, uc[:nu.value], uv[:nu.value]),
                    pivots=piv, depth_lower=dl.value, depth_upper=du.value)

    def level_gs_map(self, level: int) -> np.ndarray:
        """The dense Gauss-Seidel map of a small level (amg_level_get_gs_map), n_p x n_p."""
        n = ctypes.c_int()
        _check(load().amg_level_get_gs_map(self._h, int(level), ctypes.byref(n), None))
        M = np.zeros((n.value, n.value))
        _check(load().amg_level_get_gs_map(self._h, int(level), None, _ptr(M, ctypes.c_double)))
        return M

    def coarse_inverse(self) -> np.ndarray:
        """The coarsest level's pseudo-inverse (amg_coarse_inverse), N_c x N_c."""
        n = ctypes.c_int()
        _check(load().amg_coarse_inverse(self._h, ctypes.byref(n), None))
        X = np.zeros((n.value, n.value))
        _check(load().amg_coarse_inverse(self._h, None, _ptr(X, ctypes.c_double)))
        return X

    def set_wait_limit(self, polls: int):
        """Poll limit of the bounded device waits (amg_set_wait_limit; <= 0: the default)."""
        _check(load().amg_set_wait_limit(self._h, int(polls)))

    def level_points(self, level: int) -> dict:
        info = self.level_info(level)
        cp = np.zeros(max(info["n_cp"], 1), dtype=np.int32)
        cv = np.zeros(max(info["n_cv"], 1), dtype=np.int32)
        colors = np.zeros(max(info["n_p"], 1), dtype=np.int32)
        D = np.zeros(max(info["n_v"], 1), dtype=np.float64)
        _check(load().amg_level_get_points(self._h, level, _ptr(cp, ctypes.c_int), _ptr(cv, ctypes.c_int),
                                           _ptr(colors, ctypes.c_int), _ptr(D, ctypes.c_double)))
        return dict(Cp=cp[:info["n_cp"]], Cv=cv[:info["n_cv"]], colors=colors[:info["n_p"]], D=D[:info["n_v"]])


def _host_ptr(a, what):
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError(f"{what} must be a contiguous float64 host tensor")
        return ctypes.c_void_p(a.data_ptr())
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError(f"{what} must be a contiguous float64 host array")
    return ctypes.c_void_p(a.ctypes.data)


class Server:
    """Request server (amg_server_*): continuous batching of FGMRES solves over
    resident hierarchies.  submit() queues a solve on host buffers, progress()
    never blocks and returns the tickets that completed, result() collects one."""

    def __init__(self, max_active=16, device_bytes=0, restart=100, maxit=500, merge_k=8, policy=0):
        lib = load()
        prm = AmgServerParams()
        lib.amg_server_params_default(ctypes.byref(prm))
        prm.max_active, prm.device_bytes, prm.restart, prm.maxit = int(max_active), int(device_bytes), int(restart), \
            int(maxit)
        prm.merge_k = int(merge_k)
        prm.policy = int(policy)
        h = ctypes.c_void_p()
        self._check(lib.amg_server_create(ctypes.byref(prm), ctypes.byref(h)))
        self._s = h
        self._keep = {}  # ticket -> (hierarchy, b, x, nrhs): alive until collected

    def _check(self, st):
        if st < 0:
            raise AmgError(st, load().amg_server_last_error(getattr(self, "_s", None)).decode())
        return st

    def submit(self, H: "Hierarchy", b_host, x_host, rtol=1e-8) -> int:
        k = 1 if b_host.ndim == 1 else int(b_host.shape[1])
        t = ctypes.c_longlong()
        self._check(load().amg_server_submit(self._s, H._h, _host_ptr(b_host, "b"), _host_ptr(x_host, "x"), k,
                                             float(rtol), ctypes.byref(t)))
        self._keep[t.value] = (H, b_host, x_host, k)
        return t.value

    def reserve(self, H: "Hierarchy", nrhs: int, count: int = 1):
        """Pre-create idle slots (graphs captured) for requests of nrhs right-hand sides on H."""
        self._check(load().amg_server_reserve(self._s, H._h, int(nrhs), int(count)))

    def progress(self, cap=256):
        done = np.zeros(cap, dtype=np.int64)
        n = ctypes.c_int()
        self._check(load().amg_server_progress(self._s, _ptr(done, ctypes.c_longlong), int(cap), ctypes.byref(n)))
        return [int(v) for v in done[:n.value]]

    def result(self, ticket):
        """(status, iters, relres, (queue_s, total_s)) of a completed request; None if it is not done."""
        k = self._keep[ticket][3]
        state = ctypes.c_int()
        its = np.zeros(k, dtype=np.int32)
        rel = np.zeros(k, dtype=np.float64)
        sec = np.zeros(2, dtype=np.float64)
        st = ctypes.c_int()
        self._check(load().amg_server_result(self._s, int(ticket), ctypes.byref(state), _ptr(its, ctypes.c_int),
                                             _ptr(rel, ctypes.c_double), _ptr(sec, ctypes.c_double),
                                             ctypes.byref(st)))
        if state.value != 2:
            return None
        del self._keep[ticket]
        return st.value, its, rel, (float(sec[0]), float(sec[1]))

    def state(self, ticket) -> int:
        """0 queued, 1 running, 2 done (the request is not collected)."""
        st = ctypes.c_int()
        self._check(load().amg_server_state(self._s, int(ticket), ctypes.byref(st)))
        return st.value

    def stats(self) -> dict:
        s = AmgServerStats()
        self._check(load().amg_server_get_stats(self._s, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in AmgServerStats._fields_}

    def close(self):
        if getattr(self, "_s", None):
            load().amg_server_destroy(self._s)
            self._s = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_stream(server: Server, requests, clock=None):
    """Drive a request stream through a Server in real time.

    requests: sequence of dicts with t (arrival, seconds after the start), H (a
    Hierarchy), b and x (host float64 tensors, N x nrhs; pinned keeps the copies
    asynchronous) and rtol.  Each request is submitted once its arrival time has
    passed; progress() is polled without sleeping.  Returns, per request, a dict
    with arrival, submit and done times (seconds after the start), queued (seconds
    from submission to admission), status, iters and relres."""
    import time
    clock = clock or time.perf_counter
    order = sorted(range(len(requests)), key=lambda i: requests[i]["t"])
    out = [None] * len(requests)
    ticket_of, submitted = {}, {}
    nxt, finished = 0, 0
    t0 = clock()
    while finished < len(requests):
        now = clock() - t0
        while nxt < len(order) and requests[order[nxt]]["t"] <= now:
            i = order[nxt]
            r = requests[i]
            ticket_of[server.submit(r["H"], r["b"], r["x"], rtol=r.get("rtol", 1e-8))] = i
            submitted[i] = clock() - t0
            nxt += 1
        for t in server.progress():
            i = ticket_of.pop(t)
            st, its, rel, sec = server.result(t)
            out[i] = dict(arrival=requests[i]["t"], submit=submitted[i], done=clock() - t0, status=st, iters=its,
                          relres=rel, queued=sec[0])
            finished += 1
    return out
