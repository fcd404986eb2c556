"""ctypes declarations of include/qs3.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from .build import LIB

P = ctypes.c_void_p
I32 = ctypes.c_int32
U64 = ctypes.c_uint64
F64 = ctypes.c_double

QS3_F32, QS3_F64, QS3_C64, QS3_C128, QS3_C128DF, QS3_C128X = 0, 1, 2, 3, 4, 5
STATUS = {0: "QS3_OK", -1: "QS3_ERR_INVALID_ARG", -2: "QS3_ERR_OVERFLOW", -3: "QS3_ERR_SYMMETRY",
          -4: "QS3_ERR_OOM", -5: "QS3_ERR_CUDA", -6: "QS3_ERR_NOT_CONVERGED", -7: "QS3_ERR_TIMEOUT",
          -8: "QS3_ERR_STATE"}


class qs3_lattice(ctypes.Structure):
    _fields_ = [("n_sites", I32), ("n_bonds", I32), ("bi", P), ("bj", P), ("jxy", P), ("jz", P), ("h", P),
                ("L", I32 * 3), ("pos", P), ("n_sub", I32), ("reserved", I32)]


class qs3_solve_opts(ctypes.Structure):
    _fields_ = [("n_eig", I32), ("n_keep", I32), ("n_max", I32), ("max_iter", I32), ("min_iter", I32),
                ("check_every", I32), ("eps", F64), ("precision", I32), ("use_graphs", I32), ("seed", U64),
                ("refine_tol", F64), ("res_tol", F64), ("hphi_ieee", I32), ("strict64", I32)]


class qs3_solve_info(ctypes.Structure):
    _fields_ = [("iterations", I32), ("restarts", I32), ("converged", I32), ("refine_iterations", I32),
                ("max_residual", F64), ("seconds", F64), ("hphi_nnz", U64), ("hphi_seconds", F64),
                ("hphi_calls", I32), ("hphi_graph_calls", I32), ("gs_dot_seconds", F64), ("gs_dot_bytes", U64),
                ("gs_dot_calls", I32), ("reserved", I32), ("gs_dot_fma", U64)]


class qs3_peaks(ctypes.Structure):
    _fields_ = [("fp64_fma_per_s", F64), ("fp32_fma_per_s", F64), ("int_mad_per_s", F64), ("int_alu_per_s", F64),
                ("issue_per_s", F64), ("n_sms", I32), ("reserved", I32)]


# name -> (argtypes, restype); every entry point declared in include/qs3.h
SIGNATURES = {
    "qs3_basis_create": ([P, I32, I32, P, P], I32),
    "qs3_basis_destroy": ([P], I32),
    "qs3_basis_info": ([P, P, P], I32),
    "qs3_basis_dims": ([P, P], I32),
    "qs3_basis_ranks": ([P, I32, P, P], I32),
    "qs3_basis_nnz": ([P, P], I32),
    "qs3_basis_rep_table": ([P, I32, P], I32),
    "qs3_basis_tuning": ([P, I32, P, P, P], I32),
    "qs3_basis_store_terms": ([P, I32, P], I32),
    "qs3_full_diag": ([P, I32, P, P, P], I32),
    "qs3_thermal": ([ctypes.c_int64, P, P, P, I32, P, P, P], I32),
    "qs3_hphi": ([P, I32, P, P, P], I32),
    "qs3_gs_dots": ([P, I32, I32, P, U64, P, P, I32, P], I32),
    "qs3_split_df": ([P, P, U64, P], I32),
    "qs3_lanczos": ([P, P, P, P, P, P], I32),
    "qs3_trlanczos": ([P, P, P, P, P, P], I32),
    "qs3_batch_solve": ([I32, P, P, P, P, P, I32], I32),
    "qs3_correlations": ([P, I32, P, I32, P, P, P, P, I32, P, P, P, P], I32),
    "qs3_smq": ([P, I32, P, P, I32, P, P, P], I32),
    "qs3_smq_noalloc": ([P, I32, P, P, I32, P, P, P], I32),
    "qs3_dsf": ([P, I32, P, F64, P, I32, P, I32, F64, F64, I32, P, P, P, P, P, P], I32),
    "qs3_sq_apply": ([I32, P, I32, P, P, I32, P, P, P], I32),
    "qs3_dsf_op": ([I32, I32, P, I32, P, F64, P, I32, P, I32, F64, F64, I32, P, P, P, P, P, P], I32),
    "qs3_probe_peaks": ([P, P], I32),
    "qs3_inject_alloc_failure": ([ctypes.c_int64], ctypes.c_int64),
    "qs3_inject_wait_timeout": ([I32], I32),
    "qs3_strerror": ([I32], ctypes.c_char_p),
    "qs3_last_error": ([], ctypes.c_char_p),
    "qs3_version": ([], ctypes.c_char_p),
    "qs3_kernel_launches": ([], U64),
}

_lib = None


def load(path: str | None = None):
    """Load libqs3.so.  There is no fallback: a missing library is an error."""
    global _lib
    if _lib is None:
        p = path or LIB
        if not os.path.exists(p):
            raise RuntimeError(f"libqs3.so not built ({p}); run paper_2107_00872_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


class QS3Error(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        lib = load()
        detail = (lib.qs3_last_error() or b"").decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)} ({detail})")


def check(status: int, where: str, allow=()) -> int:
    if status != 0 and status not in allow:
        raise QS3Error(status, where)
    return status
