"""ctypes declarations of the C ABI in include/ravanka.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

P = ctypes.c_void_p
I32 = ctypes.c_int
F64 = ctypes.c_double
I64P = ctypes.POINTER(ctypes.c_int64)

RAV_OK = 0
ERRORS = {
    -1: "RAV_ERR_ARG", -2: "RAV_ERR_CUDA", -3: "RAV_ERR_SINGULAR_PATCH", -4: "RAV_ERR_SINGULAR_COARSE",
    -5: "RAV_ERR_NOT_CONVERGED", -6: "RAV_ERR_DIVERGED", -7: "RAV_ERR_NAN", -8: "RAV_ERR_TIMEOUT",
}


class RavProblem(ctypes.Structure):
    _fields_ = [("dim", I32), ("N", I32), ("coords_host", P), ("eta0", F64), ("nblobs", I32),
                ("blobs_host", P), ("bc", I32), ("element", I32), ("beta", F64)]


class RavSolveOpts(ctypes.Structure):
    _fields_ = [("tol", F64), ("maxit", I32), ("nu_pre", I32), ("nu_post", I32), ("outer", I32),
                ("restart", I32), ("diverge", F64), ("fallback_rho", F64)]


class RavSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", I32), ("status", I32), ("final_ratio", F64), ("history_host", P),
                ("fell_back", I32)]


_SIGS = {
    "mg_setup": (I32, [ctypes.POINTER(RavProblem), I32, P, ctypes.POINTER(P)]),
    "mg_destroy": (None, [P]),
    "rav_get_counts": (I32, [P, I32, I64P]),
    "rav_get_csr": (I32, [P, I32, P, P, P, P]),
    "rav_assemble_rhs": (I32, [P, I32, P, P]),
    "rav_initial_guess": (I32, [P, P, P]),
    "rav_residual": (I32, [P, I32, P, P, P, ctypes.POINTER(F64), P]),
    "rav_residual_norm_noalloc": (I32, [P, I32, P, P, P, P, P]),
    "rav_set_residual_split": (I32, [P, I32, I32]),
    "rav_get_residual_split": (I32, [P, I32]),
    "rav_set_residual_blocked": (I32, [P, I32, I32, P]),
    "rav_get_residual_blocked": (I32, [P, I32]),
    "rav_restrict": (I32, [P, I32, P, P, P]),
    "rav_prolong_add": (I32, [P, I32, P, P, P]),
    "rav_coarse_solve": (I32, [P, P, P, P]),
    "vanka_setup": (I32, [P, I32, I32, F64, P, ctypes.POINTER(P)]),
    "vanka_destroy": (None, [P]),
    "rav_set_patch_omega": (I32, [P, I32, P, P]),
    "rav_set_apply_split": (I32, [P, I32, I32, P]),
    "rav_get_apply_split": (I32, [P, I32]),
    "rav_set_apply_staged": (I32, [P, I32, I32, P]),
    "batch_set_tensor_apply": (I32, [P, I32, P]),
    "rav_fp64_fma_rate": (I32, [ctypes.POINTER(F64), P]),
    "rav_hbm_read_rate": (I32, [ctypes.c_int64, ctypes.POINTER(F64), P]),
    "rav_set_coarse_residual_f32": (I32, [P, I32, ctypes.c_int64, P]),
    "rav_get_coarse_residual_f32": (I32, [P]),
    "rav_set_transfers_f32": (I32, [P, I32, P]),
    "rav_get_transfers_f32": (I32, [P]),
    "batch_tensor_apply_levels": (I32, [P]),
    "batch_set_coarse_residual_f32": (I32, [P, I32, P]),
    "batch_coarse_residual_f32": (I32, [P]),
    "batch_set_transfers_f32": (I32, [P, I32, P]),
    "batch_transfers_f32": (I32, [P]),
    "rav_get_apply_staged": (I32, [P, I32]),
    "rav_set_fused_smoothing": (I32, [P, I32]),
    "rav_get_patch_counts": (I32, [P, I32, I64P]),
    "rav_get_patches": (I32, [P, I32, P, P, P, P]),
    "rav_get_inverse_rows": (I32, [P, I32, ctypes.c_int64, ctypes.c_int64, P, P]),
    "vanka_smooth": (I32, [P, I32, P, P, I32, P]),
    "vanka_apply": (I32, [P, I32, P, P, P]),
    "vcycle": (I32, [P, P, P, P, I32, I32, P]),
    "rav_set_graphs": (I32, [P, I32]),
    "solve": (I32, [P, P, P, P, ctypes.POINTER(RavSolveOpts), ctypes.POINTER(RavSolveInfo), P]),
    "rav_profile_enable": (I32, [P, ctypes.c_uint, I32]),
    "rav_profile_read": (I32, [P, I32, I32, I64P, ctypes.POINTER(F64)]),
    "rav_kernel_launches": (ctypes.c_int64, []),
    "rav_mlp_nparam": (I32, []),
    "rav_patch_features": (I32, [P, I32, P, P]),
    "rav_label_collection": (I32, [P, I32]),
    "rav_read_labels": (I32, [P, I32, P, P]),
    "rav_mlp_forward": (I32, [P, P, ctypes.c_int64, P, P]),
    "rav_mlp_loss_grad": (I32, [P, P, P, ctypes.c_int64, P, P, P, ctypes.c_int64, P]),
    "rav_adam_step": (I32, [P, P, P, P, ctypes.c_float, I32, P]),
    "rav_set_learned_omega": (I32, [P, P, F64, P]),
    "rav_reset_omega": (I32, [P, P]),
    "batch_setup": (I32, [P, P, I32, I32, P, ctypes.POINTER(P)]),
    "batch_destroy": (None, [P]),
    "batch_get_tuning": (I32, [P, ctypes.POINTER(I32)]),
    "batch_set_apply_tile": (I32, [P, I32, I32, P]),
    "batch_get_apply_tile": (I32, [P, I32, ctypes.POINTER(I32)]),
    "batch_profile_enable": (I32, [P, I32]),
    "batch_profile_read": (I32, [P, I32, I32, I64P, ctypes.POINTER(F64)]),
    "batch_vcycle": (I32, [P, P, P, I32, I32, P]),
    "solve_batched": (I32, [P, P, P, ctypes.POINTER(RavSolveOpts), P, P, P]),
    "rav_strerror": (ctypes.c_char_p, [I32]),
}

_lib = None


def load():
    """Loads (building first if needed) the in-tree libravanka.so; raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise ImportError("libravanka.so is missing and could not be built")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


class RavError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = load().rav_strerror(code).decode()
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({msg})")


def check(code, where=""):
    if code != RAV_OK:
        raise RavError(code, where)
    return code
