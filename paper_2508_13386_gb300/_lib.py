"""ctypes declarations of the C ABI in ``include/mls.h``.

Loads ``libmls.so`` from this package directory.  There is no fallback: if
the library is missing, importing this module raises ImportError telling the
user to build it.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmls.so")

MLS_OK = 0
STATUS = {
    0: "MLS_OK", -1: "MLS_EINVAL", -2: "MLS_ENOMEM", -3: "MLS_ECUDA", -4: "MLS_ENOTCONV",
    -5: "MLS_ELINESEARCH", -6: "MLS_ECHOL", -7: "MLS_ENONFINITE", -8: "MLS_ETIMEOUT",
    -9: "MLS_EINVERTED",
}
PRECISION = {"fp64": 0, "fp32": 1, "mixed_fp32": 1, "bf16": 2, "mixed_bf16": 2}
PRECOND = {"jacobi": 0, "block_jacobi": 0, "two_level": 1, "multilevel": 1}
CYCLE = {"additive": 0, "multiplicative": 1}


class Options(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("preconditioner", C.c_int),
        ("cycle", C.c_int),
        ("omega", C.c_double),
        ("newton_tol", C.c_double),
        ("pcg_rtol", C.c_double),
        ("max_newton", C.c_int),
        ("max_pcg", C.c_int),
        ("coarse_refresh", C.c_int),
        ("coarse_lag_steps", C.c_int),
        ("pcg_check_every", C.c_int),
        ("persistent", C.c_int),
        ("persist_blocks_per_sm", C.c_int),
        ("direction", C.c_int),
        ("refine_iters", C.c_int),
        ("paper_tol", C.c_double),
        ("stream", C.c_void_p),
        ("sub_rtol", C.c_double),
        ("hessian_lag", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("newton_iters", C.c_int),
        ("pcg_iters", C.c_int),
        ("line_search_trials", C.c_int),
        ("coarse_builds", C.c_int),
        ("step_rel", C.c_double),
        ("grad_norm", C.c_double),
        ("energy", C.c_double),
        ("kernel_launches", C.c_int64),
        ("warm_start_used", C.c_int),
        ("coarse_shifts", C.c_int),
        ("coarse_fallbacks", C.c_int),
        ("subspace_iters", C.c_int),
        ("hessian_refreshes", C.c_int),
        ("contact_pairs", C.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# (name, argtypes) for every entry point declared in include/mls.h
_P = C.c_void_p
_D = C.c_double
_I = C.c_int
_I32 = C.c_int32
SIGNATURES = {
    "mls_default_options": [C.POINTER(Options)],
    "mls_create": [C.POINTER(_P), C.POINTER(Options)],
    "mls_destroy": [_P],
    "mls_last_error": [_P],
    "mls_set_options": [_P, C.POINTER(Options)],
    "mls_smoother_omega": [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "mls_upload_cubature": [_P, _P],
    "mls_tridiag_max_eig": [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int],
    "mls_upload_mesh": [_P, _I32, _P, _I32, _P, _P, _P, _P, _P],
    "mls_upload_basis": [_P, _I32, _P, _P, _P, _P],
    "mls_set_forces": [_P, _P, _I, _P, _D, _D, _D],
    "mls_set_friction": [_P, _D, _D],
    "mls_newton_step": [_P, _P, _P, _D, _P, C.POINTER(Stats)],
    "mls_newton_step_host": [_P, _P, _P, _D, _P, C.POINTER(Stats)],
    "mls_newton_step_bdf2": [_P, _P, _P, _P, _P, _D, _P, C.POINTER(Stats)],
    "mls_eval_elements": [_P, _P, _P, _P, _P],
    "mls_assemble": [_P, _P, _P, _P, _D, _P],
    "mls_get_hessian": [_P, _P, _P, _P, C.POINTER(C.c_int64)],
    "mls_spmv": [_P, _P, _P],
    "mls_precond_apply": [_P, _P, _P],
    "mls_pcg_solve": [_P, _P, _P, _D, _I, C.POINTER(_I), C.POINTER(_D)],
    "mls_prolong": [_P, _P, _P],
    "mls_restrict": [_P, _P, _P],
    "mls_build_coarse": [_P],
    "mls_get_coarse": [_P, _P],
    "mls_coarse_shift": [_P, _P],
    "mls_get_coarse_factor": [_P, _P],
    "mls_energy": [_P, _P, _P, _D, C.POINTER(_D), C.POINTER(_I)],
    "mls_ccd_bound": [_P, _P, _P, C.POINTER(_D)],
    "mls_set_bodies": [_P, _P, _D, _D, _I32],
    "mls_contact_pairs": [_P, _P, _P, C.c_int64, _P, C.POINTER(C.c_int64), _P, C.POINTER(C.c_int64)],
    "mls_contact_pair_derivatives": [_P, _P, _I32, _D, _D, _P, _P, _P, _P],
    "mls_profile_enable": [_P, C.c_uint32],
    "mls_profile_read": [_P, _P, _P],
    "mls_elastic_energy_noalloc": [_I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P],
    "mls_gemm_bf16": [_I32, _I32, _I32, _P, _I32, _P, _I32, _P, _I32, _P],
    "mls_mlp_create": [C.POINTER(_P), _I32, _I32, _I32, _I32, _P, _P],
    "mls_mlp_destroy": [_P],
    "mls_mlp_param_count": [_P],
    "mls_mlp_forward": [_P, _P, _I32, _P],
    "mls_mlp_gradients": [_P, _P, _P, _I32, _P, C.POINTER(_D)],
    "mls_mlp_adam_step": [_P, _P, C.c_float],
    "mls_mlp_train": [_P, _P, _P, _I32, _P, _I32, _I32, C.c_float, C.POINTER(_D)],
    "mls_mlp_get_params": [_P, _P],
    "mls_mlp_set_normalization": [_P, _P, _P, _P, _P],
    "mls_mlp_column_stats": [_P, _I32, _I32, _P, _P, _P],
    "mls_warm_start_enable": [_P, _I],
    "mls_warm_start_reset": [_P],
    "mls_warm_start_attach": [_P, _P],
    "mls_warm_start_sample": [_P, _P, _P],
    "mls_coarse_project": [_P, _P, _P],
    "mls_selftest_barrier": [_I32, _I32, _I32, C.POINTER(_I32), _P],
    "mls_batch_create": [C.POINTER(_P), _P],
    "mls_batch_last_error": [_P],
    "mls_batch_destroy": [_P],
    "mls_batch_upload": [_P, _I32, _P, _P, _P, _P, _P, _P, _P, _P],
    "mls_batch_set_forces": [_P, _P, C.c_int, _P, C.c_double, C.c_double, C.c_double],
    "mls_batch_set_friction": [_P, _D, _D],
    "mls_batch_upload_basis": [_P, _I32, _P, _P, _P, _P, _P],
    "mls_batch_retune": [_P],
    "mls_batch_step": [_P, _P, _P, C.c_double, _P, _P, _P],
    "mls_batch_step_bdf2": [_P, _P, _P, _P, _P, C.c_double, _P, _P, _P],
}
class BatchMeshStats(C.Structure):
    _fields_ = [
        ("status", C.c_int32),
        ("newton_iters", C.c_int32),
        ("pcg_iters", C.c_int32),
        ("line_search_trials", C.c_int32),
        ("step_rel", C.c_double),
        ("grad_norm", C.c_double),
        ("energy", C.c_double),
    ]


class BatchInfo(C.Structure):
    _fields_ = [
        ("kernel_launches", C.c_int64),
        ("graph_launches", C.c_int32),
        ("newton_rounds", C.c_int32),
        ("pcg_rounds", C.c_int32),
        ("line_search_rounds", C.c_int32),
        ("spmv_lanes", C.c_int32),
        ("row_threads", C.c_int32),
        ("rows_per_thread", C.c_int32),
        ("tune_ms", C.c_double),
    ]


PROF_CLASSES = ["elements", "assemble", "spmv", "pcg_update", "precond", "galerkin", "cholesky",
                "linesearch", "pcg_fused"]


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -m paper_2508_13386_gb300.build, or __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = {"mls_last_error": C.c_char_p, "mls_batch_last_error": C.c_char_p,
                      "mls_mlp_param_count": C.c_int64, "mls_tridiag_max_eig": C.c_double}.get(name, C.c_int)
    return lib
