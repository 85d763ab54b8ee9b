"""ctypes view of the C ABI in include/hydot.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhydot.so")

HYDOT_OK = 0
HYDOT_ERR_ARG = -1
HYDOT_ERR_OOM = -2
HYDOT_ERR_CUDA = -3
HYDOT_ERR_NOT_CONVERGED = -4
HYDOT_ERR_TIMEOUT = -5
HYDOT_ERR_STATE = -6
HYDOT_ERR_HOST = -7
STATUS_NAMES = {0: "HYDOT_OK", -1: "HYDOT_ERR_ARG", -2: "HYDOT_ERR_OOM", -3: "HYDOT_ERR_CUDA",
                -4: "HYDOT_ERR_NOT_CONVERGED", -5: "HYDOT_ERR_TIMEOUT", -6: "HYDOT_ERR_STATE",
                -7: "HYDOT_ERR_HOST"}

HYDOT_FP64 = 0
HYDOT_MIXED = 1

# Every symbol include/hydot.h declares.
EXPORTS = ("hydot_version", "hydot_setup", "hydot_set_stream", "hydot_solve_fields", "hydot_solve_batch",
           "hydot_born_assemble",
           "hydot_born_apply", "hydot_born_apply_T", "hydot_born_apply_noalloc", "hydot_solve_adjoint",
           "hydot_born_apply_T_adjoint", "hydot_sketch_range",
           "hydot_sketch_project", "hydot_sketch_orthonormalize", "hydot_sketch_rank", "hydot_sketch_merge",
           "hydot_source_tree",
           "hydot_sketch_factor", "hydot_set_kernel_timing", "hydot_set_graphs", "hydot_get_launch_mode",
           "hydot_kernel_stats", "hydot_kernel_launches", "hydot_get_tuning", "hydot_set_absorption",
           "hydot_wait_selftest", "hydot_set_shift_guess", "hydot_shift_guess_fields",
           "hydot_pals_reconstruct", "hydot_pals_shape", "hydot_pals_project", "hydot_shape_compare",
           "hydot_last_error", "hydot_destroy")
ROLL_VARIANTS = 4  # HYDOT_ROLL_VARIANTS
KERNELS = {"dir": 0, "update": 1, "residual": 2, "born_rows": 3, "apply": 4, "apply_T": 5, "sketch_range": 6,
           "sketch_project": 7, "iter": 8, "sweep": 9, "prime": 10}


class Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("h_mm", C.c_double),
        ("robin_A", C.c_double * 6),
        ("n_lambda", C.c_int), ("n_chrom", C.c_int),
        ("eps", C.POINTER(C.c_double)), ("c_bg", C.POINTER(C.c_double)), ("mus_prime", C.POINTER(C.c_double)),
        ("omega", C.c_double), ("c_medium", C.c_double),
        ("n_src", C.c_int), ("n_det", C.c_int),
        ("src_ijk", C.POINTER(C.c_int)), ("det_ijk", C.POINTER(C.c_int)),
        ("precision", C.c_int),
        ("tol", C.c_double), ("tol_cw", C.c_double), ("inner_tol", C.c_double),
        ("max_iter", C.c_int), ("deflation_k", C.c_int), ("max_lambda_per_call", C.c_int),
        ("cw_floor", C.c_double),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("n_fields", C.c_int), ("n_not_converged", C.c_int), ("iters_max", C.c_int),
        ("iters_mean", C.c_double), ("cycles_max", C.c_int), ("resid_max", C.c_double), ("cw_max", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PalsOptions(C.Structure):
    _fields_ = [("tau", C.c_double), ("eps", C.c_double), ("nu", C.c_double), ("gamma", C.c_double),
                ("noise_norm", C.c_double), ("lm_nu0", C.c_double), ("max_outer", C.c_int), ("max_inner", C.c_int),
                ("fix_c", C.c_int)]


class PalsResult(C.Structure):
    _fields_ = [("evaluations", C.c_int), ("accepted", C.c_int), ("residual0", C.c_double), ("residual", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libhydot.so; raises (never falls back) when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhydot.so not built ({path}); run __graft_entry__.build() or "
                           "python -m paper_1410_0986_gb300._build")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.hydot_version.restype = C.c_int
    lib.hydot_set_graphs.argtypes = [vp, C.c_int]
    lib.hydot_set_graphs.restype = C.c_int
    lib.hydot_get_launch_mode.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.hydot_get_launch_mode.restype = C.c_int
    lib.hydot_setup.argtypes = [C.POINTER(Problem), vp, C.POINTER(vp)]
    lib.hydot_setup.restype = C.c_int
    lib.hydot_set_stream.argtypes = [vp, vp]
    lib.hydot_set_stream.restype = C.c_int
    lib.hydot_solve_fields.argtypes = [vp, C.c_int, C.c_int, vp, vp, C.POINTER(Stats)]
    lib.hydot_solve_fields.restype = C.c_int
    lib.hydot_solve_batch.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(vp),
                                      C.POINTER(vp), C.POINTER(Stats), C.POINTER(C.c_int)]
    lib.hydot_solve_batch.restype = C.c_int
    lib.hydot_born_assemble.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_longlong, C.c_longlong, vp, C.c_longlong]
    lib.hydot_born_assemble.restype = C.c_int
    lib.hydot_born_apply.argtypes = [vp, vp, vp, C.c_int, C.c_int, vp, vp]
    lib.hydot_born_apply.restype = C.c_int
    lib.hydot_born_apply_T.argtypes = [vp, vp, vp, C.c_int, C.c_int, vp, vp]
    lib.hydot_born_apply_T.restype = C.c_int
    lib.hydot_solve_adjoint.argtypes = [vp, C.c_int, C.c_int, vp, vp, C.POINTER(Stats)]
    lib.hydot_solve_adjoint.restype = C.c_int
    lib.hydot_born_apply_T_adjoint.argtypes = [vp, vp, vp, C.c_int, C.c_int, vp]
    lib.hydot_born_apply_T_adjoint.restype = C.c_int
    lib.hydot_born_apply_noalloc.argtypes = [C.c_longlong, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                             C.POINTER(C.c_double), vp, vp, vp, vp, vp]
    lib.hydot_born_apply_noalloc.restype = C.c_int
    lib.hydot_sketch_range.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int, vp, C.c_longlong]
    lib.hydot_sketch_range.restype = C.c_int
    lib.hydot_sketch_project.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int, C.c_longlong, vp,
                                         C.c_longlong]
    lib.hydot_sketch_project.restype = C.c_int
    lib.hydot_sketch_orthonormalize.argtypes = [vp, vp, C.c_longlong, C.c_int, C.c_longlong, C.POINTER(C.c_int),
                                                C.POINTER(C.c_double)]
    lib.hydot_sketch_orthonormalize.restype = C.c_int
    lib.hydot_sketch_rank.argtypes = [vp, vp, C.c_longlong, C.c_longlong, C.c_int, vp, C.c_longlong, C.c_int,
                                      C.c_double, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    lib.hydot_sketch_rank.restype = C.c_int
    lib.hydot_sketch_merge.argtypes = [vp, vp, C.c_longlong, C.c_longlong, C.POINTER(C.c_double), vp, C.c_longlong,
                                       C.c_int, vp, C.c_longlong, C.c_longlong, C.POINTER(C.c_double), vp,
                                       C.c_longlong, C.c_int, C.c_longlong, C.c_double, C.c_int, vp, C.c_longlong,
                                       C.POINTER(C.c_double), vp, C.c_longlong, C.POINTER(C.c_int)]
    lib.hydot_sketch_merge.restype = C.c_int
    dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
    lib.hydot_source_tree.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, ip, ip,
                                      ip, ip]
    lib.hydot_source_tree.restype = C.c_int
    lib.hydot_sketch_factor.argtypes = [vp, vp, C.c_longlong, C.c_longlong, vp, C.c_longlong, C.c_longlong, C.c_int,
                                        C.c_int, vp, C.c_longlong, C.POINTER(C.c_double), vp, C.c_longlong]
    lib.hydot_sketch_factor.restype = C.c_int
    lib.hydot_set_kernel_timing.argtypes = [vp, C.c_int]
    lib.hydot_set_kernel_timing.restype = C.c_int
    lib.hydot_kernel_stats.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                       C.POINTER(C.c_double)]
    lib.hydot_kernel_stats.restype = C.c_int
    lib.hydot_kernel_launches.argtypes = [vp]
    lib.hydot_kernel_launches.restype = C.c_longlong
    lib.hydot_get_tuning.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_double)]
    lib.hydot_get_tuning.restype = C.c_int
    lib.hydot_set_absorption.argtypes = [vp, C.POINTER(C.c_double)]
    lib.hydot_set_absorption.restype = C.c_int
    lib.hydot_wait_selftest.argtypes = [vp, C.c_int]
    lib.hydot_wait_selftest.restype = C.c_int
    lib.hydot_set_shift_guess.argtypes = [vp, C.c_int]
    lib.hydot_set_shift_guess.restype = C.c_int
    dp = C.POINTER(C.c_double)
    lib.hydot_pals_reconstruct.argtypes = [vp, vp, C.c_longlong, C.c_longlong, dp, vp, C.c_longlong, C.c_int, vp,
                                           C.c_int, dp, dp, C.POINTER(PalsOptions), C.POINTER(PalsResult)]
    lib.hydot_pals_reconstruct.restype = C.c_int
    lib.hydot_pals_shape.argtypes = [vp, C.c_int, dp, C.c_double, C.c_double, C.c_double, vp]
    lib.hydot_pals_shape.restype = C.c_int
    lib.hydot_pals_project.argtypes = [vp, vp, C.c_longlong, C.c_int, C.c_int, dp, C.c_double, C.c_double,
                                       C.c_double, dp]
    lib.hydot_pals_project.restype = C.c_int
    lib.hydot_shape_compare.argtypes = [vp, vp, vp, C.c_double, dp, dp]
    lib.hydot_shape_compare.restype = C.c_int
    lib.hydot_shift_guess_fields.argtypes = [vp, C.c_int, C.c_int, vp, vp]
    lib.hydot_shift_guess_fields.restype = C.c_int
    lib.hydot_last_error.argtypes = [vp]
    lib.hydot_last_error.restype = C.c_char_p
    lib.hydot_destroy.argtypes = [vp]
    lib.hydot_destroy.restype = None
    _lib = lib
    return lib
