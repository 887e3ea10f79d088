"""ctypes declarations of libqoc.so (include/qoc.h).  Argument marshalling only.

The library is built in-tree by paper_2309_05884_gb300.build; loading fails loudly if it is
missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqoc.so")

QOC_OK = 0
QOC_EINVAL = -1
QOC_ENOMEM = -2
QOC_ECUDA = -3
QOC_ETIMEOUT = -4
QOC_EUNSUPPORTED = -5
QOC_ENOTCONVERGED = -6

QOC_PREC_F64 = 0
QOC_PREC_F32 = 1
QOC_PREC_F32_ALL = 2
QOC_RULE_FIXED = 0
QOC_RULE_ADAM = 1
QOC_BASIS_FIRST_BLOCK_ONLY = 1
QOC_BASIS_NO_VECTORS = 2
QOC_OBJ_STATE = 0
QOC_OBJ_GATE = 1


class qoc_term(C.Structure):
    _fields_ = [("kind", C.c_int), ("dist", C.c_int), ("coeff", C.c_double)]


class qoc_system_desc(C.Structure):
    _fields_ = [("n", C.c_int), ("group", C.c_int), ("n_h0_terms", C.c_int), ("h0", C.POINTER(qoc_term)),
                ("n_ctrl", C.c_int), ("n_hc_terms", C.POINTER(C.c_int)),
                ("hc", C.POINTER(C.POINTER(qoc_term)))]


class qoc_plan_opts(C.Structure):
    _fields_ = [("prec", C.c_int), ("grad_mode", C.c_int), ("max_squarings", C.c_int),
                ("ckpt_segment", C.c_int), ("objective", C.c_int), ("reserved", C.c_int * 3)]


class qoc_opt_opts(C.Structure):
    _fields_ = [("iters", C.c_int), ("rule", C.c_int), ("step", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("f_target", C.c_double), ("check_every", C.c_int),
                ("use_graph", C.c_int), ("freeze_converged", C.c_int), ("reserved", C.c_int * 3)]


# name -> (restype, argtypes); every symbol include/qoc.h declares
P = C.c_void_p
D = C.POINTER(C.c_double)
SIGNATURES = {
    "qoc_build_symmetry_basis": (C.c_int, [C.POINTER(qoc_system_desc), C.c_int, C.POINTER(P)]),
    "qoc_basis_free": (None, [P]),
    "qoc_basis_info": (C.c_int, [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64)]),
    "qoc_basis_block": (C.c_int, [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int64),
                                  C.c_char_p]),
    "qoc_basis_block_matrices": (C.c_int, [P, C.c_int, P, P]),
    "qoc_basis_norm_bounds": (C.c_int, [P, C.c_int, P]),
    "qoc_state_to_blocks": (C.c_int, [P, P, P]),
    "qoc_blocks_to_state": (C.c_int, [P, P, P]),
    "qoc_dicke_state": (C.c_int, [P, C.c_int, P]),
    "qoc_plan_opts_default": (None, [C.POINTER(qoc_plan_opts)]),
    "qoc_plan_create": (C.c_int, [P, C.c_int, C.c_double, C.POINTER(qoc_plan_opts), P, C.POINTER(P)]),
    "qoc_plan_create_batch": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                         C.POINTER(qoc_plan_opts), C.POINTER(P), C.POINTER(P)]),
    "qoc_plan_info": (C.c_int, [P, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "qoc_plan_free": (None, [P]),
    "qoc_plan_workspace_bytes": (C.c_int, [P, C.POINTER(C.c_size_t)]),
    "qoc_plan_sync_status": (C.c_int, [P, P]),
    "qoc_assemble_blocks": (C.c_int, [P, P, P, P]),
    "qoc_expm_blocks": (C.c_int, [P, P, P, P, C.c_size_t, P]),
    "qoc_propagate": (C.c_int, [P, P, P, P, P, C.c_size_t, P]),
    "qoc_fidelity_and_grad": (C.c_int, [P, P, P, P, P, P, P, C.c_size_t, P]),
    "qoc_fidelity_forward": (C.c_int, [P, P, P, P, P, P, C.c_size_t, P]),
    "qoc_fidelity_backward": (C.c_int, [P, P, P, P, P, P, C.c_size_t, P]),
    "qoc_plan_selftest_wait": (C.c_int, [P, C.c_double, P]),
    "qoc_opt_opts_default": (None, [C.POINTER(qoc_opt_opts)]),
    "qoc_optimize_pulses": (C.c_int, [P, P, P, P, C.POINTER(qoc_opt_opts), P, P, C.POINTER(C.c_int), P,
                                      C.c_size_t, P]),
    "qoc_plan_set_profiling": (C.c_int, [P, C.c_int]),
    "qoc_plan_phase_times": (C.c_int, [P, C.POINTER(C.c_float), C.c_int]),
    "qoc_plan_work_counts": (C.c_int, [P, C.POINTER(C.c_longlong), C.c_int]),
    "qoc_plan_kernel_launches": (C.c_int, [P, C.c_int, C.POINTER(C.c_int)]),
    "qoc_expm_batch_noalloc": (C.c_int, [P, P, C.c_int, C.c_longlong, P]),
    "qoc_plan_set_expm_rules": (C.c_int, [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "qoc_plan_set_sweep_cluster": (C.c_int, [P, C.c_int]),
    "qoc_plan_sweep_cluster": (C.c_int, [P, C.POINTER(C.c_int)]),
    "qoc_plan_set_deriv_gemm": (C.c_int, [P, C.c_int, C.c_int]),
    "qoc_plan_deriv_gemm": (C.c_int, [P, C.POINTER(C.c_int)]),
    "qoc_plan_set_persistent": (C.c_int, [P, C.c_int]),
    "qoc_plan_expm_classes": (C.c_int, [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "qoc_dense_forward": (C.c_int, [P, P, P, P, P, C.c_longlong, C.c_int, C.c_int, C.c_int, P]),
    "qoc_dense_backward": (C.c_int, [P, P, P, P, P, P, P, P, C.c_longlong, C.c_int, C.c_int, C.c_int, P]),
    "qoc_adam_step": (C.c_int, [P, P, P, P, P, C.c_longlong, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, P]),
    "qoc_mse": (C.c_int, [P, P, P, P, C.c_longlong, P]),
    "qoc_to_bf16": (C.c_int, [P, P, C.c_longlong, P]),
    "qoc_tc_cgemm": (C.c_int, [P, P, P, C.c_int, C.c_longlong, P, P]),
    "qoc_trotter_create": (C.c_int, [P, C.c_double, C.POINTER(P)]),
    "qoc_trotter_propagate": (C.c_int, [P, P, C.c_int, P, P, C.c_longlong, P]),
    "qoc_trotter_free": (None, [P]),
    "qoc_strerror": (C.c_char_p, [C.c_int]),
    "qoc_last_error": (C.c_char_p, []),
    "qoc_version": (C.c_int, []),
}

_lib = None


class QocError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.qoc_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib.qoc_strerror(code).decode()} ({code}): {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load libqoc.so and declare its symbols; raises if the library was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2309_05884_gb300.build` "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int, where: str) -> None:
    if code != QOC_OK:
        raise QocError(code, where)
