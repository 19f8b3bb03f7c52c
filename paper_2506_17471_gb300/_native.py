"""ctypes declarations of the C-ABI in include/feaction.h (argument marshalling only).

The shared library is built in-tree by ``paper_2506_17471_gb300.build`` into
``_build/libfeaction.so``.  Importing this module without that file raises
ImportError: there is no fallback implementation.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfeaction.so")

FE_OK = 0
STATUS_NAMES = {0: "FE_OK", 1: "FE_ERR_INVALID_ARG", 2: "FE_ERR_UNSUPPORTED", 3: "FE_ERR_CUDA",
                4: "FE_ERR_BAD_MESH", 5: "FE_ERR_INDEX", 6: "FE_ERR_TIMEOUT", 7: "FE_ERR_NO_MEMORY",
                8: "FE_ERR_NONFINITE"}
globals().update({name: code for code, name in STATUS_NAMES.items()})

FE_FORM_MASS = 0
FE_FORM_ELASTICITY = 1
FE_FORM_NH_RESIDUAL = 2
FE_FORM_NH_JACOBIAN = 3
FE_FORM_LAPLACE = 4
FE_FORM_HELMHOLTZ = 5
FE_FORM_SVK_RESIDUAL = 6
FE_FORM_SVK_JACOBIAN = 7
FE_PREC_FP64 = 0
FE_PREC_FP32 = 1
FE_PREC_BF16 = 2
FE_PREC_FP16 = 3
FE_PREC_FP16X2 = 4
FE_PREC_TF32 = 5
FE_FLAG_ACCUMULATE = 1
FE_FLAG_COOPERATIVE = 2
FE_FLAG_TABLES_GLOBAL = 4
FE_FLAG_GATHER_SCATTER = 8

# every symbol declared in include/feaction.h
FE_QUAD_CONICAL = 0
FE_QUAD_SYMMETRIC = 1

EXPORTS = ("fe_status_string", "fe_tabulate", "fe_tabulate_scheme", "fe_plan_create", "fe_plan_destroy", "fe_action",
           "fe_action_adjoint", "fe_action_host", "fe_plan_status", "fe_plan_get_info",
           "fe_measure_fp64_peak", "fe_action_noalloc", "fe_cg_start", "fe_cg_direction",
           "fe_cg_update", "fe_cg_new_direction", "fe_vec_axpy", "fe_vec_dot",
           "fe_selftest_conversions", "fe_batch_create", "fe_batch_run", "fe_batch_status",
           "fe_batch_get_info", "fe_batch_destroy", "fe_selftest_conversions16", "fe_round16", "fe_round_tf32", "fe_order_cells_morton", "fe_order_first_touch", "fe_selftest_bounded_wait",
           "fe_action_host_pipelined", "fe_selftest_log_rcp")
FE_LOG_TABLE_DOUBLES = 370
FE_CG_PARTIALS = 1024
FE_CG_WORKSPACE_DOUBLES = FE_CG_PARTIALS + 16


class FeMesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("degree", ctypes.c_int32), ("n_vertices", ctypes.c_int32),
                ("n_cells", ctypes.c_int32), ("n_nodes", ctypes.c_int32),
                ("coords", ctypes.c_void_p), ("cell2vertex", ctypes.c_void_p),
                ("cell2node", ctypes.c_void_p)]


class FeForm(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("quad_degree", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("lambda_", ctypes.c_double), ("mu", ctypes.c_double),
                ("lambda_cell", ctypes.c_void_p), ("mu_cell", ctypes.c_void_p),
                ("u_lin", ctypes.c_void_p), ("tile_cells", ctypes.c_int32),
                ("quad_scheme", ctypes.c_int32)]


class FeBatchProblem(ctypes.Structure):
    _fields_ = [("form", FeForm), ("mesh", FeMesh), ("u", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("kernel", ctypes.c_int32), ("tile_cells", ctypes.c_int32)]


class FeBatchInfo(ctypes.Structure):
    _fields_ = [("problems", ctypes.c_int32), ("items", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int64), ("dofs", ctypes.c_int64),
                ("contraction_flops", ctypes.c_double)]


class FePlanInfo(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_int32), ("n_loc", ctypes.c_int32), ("ncomp", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("n_dofs", ctypes.c_int64),
                ("flops_per_cell", ctypes.c_double), ("bytes_min", ctypes.c_double),
                ("flops_per_cell_dense", ctypes.c_double)]


class FeError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        super().__init__(f"{STATUS_NAMES.get(self.code, self.code)}{': ' + what if what else ''}")


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, Z, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
    lib.fe_status_string.argtypes = [I]
    lib.fe_status_string.restype = ctypes.c_char_p
    lib.fe_tabulate.argtypes = [I, I, I, ctypes.POINTER(I), P, P, P, Z]
    lib.fe_tabulate_scheme.argtypes = [I, I, I, I, ctypes.POINTER(I), P, P, P, Z]
    lib.fe_plan_create.argtypes = [ctypes.POINTER(FeForm), ctypes.POINTER(FeMesh), ctypes.POINTER(P)]
    lib.fe_plan_destroy.argtypes = [P]
    lib.fe_action.argtypes = [P, P, P, P]
    lib.fe_action_adjoint.argtypes = [P, P, P, P, P, P, P]
    lib.fe_action_host.argtypes = [P, P, P, P, P, P]
    lib.fe_action_host_pipelined.argtypes = [P, I, P, P, P, P, P]
    lib.fe_plan_status.argtypes = [P, ctypes.POINTER(I)]
    lib.fe_plan_get_info.argtypes = [P, ctypes.POINTER(FePlanInfo)]
    lib.fe_measure_fp64_peak.argtypes = [P, Z, ctypes.POINTER(D)]
    lib.fe_action_noalloc.argtypes = [ctypes.POINTER(FeForm), ctypes.POINTER(FeMesh), P, P, I, P, P,
                                      ctypes.POINTER(I), P]
    LL = ctypes.c_longlong
    lib.fe_cg_start.argtypes = [LL, P, P, P, P, P, P, P]
    lib.fe_cg_direction.argtypes = [LL, P, P, P, P, P]
    lib.fe_cg_update.argtypes = [LL, P, P, P, P, P, P]
    lib.fe_cg_new_direction.argtypes = [LL, P, P, P, P]
    lib.fe_vec_axpy.argtypes = [LL, D, P, P, P]
    lib.fe_vec_dot.argtypes = [LL, P, P, P, P, I, P]
    lib.fe_selftest_conversions.argtypes = [P, LL, P, P]
    lib.fe_selftest_conversions16.argtypes = [P, LL, P, P]
    lib.fe_round16.argtypes = [P, ctypes.c_size_t, I, P]
    lib.fe_round_tf32.argtypes = [P, ctypes.c_size_t, I, P]
    lib.fe_order_cells_morton.argtypes = [I, I, I, P, P, P]
    lib.fe_order_first_touch.argtypes = [I, I, I, P, P, P]
    lib.fe_selftest_bounded_wait.argtypes = [P, I, P]
    lib.fe_batch_create.argtypes = [ctypes.POINTER(FeBatchProblem), I, ctypes.POINTER(P)]
    lib.fe_batch_run.argtypes = [P, P]
    lib.fe_batch_status.argtypes = [P, ctypes.POINTER(I)]
    lib.fe_batch_get_info.argtypes = [P, ctypes.POINTER(FeBatchInfo)]
    lib.fe_batch_destroy.argtypes = [P]
    for name in EXPORTS:
        if name != "fe_status_string":
            getattr(lib, name).restype = I
    return lib


lib = _load()


def check(code: int, what: str = "") -> None:
    if code != FE_OK:
        raise FeError(code, what)
