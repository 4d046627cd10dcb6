"""ctypes declarations of the C ABI in include/mg.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmgpcg.so")

MG_OK = 0
STATUS = {
    0: "MG_OK", 1: "MG_ERR_ARG", 2: "MG_ERR_ALLOC", 3: "MG_ERR_CUDA", 4: "MG_ERR_NONFINITE",
    5: "MG_ERR_NOT_CONVERGED", 6: "MG_ERR_BREAKDOWN", 7: "MG_ERR_DEVICE_TIMEOUT", 8: "MG_ERR_NOT_SPD",
}
PRECISION = {"fp64": 0, "mixed_fp32": 1, "mixed_bf16k": 2}
# statuses that report how the iteration ended (the iterate and statistics are valid)
SOLVE_OUTCOMES = (4, 5, 6, 7)

# every symbol include/mg.h declares
EXPORTS = [
    "mg_params_default", "mg_setup", "mg_set_stream", "mg_solve", "mg_solve_adjoint", "mg_free", "mg_last_error",
    "mg_num_levels", "mg_level_dims", "mg_level_interval", "mg_history", "mg_apply", "mg_smooth", "mg_residual_restrict",
    "mg_prolong_add", "mg_coarse_solve", "mg_vcycle", "mg_gradient", "mg_residual_norm", "mg_timing_enable",
    "mg_timing_read", "mg_residual_norm_noalloc", "mg_solve_host", "mg_slab_plan", "mg_slab_transport_sizes",
    "mg_set_transport", "mg_fp64_fma_peak",
]
KERNEL_CLASSES = ["cheb_zero", "cheb_step", "resid", "restrict", "prolong", "bottom", "cg_dir", "cg_upd", "dot",
                  "cast", "cg_apply", "host_gap"]


class MgParams(C.Structure):
    _fields_ = [
        ("levels", C.c_int), ("nu_pre", C.c_int), ("nu_post", C.c_int), ("cheby_degree", C.c_int),
        ("eig_lo_frac", C.c_double), ("eig_hi", C.c_double),
        ("coarse_k_rule", C.c_int), ("face_rule", C.c_int), ("k_is_log", C.c_int), ("precision", C.c_int),
        ("maxit", C.c_int), ("nonzero_guess", C.c_int), ("flexible", C.c_int), ("telescope_max_n", C.c_int),
        ("use_graph", C.c_int), ("stencil_kernel", C.c_int), ("use_pdl", C.c_int),
        ("smoother", C.c_int), ("richardson_omega", C.c_double), ("coarse_op", C.c_int),
        ("krylov", C.c_int), ("gmres_restart", C.c_int), ("eig_mode", C.c_int), ("eig_safety", C.c_double),
        ("coarse_solve", C.c_int), ("coarse_rtol", C.c_double), ("coarse_maxit", C.c_int),
        ("bottom_blocks", C.c_int), ("test_inject", C.c_int), ("slabs", C.c_int), ("slab_level", C.c_int),
        ("slab_rank", C.c_int),
    ]


EXCHANGE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_longlong, C.c_int, C.c_int, C.c_void_p)
ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_void_p)
ALLGATHER_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_longlong, C.c_void_p)


class MgTransport(C.Structure):
    _fields_ = [
        ("ctx", C.c_void_p), ("exchange", EXCHANGE_FN), ("allreduce", ALLREDUCE_FN), ("allgather", ALLGATHER_FN),
        ("send_lo", C.c_void_p), ("send_hi", C.c_void_p), ("recv_lo", C.c_void_p), ("recv_hi", C.c_void_p),
        ("reduce_buf", C.c_void_p), ("gather_send", C.c_void_p), ("gather_recv", C.c_void_p),
    ]


class MgStats(C.Structure):
    _fields_ = [
        ("iters", C.c_int), ("rel_resid", C.c_double), ("true_rel_resid", C.c_double), ("bnorm", C.c_double),
        ("setup_s", C.c_double), ("solve_s", C.c_double), ("kernel_launches", C.c_longlong),
    ]


class MgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


_lib = None


def load():
    """Load the in-tree CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1604_07163_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    P = C.POINTER
    sig = {
        "mg_params_default": ([P(MgParams)], i),
        "mg_setup": ([P(vp), i, i, i, vp, i, P(MgParams), vp], i),
        "mg_set_stream": ([vp, vp], i),
        "mg_solve": ([vp, vp, vp, d, P(MgStats)], i),
        "mg_solve_host": ([vp, vp, vp, d, P(MgStats)], i),
        "mg_slab_plan": ([i, i, i, P(MgParams), P(C.c_int), i, P(C.c_int)], i),
        "mg_slab_transport_sizes": ([vp, P(C.c_longlong), P(C.c_longlong)], i),
        "mg_set_transport": ([vp, P(MgTransport)], i),
        "mg_solve_adjoint": ([vp, vp, vp, d, vp, vp, P(MgStats)], i),
        "mg_free": ([vp], i),
        "mg_last_error": ([vp], C.c_char_p),
        "mg_num_levels": ([vp], i),
        "mg_level_dims": ([vp, i, P(C.c_int)], i),
        "mg_level_interval": ([vp, i, P(C.c_double), P(C.c_double)], i),
        "mg_history": ([vp, P(C.c_double), i], i),
        "mg_apply": ([vp, i, vp, vp], i),
        "mg_smooth": ([vp, i, vp, vp, i], i),
        "mg_residual_restrict": ([vp, i, vp, vp, vp], i),
        "mg_prolong_add": ([vp, i, vp, vp], i),
        "mg_coarse_solve": ([vp, vp, vp], i),
        "mg_vcycle": ([vp, vp, vp], i),
        "mg_gradient": ([vp, vp, vp, vp], i),
        "mg_residual_norm": ([vp, vp, vp, P(C.c_double)], i),
        "mg_timing_enable": ([vp, i, i], i),
        "mg_residual_norm_noalloc": ([vp, vp, vp, vp], i),
        "mg_timing_read": ([vp, i, i, P(C.c_double), P(C.c_longlong), P(C.c_double)], i),
        "mg_fp64_fma_peak": ([i, P(C.c_double)], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib
