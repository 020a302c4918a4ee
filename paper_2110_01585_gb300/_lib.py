"""ctypes binding of libeptv (include/ep_tv.h).

Argument marshalling only: every step of the method runs in the CUDA library.
There is no fallback; if the library is missing or fails to load, importing the
binding raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

OK = 0
STATUS_NAMES = {
    0: "EP_TV_OK", 1: "EP_TV_ERR_ARG", 2: "EP_TV_ERR_NOMEM", 3: "EP_TV_ERR_CUDA",
    4: "EP_TV_ERR_NONFINITE", 5: "EP_TV_ERR_CG_NOCONV", 6: "EP_TV_ERR_TIMEOUT",
    7: "EP_TV_ERR_STATE", 8: "EP_TV_ERR_UNSUPPORTED",
}

OP_IDENTITY, OP_CONV_PERIODIC, OP_DENSE, OP_HADAMARD = 0, 1, 2, 3
PRIOR_L1, PRIOR_MOG2, PRIOR_BG = 0, 1, 2
KERNELS = {0: "prior_sweep", 1: "cg_direction", 2: "cg_update", 3: "cg_residual", 4: "site0",
           5: "cg_precond", 6: "cs_woodbury", 7: "cg_commit", 8: "cs_mma"}

# Every function declared in include/ep_tv.h, with its ctypes signature.
c_void_p, c_int32, c_double, c_size_t = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_size_t


class Operator(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("m", ctypes.c_int32), ("kernel", ctypes.POINTER(ctypes.c_float)),
                ("kh", ctypes.c_int32), ("kw", ctypes.c_int32), ("dense", ctypes.c_void_p),
                ("patterns", ctypes.POINTER(ctypes.c_int32))]


class Block(ctypes.Structure):
    _fields_ = [("global_height", ctypes.c_int32), ("row0", ctypes.c_int32), ("rows", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("xi", ctypes.c_double), ("beta", ctypes.c_double), ("damping", ctypes.c_double),
                ("var_cap", ctypes.c_double), ("periodic", ctypes.c_int32),
                ("order_mode", ctypes.c_int32), ("rbmc_samples", ctypes.c_int32),
                ("cg_max_iter", ctypes.c_int32), ("cg_rtol", ctypes.c_double),
                ("precision", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("prior", ctypes.c_int32), ("omega", ctypes.c_double), ("s1_sq", ctypes.c_double),
                ("s2_sq", ctypes.c_double), ("em_option", ctypes.c_int32)]


SIGNATURES = {
    "ep_tv_default_params": (c_int32, [ctypes.POINTER(Params)]),
    "ep_tv_init": (c_int32, [ctypes.POINTER(Operator), c_void_p, ctypes.POINTER(Params), c_void_p,
                             ctypes.POINTER(c_void_p)]),
    "ep_tv_set_probes": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32]),
    "ep_tv_init_noise": (c_int32, [ctypes.POINTER(Operator), c_void_p, c_void_p, ctypes.POINTER(Params),
                                   c_void_p, ctypes.POINTER(c_void_p)]),
    "ep_tv_init_block": (c_int32, [ctypes.POINTER(Operator), c_void_p, ctypes.POINTER(Params),
                                   ctypes.POINTER(Block), c_void_p, ctypes.POINTER(c_void_p)]),
    "ep_tv_block_halo_out": (c_int32, [c_void_p, c_int32, c_void_p]),
    "ep_tv_block_halo_in": (c_int32, [c_void_p, c_int32, c_void_p]),
    "ep_tv_sweep": (c_int32, [c_void_p, c_int32, ctypes.POINTER(ctypes.c_int8), c_int32]),
    "ep_tv_em_beta": (c_int32, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "ep_tv_set_beta": (c_int32, [c_void_p, c_double]),
    "ep_tv_ep_em": (c_int32, [c_void_p, c_int32, c_int32, c_double, ctypes.POINTER(c_double),
                              ctypes.POINTER(c_int32)]),
    "ep_tv_posterior": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "ep_tv_get_sites": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "ep_tv_status_check": (c_int32, [c_void_p]),
    "ep_tv_stats": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(ctypes.c_uint64),
                              ctypes.POINTER(ctypes.c_uint64)]),
    "ep_tv_solver_report": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                      ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "ep_tv_state_export": (c_int32, [c_void_p, c_void_p, ctypes.POINTER(c_size_t)]),
    "ep_tv_state_import": (c_int32, [c_void_p, c_void_p, c_size_t]),
    "ep_tv_reset": (c_int32, [c_void_p]),
    "ep_tv_solve_host": (c_int32, [ctypes.POINTER(Operator), c_void_p, ctypes.POINTER(Params),
                                   c_int32, c_int32, c_void_p, c_void_p, ctypes.POINTER(c_double)]),
    "ep_tv_trace_enable": (c_int32, [c_void_p, c_int32]),
    "ep_tv_trace_read": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_double),
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(c_double),
                                   ctypes.POINTER(c_double)]),
    "ep_tv_prior_sweep_noalloc": (c_int32, [c_int32, c_int32, ctypes.POINTER(Params), c_void_p,
                                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p, ctypes.POINTER(ctypes.c_int8),
                                            c_void_p, c_void_p, c_void_p]),
    "ep_tv_batch_create": (c_int32, [c_int32, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p)]),
    "ep_tv_batch_sweep": (c_int32, [c_void_p, c_int32, c_int32]),
    "ep_tv_batch_destroy": (None, [c_void_p]),
    "ep_tv_graph_sweeps": (ctypes.c_int64, [c_void_p]),
    "ep_tv_conv3x3_forward": (c_int32, [c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p,
                                        c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "ep_tv_conv3x3_backward_work": (c_size_t, [c_int32, c_int32, c_int32, c_int32, c_int32]),
    "ep_tv_conv3x3_backward": (c_int32, [c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p, c_size_t, c_void_p]),
    "ep_tv_adam_step": (c_int32, [ctypes.c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                  ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                  c_void_p]),
    "ep_tv_warmstart_loss": (c_int32, [c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p, ctypes.c_float, c_void_p, c_void_p,
                                       c_void_p]),
    "ep_tv_warm_start": (c_int32, [c_void_p, c_void_p, c_int32]),
    "ep_tv_tc_gemm_f64": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p]),
    "ep_tv_destroy": (None, [c_void_p]),
    "ep_tv_status_str": (ctypes.c_char_p, [c_int32]),
}


class EPTVError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}")


_LIB = None


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load (and if needed build) libeptv.so; raises if it cannot be loaded."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_needed and not _build.up_to_date():
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libeptv is not built ({path}); run paper_2110_01585_gb300/build.py")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(code: int, where: str):
    if code != OK:
        raise EPTVError(code, where)
