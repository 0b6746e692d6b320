"""ctypes declarations of the C ABI in include/blp.h (argument marshalling only).

Every computation happens in libblp.so.  If the library is missing this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libblp.so")

BLP_OK, BLP_ERR_ARG, BLP_ERR_COEF, BLP_ERR_NOCONV, BLP_ERR_TIMEOUT, BLP_ERR_CUDA, BLP_ERR_MEM = range(7)
BLP_FP64, BLP_MIXED = 0, 1
BLP_STOP_SCALED, BLP_STOP_REL2, BLP_STOP_ABS2 = 0, 1, 2
BLP_NOALLOC_MAX_N = 8192
BLP_MESH_SHISHKIN, BLP_MESH_GRADED, BLP_MESH_PARABOLIC = 0, 1, 2
BLP_1D_MAX_N, BLP_1D_MAXIT = 65536, 128

c_int, c_double, c_void_p, c_ll = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong
_DP = ctypes.POINTER(ctypes.c_double)


class Params(ctypes.Structure):
    _fields_ = [("eps", c_double), ("N", c_int), ("sigma", c_double), ("beta_x", c_double), ("beta_y", c_double),
                ("restart", c_int), ("maxit", c_int), ("precision", c_int), ("stop_mode", c_int),
                ("corner_reduction", c_double), ("corner_max_cycles", c_int), ("corner_fixed_cycles", c_int),
                ("check_coefficients", c_int), ("mesh", c_int), ("layer_intervals", c_int), ("device_driven", c_int)]


class Info(ctypes.Structure):
    _fields_ = [("status", c_int), ("iters", c_int), ("restarts", c_int), ("corner_cycles_max", c_int),
                ("relres", c_double), ("relres_unscaled", c_double), ("t_solve_ms", c_double),
                ("t_setup_ms", c_double), ("device_driven", c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchItem(ctypes.Structure):
    _fields_ = [("params", Params), ("c1", c_void_p), ("c2", c_void_p), ("r", c_void_p), ("f", c_void_p),
                ("u", c_void_p), ("tol", c_double), ("info", Info), ("status", c_int)]


class Problem1D(ctypes.Structure):
    _fields_ = [("N", c_int), ("eps", c_double), ("c_low", c_double), ("sigma", c_double), ("c", c_void_p),
                ("r", c_void_p), ("f", c_void_p), ("u", c_void_p), ("stop", c_double), ("maxit", c_int),
                ("iters", c_int), ("resid", c_double), ("status", c_int)]


class Tuning(ctypes.Structure):
    _fields_ = [("dts_chunk", c_int), ("dts_cluster", c_int), ("two_step", c_int), ("precond_ms", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# exported symbol -> (restype, argtypes); the ABI test checks this against include/blp.h
SIGNATURES = {
    "blp_params_default": (None, [ctypes.POINTER(Params)]),
    "blp_mesh": (c_double, [c_int, c_double, c_double, c_double, _DP]),
    "blp_mesh_graded": (c_double, [c_int, c_double, c_double, c_double, _DP]),
    "blp_mesh_parabolic": (c_double, [c_int, c_double, c_double, _DP]),
    "blp_mesh_q": (c_double, [c_int, c_int, c_double, c_double, c_double, _DP]),
    "blp_setup": (c_int, [ctypes.POINTER(Params), c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_void_p)]),
    "blp_set_stream": (c_int, [c_void_p, c_void_p]),
    "blp_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, ctypes.POINTER(Info)]),
    "blp_solve_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_double, ctypes.POINTER(Info)]),
    "blp_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "blp_apply_operator": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "blp_precond_apply": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, ctypes.POINTER(c_int)]),
    "blp_destroy": (None, [c_void_p]),
    "blp_strerror": (ctypes.c_char_p, [c_int]),
    "blp_kernel_launches": (c_ll, [c_void_p]),
    "blp_profile": (c_int, [c_void_p, c_int]),
    "blp_profile_read": (c_int, [c_void_p, c_int, ctypes.POINTER(c_ll), ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "blp_profile_chain_steps": (c_int, [c_void_p, c_int, _DP]),
    "blp_kernel_class_count": (c_int, []),
    "blp_kernel_class_name": (ctypes.c_char_p, [c_int]),
    "blp_check_wait_timeout": (c_int, [c_void_p]),
    "blp_solve_batched": (c_int, [ctypes.POINTER(BatchItem), c_int, c_int]),
    "blp_solve_batched_tuned": (c_int, [ctypes.POINTER(BatchItem), c_int, c_int]),
    "blp_solve_1d_batched": (c_int, [ctypes.POINTER(Problem1D), c_int, c_void_p]),
    "blp_get_tuning": (c_int, [c_void_p, ctypes.POINTER(Tuning)]),
    "blp_set_tuning": (c_int, [c_void_p, ctypes.POINTER(Tuning)]),
    "blp_autotune": (c_int, [c_void_p, c_int, c_int, ctypes.POINTER(Tuning)]),
    "blp_residual_noalloc": (c_int, [c_int, c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_void_p]),
    # host-side layout inspection (no GPU needed)
    "blp_layout_npad": (c_ll, [c_int]),
    "blp_layout_addr": (c_ll, [c_int, c_int, c_int]),
    "blp_layout_node": (c_int, [c_int, c_ll, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
}

_lib = None


def load():
    """Load libblp.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    try:
        _build.build()
    except Exception as exc:  # no toolkit: only a prebuilt library will do
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libblp.so is not built and cannot be built here: {exc}") from exc
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class BlpError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = load().blp_strerror(status).decode()
        super().__init__(f"{what}: {msg} (status {status})" if what else f"{msg} (status {status})")


def check(status, what=""):
    if status != BLP_OK:
        raise BlpError(status, what)
    return status
