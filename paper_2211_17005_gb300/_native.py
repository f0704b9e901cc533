"""ctypes binding of the C ABI declared in include/cva.h (argument marshalling only).

Every function here forwards to ``_build/libcva.so``. If the library is missing
the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

CVA_OK, CVA_EINVAL, CVA_ENOMEM, CVA_ECUDA, CVA_ETIMEOUT, CVA_ENOTSUP, CVA_ENUMERIC = range(7)
STATUS_NAMES = {0: "CVA_OK", 1: "CVA_EINVAL", 2: "CVA_ENOMEM", 3: "CVA_ECUDA", 4: "CVA_ETIMEOUT",
                5: "CVA_ENOTSUP", 6: "CVA_ENUMERIC"}
KEEP_DEFAULTS, KEEP_EXPOSURES, PROFILE, GENERIC_KERNELS = 1, 2, 4, 8
VIEW_FEATURES, VIEW_TARGETS, VIEW_DISCOUNT, VIEW_THRESHOLD, VIEW_EXPOSURE, VIEW_MTM, VIEW_DEFAULTS = range(7)
BASIS_LINEAR, BASIS_POLY2 = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_fp = ctypes.POINTER(ctypes.c_float)


class ModelDesc(ctypes.Structure):
    _fields_ = [("E", ctypes.c_int), ("C", ctypes.c_int)] + [
        (n, _dp) for n in ("hw_a", "hw_sigma", "curve", "fx_vol", "fx0", "cir_kappa", "cir_theta",
                           "cir_nu", "gamma0", "recovery", "corr")]


class PortfolioDesc(ctypes.Structure):
    _fields_ = [("n_swaps", ctypes.c_int), ("ccy", _ip), ("cpty", _ip), ("omega", _ip),
                ("n_periods", _ip), ("notional", _dp), ("delta", ctypes.c_double), ("fixed_rate", _dp)]


class GridDesc(ctypes.Structure):
    _fields_ = [("horizon", ctypes.c_double), ("n_steps", ctypes.c_int), ("substeps", ctypes.c_int)]


# name -> (restype, argtypes)
SIGNATURES = {
    "cva_sim_create": (ctypes.c_int, [ctypes.POINTER(ModelDesc), ctypes.POINTER(PortfolioDesc), ctypes.c_int,
                                      ctypes.POINTER(GridDesc), ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)]),
    "cva_simulate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]),
    "cva_simulate_twin": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                         ctypes.c_uint32, ctypes.c_void_p]),
    "cva_twin_l2": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, _dp,
                                   ctypes.c_void_p]),
    "cva_nested_reference": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "cva_relative_rmse": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, _dp, ctypes.c_void_p]),
    "cva_oversim_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, _dp,
                                         ctypes.c_void_p]),
    "cva_oversim_choice": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]),
    "cva_inner_cost_ratio": (ctypes.c_int, [ctypes.c_double, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint32,
                                            _dp]),
    "cva_sim_view": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.POINTER(ctypes.c_size_t)]),
    "cva_sim_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "cva_sim_kernel_ms": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "cva_sim_destroy": (None, [ctypes.c_void_p]),
    "cva_cva0": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, _dp, ctypes.c_void_p]),
    "cva_regress": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                   ctypes.c_int, ctypes.c_void_p, _dp, ctypes.c_void_p]),
    "cva_regress_partial": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                           ctypes.c_int, ctypes.c_void_p, _dp, ctypes.c_void_p]),
    "cva_regress_solve": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp,
                                         ctypes.POINTER(ctypes.c_int)]),
    "cva_regress_predict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                           ctypes.c_void_p, _dp, ctypes.c_void_p, ctypes.c_void_p]),
    "cva_cva0_partials": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, _dp, ctypes.c_void_p]),
    "cva_cva0_combine": (ctypes.c_int, [_dp, ctypes.c_int, _dp]),
    "cva_regress_all": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, _dp,
                                       ctypes.c_void_p]),
    "cva_regress_portfolios": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, _dp, ctypes.c_void_p]),
    "cva_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t,
                                    ctypes.c_void_p]),
    "cva_regress_alive": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, _dp,
                                         ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "cva_set_tiles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int]),
    "cva_grad_cva0": (ctypes.c_int, [ctypes.POINTER(ModelDesc), ctypes.POINTER(PortfolioDesc),
                                     ctypes.POINTER(GridDesc), ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_void_p]),
    "cva_grad_num_params": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "cva_par_rates": (ctypes.c_int, [ctypes.POINTER(ModelDesc), ctypes.POINTER(PortfolioDesc), _dp]),
    "cva_mlp_fit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p]),
    "cva_mlp_num_params": (ctypes.c_int, [ctypes.c_int]),
    "cva_mlp_set_wait_limit": (ctypes.c_int, [ctypes.c_uint32]),
    "cva_mlp_kernel_timing": (ctypes.c_int, [ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_uint64)]),
    "cva_mlp_plan": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]),
    "cva_mlp_first_gradient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                              ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p]),
    "cva_mlp_regress_all": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cva_regress_batched_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, _dp,
                                                  ctypes.c_void_p]),
    "cva_philox4x32_10": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_void_p]),
    "cva_pipe_peaks": (ctypes.c_int, [_dp, ctypes.c_void_p]),
    "cva_last_error": (ctypes.c_char_p, []),
    "cva_version": (ctypes.c_char_p, []),
}


class CvaError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn} -> {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.SO


def lib(build_if_missing: bool = False):
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.SO
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"CUDA library {path} is missing: run "
                                       "`python -c 'import __graft_entry__ as g; g.build()'`")
                _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int, fn: str):
    if status != CVA_OK:
        raise CvaError(status, fn, lib().cva_last_error().decode())
