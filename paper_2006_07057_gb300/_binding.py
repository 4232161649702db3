"""ctypes view of libsinkhorn_pf.so: struct layouts and raw entry points.

Argument marshalling only: every computation runs in the CUDA library. The
library is built in-tree on first use; if it cannot be built or loaded, the
import fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import build as _build

c_void_p = ctypes.c_void_p
c_int = ctypes.c_int
c_int64 = ctypes.c_int64
c_double = ctypes.c_double
c_size_t = ctypes.c_size_t

LSF_OK = 0
LSF_ERR_ARG = 1
LSF_ERR_NONFINITE = 2
LSF_ERR_TIMEOUT = 4
LSF_ERR_WORKSPACE = 8
LSF_ERR_CUDA = 16
LSF_ERR_UNSUPPORTED = 32

LSF_MODE_STORED = 0
LSF_MODE_RECOMPUTE = 1
LSF_MODE_LOG = 2
LSF_MODE_HYBRID = 3
LSF_MODE_AUTO = 4
LSF_AUTO_SPREAD = 4000.0

LSF_KERNEL_PASS = 0
LSF_KERNEL_PASS_RECOMPUTE = 1
LSF_KERNEL_FEATURES = 2
LSF_KERNEL_OTHER = 3
LSF_KERNEL_PASS_LOG = 4
LSF_KERNEL_BATCHED = 5
LSF_KERNEL_ADJOINT = 6
LSF_KERNEL_SMALL = 7
LSF_KERNEL_PASS_MULTI = 8
LSF_KERNEL_PASS_HYBRID = 9


class LsfTheta(ctypes.Structure):
    _fields_ = [("U", c_void_p), ("c", c_void_p), ("r", c_int), ("ldr", c_int), ("d", c_int),
                ("eps", c_double)]


class LsfArccos(ctypes.Structure):
    _fields_ = [("U", c_void_p), ("c", c_void_p), ("r", c_int), ("ldr", c_int), ("d", c_int),
                ("s", c_int), ("kappa", c_double)]


class LsfCloud(ctypes.Structure):
    _fields_ = [("X", c_void_p), ("F", c_void_p), ("shift", c_void_p), ("w", c_void_p),
                ("n", c_int64)]


class LsfScalings(ctypes.Structure):
    _fields_ = [("u", c_void_p), ("v", c_void_p), ("t_u", c_void_p), ("t_v", c_void_p)]


class LsfResult(ctypes.Structure):
    _fields_ = [("W", c_double), ("residual", c_double), ("log_scale", c_double),
                ("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


RESULT_BYTES = ctypes.sizeof(LsfResult)


class LsfPipeline(ctypes.Structure):
    _fields_ = [("n", c_int64), ("m", c_int64), ("d", c_int), ("r", c_int), ("ldr", c_int),
                ("eps", c_double), ("iters", c_int), ("debiased", c_int), ("mode", c_int)]


class LsfPipelineOut(ctypes.Structure):
    _fields_ = [("W", c_double), ("W_xy", c_double), ("W_xx", c_double), ("W_yy", c_double),
                ("residual_xy", c_double), ("residual_xx", c_double), ("residual_yy", c_double),
                ("R", c_double), ("q", c_double), ("sigma", c_double), ("status", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("iters", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class LsfPipelineViews(ctypes.Structure):
    _fields_ = [("theta", LsfTheta), ("x", LsfCloud), ("y", LsfCloud), ("s", LsfScalings * 3),
                ("result", c_void_p)]


class LsfBatchProblem(ctypes.Structure):
    _fields_ = [("Fx", c_void_p), ("Fy", c_void_p), ("shift_x", c_void_p), ("shift_y", c_void_p),
                ("a", c_void_p), ("b", c_void_p), ("n", c_int64), ("m", c_int64),
                ("eps", c_double), ("u", c_void_p), ("v", c_void_p), ("t_u", c_void_p),
                ("t_v", c_void_p), ("result", c_void_p)]


class LsfBatchInfo(ctypes.Structure):
    _fields_ = [("count", c_int), ("ldr", c_int), ("mode", c_int), ("tile_rows", c_int), ("stages", c_int),
                ("grid", c_int), ("tiles_x", c_int64), ("tiles_y", c_int64), ("rows_x", c_int64),
                ("rows_y", c_int64), ("plan_bytes", c_size_t), ("smem_bytes", c_size_t),
                ("strategy", c_int)]

class LsfMultiCloud(ctypes.Structure):
    _fields_ = [("F2", c_void_p), ("shift", c_void_p), ("W", c_void_p), ("n", c_int64)]


class LsfMultiScalings(ctypes.Structure):
    _fields_ = [("U", c_void_p), ("V", c_void_p), ("Tu", c_void_p), ("Tv", c_void_p)]


class LsfAccelInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("attempts", ctypes.c_int32), ("A", c_double),
                ("L", c_double)]


_P = ctypes.POINTER
_SIGNATURES = {
    "lsf_version": (c_int, []),
    "lsf_last_error": (ctypes.c_char_p, []),
    "lsf_gaussian_params": (c_int, [c_double, c_double, c_int, _P(c_double), _P(c_double)]),
    "lsf_radius": (c_int, [c_void_p, c_int64, c_void_p, c_int64, c_int, c_void_p, c_void_p]),
    "lsf_anchors": (c_int, [c_void_p, c_int, c_int, c_double, c_double, c_double, c_void_p,
                            c_void_p, c_void_p]),
    "lsf_arccos_anchors": (c_int, [c_void_p, c_int, c_int, c_double, c_void_p, c_void_p, c_void_p]),
    "lsf_arccos_features": (c_int, [c_void_p, c_int64, _P(LsfArccos), c_void_p, c_void_p, c_void_p,
                                    c_void_p]),
    "lsf_arccos_log_features": (c_int, [c_void_p, c_int64, _P(LsfArccos), c_void_p, c_void_p,
                                        c_void_p, c_void_p]),
    "lsf_features": (c_int, [c_void_p, c_int64, _P(LsfTheta), c_void_p, c_void_p, c_void_p,
                             c_void_p]),
    "lsf_row_shift": (c_int, [c_void_p, c_int64, _P(LsfTheta), c_void_p, c_void_p, c_void_p]),
    "lsf_log_features": (c_int, [c_void_p, c_int64, _P(LsfTheta), c_void_p, c_void_p, c_void_p,
                                 c_void_p]),
    "lsf_hybrid_columns": (c_int, [c_int, _P(c_int)]),
    "lsf_hybrid_features": (c_int, [c_void_p, c_int64, _P(LsfTheta), c_void_p, c_void_p, c_void_p,
                                    c_void_p]),
    "lsf_workspace_bytes": (c_int, [c_int, _P(c_size_t)]),
    "lsf_pipeline_bytes": (c_int, [_P(LsfPipeline), _P(c_size_t)]),
    "lsf_pipeline_run": (c_int, [_P(LsfPipeline), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 c_void_p, c_size_t, _P(LsfPipelineOut), c_void_p]),
    "lsf_pipeline_layout": (c_int, [_P(LsfPipeline), c_void_p, _P(LsfPipelineViews)]),
    "lsf_pipeline_finish": (c_int, [_P(LsfPipeline), c_void_p, _P(LsfPipelineOut), c_void_p]),
    "lsf_accel_workspace_bytes": (c_int, [c_int64, c_int64, c_int, _P(c_size_t)]),
    "lsf_solve_accelerated": (c_int, [_P(LsfTheta), _P(LsfCloud), _P(LsfCloud), c_int, c_double,
                                      _P(LsfScalings), c_void_p, _P(LsfAccelInfo), c_void_p,
                                      c_size_t, c_void_p]),
    "lsf_split_features": (c_int, [c_void_p, c_int64, c_int, c_int, c_void_p, c_int, c_void_p]),
    "lsf_multi_workspace_bytes": (c_int, [c_int, c_int, _P(c_size_t)]),
    "lsf_set_multi_tuning": (c_int, [c_int, c_int, c_int]),
    "lsf_solve_multi": (c_int, [_P(LsfTheta), c_int, _P(LsfMultiCloud), _P(LsfMultiCloud), c_int,
                                c_int, _P(LsfMultiScalings), c_void_p, c_void_p, c_size_t,
                                c_void_p]),
    "lsf_multi_debiased": (c_int, [_P(LsfTheta), c_int, _P(LsfMultiCloud), _P(LsfMultiCloud), c_int,
                                   c_int, _P(LsfMultiScalings), _P(LsfMultiScalings),
                                   _P(LsfMultiScalings), c_void_p, c_void_p, c_void_p, c_size_t,
                                   c_void_p]),
    "lsf_solve": (c_int, [_P(LsfTheta), _P(LsfCloud), _P(LsfCloud), c_int, c_int,
                          _P(LsfScalings), c_void_p, c_void_p, c_size_t, c_void_p]),
    "lsf_divergence": (c_int, [_P(LsfTheta), c_int, _P(_P(LsfCloud)), _P(_P(LsfCloud)),
                               _P(_P(LsfScalings)), _P(c_void_p), _P(c_double), c_void_p,
                               c_int, c_void_p, c_size_t, c_void_p]),
    "lsf_solve_noalloc": (c_int, [_P(LsfTheta), _P(LsfCloud), _P(LsfCloud), c_int, c_int,
                                  _P(LsfScalings), c_void_p, c_void_p]),
    "lsf_debiased": (c_int, [_P(LsfTheta), _P(LsfCloud), _P(LsfCloud), c_int, c_int,
                             _P(LsfScalings), _P(LsfScalings), _P(LsfScalings), c_void_p,
                             c_void_p, c_void_p, c_size_t, c_void_p]),
    "lsf_solve_tol": (c_int, [_P(LsfTheta), _P(LsfCloud), _P(LsfCloud), c_int, c_double, c_int,
                              c_int, _P(LsfScalings), c_void_p, c_void_p, c_size_t, c_void_p]),
    "lsf_debiased_tol": (c_int, [_P(LsfTheta), _P(LsfCloud), _P(LsfCloud), c_int, c_double, c_int,
                                 c_int, _P(LsfScalings), _P(LsfScalings), _P(LsfScalings),
                                 c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "lsf_gradient": (c_int, [_P(LsfTheta), _P(LsfCloud), _P(LsfCloud), _P(LsfScalings),
                             _P(LsfScalings), _P(LsfScalings), c_void_p, c_int, c_int,
                             c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lsf_anchor_gradient": (c_int, [_P(LsfTheta), c_double, _P(LsfCloud), _P(LsfCloud),
                                    _P(LsfScalings), _P(LsfScalings), _P(LsfScalings), c_int,
                                    c_int, c_double, c_void_p, c_void_p, c_size_t, c_void_p]),
    "lsf_batch_plan": (c_int, [_P(LsfBatchProblem), c_int, c_int, c_int, c_int, _P(LsfBatchInfo),
                               c_void_p, c_size_t, c_void_p]),
    "lsf_solve_batched": (c_int, [_P(LsfBatchInfo), c_void_p, c_int, c_void_p]),
    "lsf_set_batch_strategy": (c_int, [c_int]),
    "lsf_set_batch_fault": (c_int, [ctypes.c_ulonglong, c_int]),
    "lsf_set_pass_tiling": (c_int, [c_int, c_int]),
    "lsf_set_small_solver": (c_int, [c_int, ctypes.c_int64]),
    "lsf_get_pass_tiling": (c_int, [_P(c_int), _P(c_int)]),
    "lsf_profile_enable": (c_int, [c_int]),
    "lsf_set_tracing": (c_int, [c_int, c_void_p]),
    "lsf_profile_read": (c_int, [c_int, _P(c_double), _P(c_int64), _P(c_double)]),
    "lsf_probe_pipe_rates": (c_int, [_P(c_double), _P(c_double), _P(c_double), c_void_p]),
    "lsf_launch_count": (c_int64, []),
    "lsf_launch_count_reset": (None, []),
}

_lock = threading.Lock()
_lib = None


def header_symbols() -> list[str]:
    """Names of every function the public header declares."""
    path = os.path.join(_build.INCLUDE, "sinkhorn_pf.h")
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lsf_[a-z0-9_]+)\s*\(", text)))


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libsinkhorn_pf.so missing at {path}")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


class LsfError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != LSF_OK:
        msg = lib().lsf_last_error().decode(errors="replace")
        raise LsfError(status, where, msg)
