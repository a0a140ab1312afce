"""ctypes binding of libadiwave.so (the C ABI declared in include/adiwave.h).

Argument marshalling only.  Loading fails loudly (RuntimeError) when the
library cannot be built or loaded; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

ADI_OK = 0
ADI_EINVAL = 1
ADI_ENOMEM = 2
ADI_ECUDA = 3
ADI_ENUMERIC = 4
ADI_ETIMEOUT = 5
ADI_ESTATE = 6
ADI_EUNSUPPORTED = 7

ADI_START_PAPER = 0
ADI_START_TAYLOR2 = 1
ADI_FP64_AUTO = 0
ADI_FP64_NEVER = 1
ADI_FP64_ALWAYS = 2

ADI_SOLVER_AUTO = 0
ADI_SOLVER_TREE = 1
ADI_SOLVER_CR_SMEM = 2

ADI_KERNEL_X = 0
ADI_KERNEL_Y = 1
ADI_KERNEL_OTHER = 2
ADI_KERNEL_KINDS = 3

# every symbol include/adiwave.h declares
EXPORTS = (
    "adi_wave_init", "adi_wave_reset", "adi_wave_step", "adi_wave_run", "adi_wave_set_checkpointing",
    "adi_wave_adjoint", "adi_wave_get_state", "adi_wave_set_state", "adi_wave_sync_status",
    "adi_wave_destroy", "adi_wave_strerror", "adi_wave_last_error", "adi_wave_get_tuning",
    "adi_wave_set_tuning", "adi_wave_profile", "adi_wave_profile_read", "adi_wave_launch_count",
    "adi_wave_version", "adi_wave_set_batch_mode", "adi_wave_set_wait_hook",
    "adi_wave_step_noalloc", "adi_wave_set_model",
)


class Desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("lx", ctypes.c_double),
                ("ly", ctypes.c_double), ("dt", ctypes.c_double), ("start", ctypes.c_int32),
                ("fp64_solve", ctypes.c_int32)]


class Source(ctypes.Structure):
    _fields_ = [("ix", ctypes.c_int32), ("iy", ctypes.c_int32), ("wavelet", ctypes.c_void_p),
                ("n_wavelet", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("chunk_x", ctypes.c_int32), ("chunk_y", ctypes.c_int32),
                ("rows_per_cta", ctypes.c_int32), ("cols_per_cta", ctypes.c_int32),
                ("pcr_size", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("solver", ctypes.c_int32), ("cta_threads", ctypes.c_int32),
                ("cta_threads_y", ctypes.c_int32), ("y_stage", ctypes.c_int32),
                ("persist", ctypes.c_int32), ("x_stage", ctypes.c_int32),
                ("x_cluster", ctypes.c_int32)]


class Model(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("g", ctypes.c_void_p), ("n_g", ctypes.c_int32),
                ("f", ctypes.c_void_p), ("n_f", ctypes.c_int32)]


class AdiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libadiwave.so (building it first if needed) and declare signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libadiwave.so is missing (%s); run paper_2006_10142_gb300/build.py"
                               % path)
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        pp = ctypes.POINTER(ctypes.c_void_p)
        lib.adi_wave_init.argtypes = [pp, ctypes.POINTER(Desc), i32, pp, pp, pp,
                                      ctypes.POINTER(Source), P]
        lib.adi_wave_reset.argtypes = [P, pp, pp, pp, ctypes.POINTER(Source), P]
        lib.adi_wave_step.argtypes = [P, ctypes.POINTER(Source), P]
        lib.adi_wave_run.argtypes = [P, i32, ctypes.POINTER(Source), ctypes.POINTER(i32), i32, P, P]
        lib.adi_wave_set_checkpointing.argtypes = [P, i32]
        lib.adi_wave_adjoint.argtypes = [P, P, P, P, i32, P]
        lib.adi_wave_get_state.argtypes = [P, i32, P, P, ctypes.POINTER(i64), P]
        lib.adi_wave_set_state.argtypes = [P, i32, P, P, i64, P]
        lib.adi_wave_sync_status.argtypes = [P, P]
        lib.adi_wave_destroy.argtypes = [P]
        lib.adi_wave_destroy.restype = None
        lib.adi_wave_strerror.argtypes = [ctypes.c_int]
        lib.adi_wave_strerror.restype = ctypes.c_char_p
        lib.adi_wave_last_error.argtypes = [P]
        lib.adi_wave_last_error.restype = ctypes.c_char_p
        lib.adi_wave_get_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
        lib.adi_wave_set_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
        lib.adi_wave_profile.argtypes = [P, i32]
        lib.adi_wave_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(i64), i32]
        lib.adi_wave_launch_count.argtypes = [P]
        lib.adi_wave_launch_count.restype = i64
        lib.adi_wave_version.argtypes = []
        lib.adi_wave_version.restype = ctypes.c_char_p
        lib.adi_wave_set_batch_mode.argtypes = [P, i32]
        lib.adi_wave_set_wait_hook.argtypes = [P, i64, i32]
        lib.adi_wave_set_model.argtypes = [P, ctypes.POINTER(Model)]
        lib.adi_wave_step_noalloc.argtypes = [ctypes.POINTER(Desc), i32, ctypes.c_double, P, P, P,
                                              ctypes.POINTER(Source), i64, P]
        for name in EXPORTS:
            if not hasattr(lib, name):
                raise RuntimeError("libadiwave.so does not export %s" % name)
        _lib = lib
        return lib


def check(rc: int, handle=None, what: str = ""):
    if rc == ADI_OK:
        return
    lib = load()
    msg = lib.adi_wave_strerror(rc).decode()
    detail = lib.adi_wave_last_error(handle if handle else None).decode()
    if detail:
        msg += ": " + detail
    if what:
        msg = what + ": " + msg
    raise AdiError(rc, msg)
