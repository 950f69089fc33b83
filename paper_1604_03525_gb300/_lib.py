"""ctypes binding of the C ABI declared in include/epw.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double

EPW_OK = 0
STATUS_NAMES = {
    0: "EPW_OK", 1: "EPW_ERR_INVALID_ARG", 2: "EPW_ERR_CUDA", 3: "EPW_ERR_OOM",
    4: "EPW_ERR_NOT_CONVERGED", 5: "EPW_ERR_TIMEOUT", 6: "EPW_ERR_UNSUPPORTED",
}

# Every symbol include/epw.h declares, with (restype, argtypes).
SIGNATURES = {
    "epw_load_wannier": (I, [P, P]),
    "epw_free_model": (None, [P]),
    "epw_set_vertex": (I, [P, P, I, P]),
    "epw_reserve": (I, [P, I, I, I]),
    "epw_plan_linewidth": (I, [I, I, I, I, I, I, I, I, I, I, I, P, P]),
    "epw_interp_g": (I, [P, I, P, I, P, I, D, P, P, P, P, P]),
    "epw_linewidth": (I, [P, I, P, I, P, P, P, P, P]),
    "epw_linewidth_backward": (I, [P, I, P, I, P, P, P, P, P, P, P, P]),
    "epw_linewidth_noalloc": (I, [P, I, P, I, P, P, P, P, P]),
    "epw_phonon_selfenergy": (I, [P, I, P, P, I, P, P, P, P, P, P, P]),
    "epw_eliashberg": (I, [I, I, P, P, P, I, P, D, P, P]),
    "epw_selfenergy": (I, [P, I, P, I, P, P, P, D, I, P, P, P, P]),
    "epw_batch_create": (I, [I, P, P]),
    "epw_batch_run": (I, [P, P]),
    "epw_batch_info": (I, [P, P, P, P]),
    "epw_batch_free": (None, [P]),
    "epw_linewidth_batched": (I, [I, P, P]),
    "epw_set_polar": (I, [P, P]),
    "epw_selftest_wait_timeout": (I, [ctypes.c_longlong, P]),
    "epw_sync": (I, [P, P]),
    "epw_model_info": (I, [P, P, P, P, P, P]),
    "epw_launch_count": (ctypes.c_uint64, []),
    "epw_timing_enable": (I, [P, I]),
    "epw_timing_read": (I, [P, P, P]),
    "epw_timing_read_tags": (I, [P, P, P]),
    "epw_last_error": (ctypes.c_char_p, []),
    "epw_abi_version": (I, []),
}


class WannierDesc(ctypes.Structure):
    _fields_ = [
        ("nw", I), ("nat", I), ("mass", P),
        ("nRe", I), ("Re", P), ("wRe", P), ("H", P),
        ("nRph", I), ("Rph", P), ("wRph", P), ("Phi", P),
        ("nRp", I), ("Rp", P), ("wRp", P), ("g", P), ("g_is_c64", I),
    ]


class Params(ctypes.Structure):
    _fields_ = [("T_K", D), ("EF_eV", D), ("sigma_eV", D), ("omega_min_eV", D),
                ("precision", I), ("reserved", I)]


class PolarDesc(ctypes.Structure):
    _fields_ = [("A", D * 9), ("eps_inf", D * 9), ("Zstar", P), ("alpha", D), ("prefactor", D), ("gmax", I)]


class LinewidthJob(ctypes.Structure):
    _fields_ = [("model", P), ("nk", I), ("nq", I), ("k", P), ("q", P), ("wq", P),
                ("params", Params), ("imsigma", P)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libepw.so (building it first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path}")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib
