"""ctypes declarations of the C ABI in include/hasf.h (argument marshalling only).

The shared library is built in-tree by ``paper_1603_09337_gb300.build`` into
``_build/libhasf.so``.  Loading fails loudly when it is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhasf.so")

HASF_OK, HASF_EINVAL, HASF_ENOMEM, HASF_EBUDGET, HASF_EPENDING = 0, 1, 2, 3, 4
HASF_ETIMEOUT, HASF_ECUDA, HASF_ENOTFOUND, HASF_ECANCELLED = 5, 6, 7, 8
HASF_EUNSTABLE = 9
RMAX_STABLE = -64   # rmax < 0: run to stability, at most -rmax steps

OPT_FORCE_GANG, OPT_GANG_CTAS, OPT_ROUND_CAP, OPT_SERVE_STREAMS, OPT_SERVE_BATCH = 1, 2, 3, 4, 5
OPT_STATS = 6
OPT_GENERIC_ONLY = 7
OPT_TILES = 8
OPT_HOST_MAPPED = 9
OPT_WAIT_DEADLINE_MS = 10
OPT_FAULT_GANG_SKIP = 11
OPT_FAULT_ALLOC = 12
OPT_ROW_GROUP = 13
OPT_SIMPLE3_TABLE = 14
STAT_NAMES = ("word_tests", "ring_evals", "passes", "levels", "rounds", "launches")

OP_THIN, OP_THICK, OP_HC, OP_HF = 1, 2, 3, 4

# Every symbol include/hasf.h declares.
EXPORTS = (
    "hasf_create", "hasf_destroy", "hasf_smooth", "hasf_smooth_batch", "hasf_status_of",
    "hasf_smooth_host", "hasf_submit", "hasf_poll", "hasf_cancel", "hasf_drain",
    "hasf_set_option", "hasf_strerror", "hasf_edt", "hasf_operator", "hasf_simple_table",
    "hasf_simple3_table", "hasf_levels", "hasf_read_stats", "hasf_smooth_noalloc", "hasf_graph_create",
    "hasf_graph_launch", "hasf_graph_destroy", "hasf_autotune", "hasf_tuning_save",
    "hasf_tuning_load", "hasf_tuning_get", "hasf_smooth3d",
)


class HasfImage(ctypes.Structure):
    _fields_ = [
        ("in_", ctypes.c_void_p),
        ("out", ctypes.c_void_p),
        ("C", ctypes.c_void_p),
        ("D", ctypes.c_void_p),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("pitch", ctypes.c_int32),
        ("rmax", ctypes.c_int32),
        ("connectivity", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class HasfVolume(ctypes.Structure):
    _fields_ = [
        ("in_", ctypes.c_void_p),
        ("out", ctypes.c_void_p),
        ("C", ctypes.c_void_p),
        ("D", ctypes.c_void_p),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("depth", ctypes.c_int32),
        ("rmax", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 2),
    ]


class HasfError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} (status {code})")


_lock = threading.Lock()
_lib = None


def _declare(lib):
    vp, ci, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
    img_p = ctypes.POINTER(HasfImage)
    lib.hasf_create.argtypes = [ctypes.POINTER(vp), ci, ctypes.c_size_t]
    lib.hasf_destroy.argtypes = [vp]
    lib.hasf_smooth.argtypes = [vp, img_p, vp]
    lib.hasf_smooth_batch.argtypes = [vp, img_p, ci, vp]
    lib.hasf_status_of.argtypes = [vp, vp]
    lib.hasf_smooth_host.argtypes = [vp, img_p, ci]
    lib.hasf_submit.argtypes = [vp, img_p, ctypes.POINTER(u64)]
    lib.hasf_poll.argtypes = [vp, u64, ctypes.POINTER(ci), ctypes.POINTER(ci)]
    lib.hasf_cancel.argtypes = [vp, u64]
    lib.hasf_drain.argtypes = [vp]
    lib.hasf_set_option.argtypes = [vp, ci, ctypes.c_int64]
    lib.hasf_strerror.argtypes = [ci]
    lib.hasf_strerror.restype = ctypes.c_char_p
    lib.hasf_edt.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                             ctypes.c_int32, vp, vp]
    lib.hasf_operator.argtypes = [vp, ci, img_p, vp]
    lib.hasf_simple_table.argtypes = [vp, ctypes.c_int32, vp]
    lib.hasf_simple3_table.argtypes = [vp, vp, vp]
    lib.hasf_levels.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_int32, vp, vp]
    lib.hasf_read_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ci]
    lib.hasf_smooth_noalloc.argtypes = [img_p, vp, vp]
    lib.hasf_graph_create.argtypes = [vp, img_p, ci, ctypes.POINTER(vp)]
    lib.hasf_graph_launch.argtypes = [vp, vp]
    lib.hasf_graph_destroy.argtypes = [vp]
    i32 = ctypes.c_int32
    lib.hasf_autotune.argtypes = [vp, i32, i32, i32, i32, ctypes.POINTER(i32)]
    lib.hasf_tuning_save.argtypes = [vp, ctypes.c_char_p]
    lib.hasf_tuning_load.argtypes = [vp, ctypes.c_char_p]
    lib.hasf_tuning_get.argtypes = [vp, i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.hasf_smooth3d.argtypes = [vp, ctypes.POINTER(HasfVolume), ci, vp]
    for name in EXPORTS:
        if name != "hasf_strerror":
            getattr(lib, name).restype = ci


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    f"HASF CUDA library not found at {p}; build it with "
                    "`python -m paper_1603_09337_gb300.build` (nvcc, sm_103a)")
            lib = ctypes.CDLL(p)
            _declare(lib)
            _lib = lib
    return _lib


def strerror(code: int) -> str:
    try:
        return load().hasf_strerror(code).decode()
    except Exception:  # the library may be the thing that is missing
        return f"status {code}"


def check(code: int, what: str):
    if code != HASF_OK:
        raise HasfError(code, what)
