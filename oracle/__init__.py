"""CPU oracle for the homotopic alternating sequential filter (HASF).

TEST INFRASTRUCTURE ONLY.  The plain single-threaded C programs in
``hasf_oracle.c`` and ``hasf3d_oracle.c`` restate what the method of Mahmoudi & Akil (arXiv
1603.09337) computes; this module compiles it with gcc and wraps it with
ctypes and numpy.  Only the test suite, the smoke check and the CPU-baseline
leg of the benchmark may import it.  The CUDA library never does, and the two
share no code.

Every 2D wrapper takes and returns numpy arrays of shape (h, w); the 3D ones
(``*3d``, in ``hasf3d_oracle.c``) arrays of shape (d, h, w).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "hasf_oracle.c"), os.path.join(_HERE, "hasf3d_oracle.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libhasf_oracle.so")

INF = 1 << 62  # "no feature" distance, as returned by edt()

_lock = threading.Lock()
_lib = None


class Stats(ctypes.Structure):
    """Work counters of the sweeps (levels, rounds, changed points)."""

    _fields_ = [
        ("levels", ctypes.c_int64),
        ("rounds", ctypes.c_int64),
        ("changes", ctypes.c_int64),
        ("max_rounds_per_level", ctypes.c_int64),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libhasf_oracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(f) for f in _SRCS))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-Wextra",
                        "-o", tmp, *_SRCS], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load():
    """Return the ctypes handle of the oracle library, building it if needed."""
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i64p = ctypes.POINTER(ctypes.c_int64)
            sp = ctypes.POINTER(Stats)
            ci = ctypes.c_int
            lib.hasf_oracle_simple_lut.argtypes = [ci, u8p]
            lib.hasf_oracle_edt.argtypes = [u8p, ci, ci, ci, i64p]
            lib.hasf_oracle_dilate.argtypes = [u8p, ci, ci, ci, u8p]
            lib.hasf_oracle_erode.argtypes = [u8p, ci, ci, ci, u8p]
            lib.hasf_oracle_thin.argtypes = [u8p, u8p, i64p, ci, ci, ci, sp]
            lib.hasf_oracle_thicken.argtypes = [u8p, u8p, i64p, ci, ci, ci, sp]
            lib.hasf_oracle_hc.argtypes = [u8p, u8p, ci, ci, ci, ci, sp]
            lib.hasf_oracle_hf.argtypes = [u8p, u8p, ci, ci, ci, ci, sp]
            lib.hasf_oracle_hasf.argtypes = [u8p, u8p, u8p, ci, ci, ci, ci, u8p, sp]
            lib.hasf_oracle_hasf_stable.argtypes = [u8p, u8p, u8p, ci, ci, ci, ci, u8p, sp]
            lib.hasf3d_oracle_simple.argtypes = [ctypes.c_uint32]
            lib.hasf3d_oracle_edt.argtypes = [u8p, ci, ci, ci, ci, ci, i64p]
            lib.hasf3d_oracle_hasf.argtypes = [u8p, u8p, u8p, ci, ci, ci, ci, u8p]
            lib.hasf3d_oracle_operator.argtypes = [u8p, u8p, ci, ci, ci, ci, ci]
            for name in ("hasf_oracle_simple_lut", "hasf_oracle_edt", "hasf_oracle_dilate",
                         "hasf_oracle_erode", "hasf_oracle_thin", "hasf_oracle_thicken",
                         "hasf_oracle_hc", "hasf_oracle_hf", "hasf_oracle_hasf",
                         "hasf_oracle_hasf_stable", "hasf3d_oracle_simple", "hasf3d_oracle_edt",
                         "hasf3d_oracle_hasf", "hasf3d_oracle_operator"):
                getattr(lib, name).restype = ci
            lib.hasf_oracle_stats_size.restype = ci
            assert lib.hasf_oracle_stats_size() == ctypes.sizeof(Stats)
            _lib = lib
    return _lib


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray((np.asarray(a) != 0).astype(np.uint8))


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed (rc={rc})")


def simple_lut(conn: int = 8) -> np.ndarray:
    """256-entry table: 1 where a neighbour code describes a simple point."""
    out = np.zeros(256, np.uint8)
    _check(load().hasf_oracle_simple_lut(conn, _p(out, ctypes.c_uint8)), "simple_lut")
    return out


def edt(feature, outside_is_feature: bool = False) -> np.ndarray:
    """Exact squared Euclidean distance of every pixel to the feature set."""
    f = _u8(feature)
    h, w = f.shape
    d = np.zeros((h, w), np.int64)
    _check(load().hasf_oracle_edt(_p(f, ctypes.c_uint8), w, h, int(outside_is_feature),
                                  _p(d, ctypes.c_int64)), "edt")
    return d


def dilate(S, r: int) -> np.ndarray:
    s = _u8(S)
    h, w = s.shape
    out = np.zeros_like(s)
    _check(load().hasf_oracle_dilate(_p(s, ctypes.c_uint8), w, h, r, _p(out, ctypes.c_uint8)),
           "dilate")
    return out


def erode(S, r: int) -> np.ndarray:
    s = _u8(S)
    h, w = s.shape
    out = np.zeros_like(s)
    _check(load().hasf_oracle_erode(_p(s, ctypes.c_uint8), w, h, r, _p(out, ctypes.c_uint8)),
           "erode")
    return out


def thin(Z, W, prio, conn: int = 8, stats: Stats | None = None) -> np.ndarray:
    """H(Z, W) with the given priority map; returns the thinned set."""
    z = _u8(Z).copy()
    k = _u8(W)
    p = np.ascontiguousarray(prio, dtype=np.int64)
    h, w = z.shape
    _check(load().hasf_oracle_thin(_p(z, ctypes.c_uint8), _p(k, ctypes.c_uint8),
                                   _p(p, ctypes.c_int64), w, h, conn,
                                   ctypes.byref(stats) if stats is not None else None), "thin")
    return z


def thicken(Y, V, prio, conn: int = 8, stats: Stats | None = None) -> np.ndarray:
    """*H(Y, V) with the given priority map; returns the thickened set."""
    y = _u8(Y).copy()
    k = _u8(V)
    p = np.ascontiguousarray(prio, dtype=np.int64)
    h, w = y.shape
    _check(load().hasf_oracle_thicken(_p(y, ctypes.c_uint8), _p(k, ctypes.c_uint8),
                                      _p(p, ctypes.c_int64), w, h, conn,
                                      ctypes.byref(stats) if stats is not None else None),
           "thicken")
    return y


def hc(X, r: int, C=None, conn: int = 8, stats: Stats | None = None) -> np.ndarray:
    """Homotopic cutting HC_r^C(X)."""
    x = _u8(X).copy()
    h, w = x.shape
    c = _u8(C) if C is not None else None
    _check(load().hasf_oracle_hc(_p(x, ctypes.c_uint8),
                                 _p(c, ctypes.c_uint8) if c is not None else None,
                                 w, h, r, conn,
                                 ctypes.byref(stats) if stats is not None else None), "hc")
    return x


def hf(X, r: int, D=None, conn: int = 8, stats: Stats | None = None) -> np.ndarray:
    """Homotopic filling HF_r^D(X)."""
    x = _u8(X).copy()
    h, w = x.shape
    d = _u8(D) if D is not None else None
    _check(load().hasf_oracle_hf(_p(x, ctypes.c_uint8),
                                 _p(d, ctypes.c_uint8) if d is not None else None,
                                 w, h, r, conn,
                                 ctypes.byref(stats) if stats is not None else None), "hf")
    return x


def hasf(X, rmax: int, C=None, D=None, conn: int = 8, stats: Stats | None = None) -> np.ndarray:
    """HASF_rmax^{C,D}(X): cutting then filling for r = 1..rmax."""
    x = _u8(X)
    h, w = x.shape
    c = _u8(C) if C is not None else None
    d = _u8(D) if D is not None else None
    out = np.zeros_like(x)
    _check(load().hasf_oracle_hasf(_p(x, ctypes.c_uint8),
                                   _p(c, ctypes.c_uint8) if c is not None else None,
                                   _p(d, ctypes.c_uint8) if d is not None else None,
                                   w, h, rmax, conn, _p(out, ctypes.c_uint8),
                                   ctypes.byref(stats) if stats is not None else None), "hasf")
    return out


def hasf_stable(X, rcap: int = 64, C=None, D=None, conn: int = 8,
                stats: Stats | None = None) -> tuple[np.ndarray, int]:
    """HASF steps r = 1, 2, ... until one leaves the image unchanged (at most
    rcap steps).  Returns (image, r) with r the radius of the step that changed
    nothing, or 0 if step rcap still changed the image."""
    x = _u8(X)
    h, w = x.shape
    c = _u8(C) if C is not None else None
    d = _u8(D) if D is not None else None
    out = np.zeros_like(x)
    r = load().hasf_oracle_hasf_stable(_p(x, ctypes.c_uint8),
                                      _p(c, ctypes.c_uint8) if c is not None else None,
                                      _p(d, ctypes.c_uint8) if d is not None else None,
                                      w, h, rcap, conn, _p(out, ctypes.c_uint8),
                                      ctypes.byref(stats) if stats is not None else None)
    if r < 0:
        raise ValueError("hasf_stable: bad arguments")
    return out, r


# ---- 3D: (26, 6) adjacency, volumes indexed [z, y, x] --------------------------

def simple3d(code: int) -> bool:
    """Simplicity of the centre of a 3 x 3 x 3 neighbourhood; bit
    (dz+1)*9 + (dy+1)*3 + (dx+1) of code = object (the centre bit is ignored)."""
    return bool(load().hasf3d_oracle_simple(code & 0x7FFFFFF))


def edt3d(feat, r: int, outside_is_feature: bool = False) -> np.ndarray:
    """Squared distance to the nearest feature voxel, clamped at r^2 + 1."""
    f = _u8(feat)
    d, h, w = f.shape
    out = np.zeros(f.shape, np.int64)
    _check(load().hasf3d_oracle_edt(_p(f, ctypes.c_uint8), w, h, d, int(outside_is_feature), r,
                                    _p(out, ctypes.c_int64)), "edt3d")
    return out


def operator3d(S, K, r: int, thin: bool) -> np.ndarray:
    """H(S, K) (thin) or *H(S, K) in 3D with the clamped priority of radius r."""
    s = _u8(S).copy()
    k = _u8(K)
    d, h, w = s.shape
    _check(load().hasf3d_oracle_operator(_p(s, ctypes.c_uint8), _p(k, ctypes.c_uint8), w, h, d,
                                         r, int(thin)), "operator3d")
    return s


def hasf3d(X, rmax: int, C=None, D=None) -> np.ndarray:
    """HASF_rmax^{C,D} of a volume X (d, h, w) with (26, 6) adjacency."""
    x = _u8(X)
    d, h, w = x.shape
    c = _u8(C) if C is not None else None
    dd = _u8(D) if D is not None else None
    out = np.zeros_like(x)
    _check(load().hasf3d_oracle_hasf(_p(x, ctypes.c_uint8),
                                     _p(c, ctypes.c_uint8) if c is not None else None,
                                     _p(dd, ctypes.c_uint8) if dd is not None else None,
                                     w, h, d, rmax, _p(out, ctypes.c_uint8)), "hasf3d")
    return out

