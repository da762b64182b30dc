"""GB300 (sm_103a) homotopic alternating sequential filter (HASF).

Topology-preserving smoothing of binary images after Mahmoudi & Akil,
"Real Time Topological Image Smoothing On Shared Memory Parallel Machines"
(arXiv:1603.09337): for r = 1..rmax, a homotopic cutting HC_r (eq. (i)) then a
homotopic filling HF_r (eq. (ii)) by Euclidean discs.

Every step runs in the CUDA library behind the C ABI of include/hasf.h; this
package only marshals arguments (PyTorch supplies device memory and streams).
Importing it does not load the library; the first call does, and fails loudly
if it has not been built.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import _lib
from ._lib import HasfError, check

__all__ = ["Context", "HasfError", "Image", "build_library"]


def build_library(force: bool = False) -> str:
    from . import build
    return build.build(force=force)


@dataclass
class Image:
    """One job: X (h, w) uint8 tensor; optional C, D of the same shape."""

    X: object
    rmax: int
    C: object = None
    D: object = None
    conn: int = 8
    out: object = None


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _desc(X, out, C, D, rmax, conn) -> _lib.HasfImage:
    h, w = X.shape[-2], X.shape[-1]
    pitch = X.stride(-2) if X.dim() >= 2 else w
    for t in (out, C, D):
        if t is not None and (tuple(t.shape[-2:]) != (h, w) or t.stride(-2) != pitch):
            raise ValueError("in, out, C and D must share shape and row pitch")
    if X.dtype.itemsize != 1 or X.stride(-1) != 1:
        raise ValueError("images must be uint8 with unit column stride")
    return _lib.HasfImage(X.data_ptr(), out.data_ptr(),
                          C.data_ptr() if C is not None else None,
                          D.data_ptr() if D is not None else None,
                          w, h, pitch, rmax, conn, 0)


class Context:
    """A library context on one CUDA device (hasf_create / hasf_destroy)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        check(self.lib.hasf_create(ctypes.byref(h), device, budget_bytes), "hasf_create")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self.lib.hasf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- options -------------------------------------------------------------
    def set_option(self, option: int, value: int):
        check(self.lib.hasf_set_option(self.h, option, value), "hasf_set_option")

    # -- device-pointer entry points -------------------------------------------
    def smooth(self, X, rmax: int, C=None, D=None, conn: int = 8, out=None, stream=None):
        """HASF_rmax^{C,D}(X) on the device; returns `out` (allocated if None)."""
        import torch
        if out is None:
            out = torch.empty_like(X)
        d = _desc(X, out, C, D, rmax, conn)
        check(self.lib.hasf_smooth(self.h, ctypes.byref(d), _stream_handle(stream)), "hasf_smooth")
        return out

    def smooth_batch(self, images: list[Image], stream=None):
        """One launch over many images; fills each Image.out (allocating if None)."""
        import torch
        arr = (_lib.HasfImage * max(1, len(images)))()
        for i, im in enumerate(images):
            if im.out is None:
                im.out = torch.empty_like(im.X)
            arr[i] = _desc(im.X, im.out, im.C, im.D, im.rmax, im.conn)
        check(self.lib.hasf_smooth_batch(self.h, arr, len(images), _stream_handle(stream)),
              "hasf_smooth_batch")
        return [im.out for im in images]

    def batch_descriptors(self, images: list[Image]):
        """Pre-built descriptor array for repeated hasf_smooth_batch calls."""
        import torch
        arr = (_lib.HasfImage * max(1, len(images)))()
        for i, im in enumerate(images):
            if im.out is None:
                im.out = torch.empty_like(im.X)
            arr[i] = _desc(im.X, im.out, im.C, im.D, im.rmax, im.conn)
        return arr

    def smooth_batch_raw(self, arr, n: int, stream=None):
        check(self.lib.hasf_smooth_batch(self.h, arr, n, _stream_handle(stream)),
              "hasf_smooth_batch")

    def read_stats(self) -> dict:
        """Work counters of launches made with OPT_STATS on (then reset)."""
        buf = (ctypes.c_uint64 * len(_lib.STAT_NAMES))()
        check(self.lib.hasf_read_stats(self.h, buf, len(_lib.STAT_NAMES)), "hasf_read_stats")
        return dict(zip(_lib.STAT_NAMES, (int(v) for v in buf)))

    def stats_step(self, arr, n: int, stream=None) -> dict:
        """Counters of one batched launch of the descriptor array `arr` (untimed)."""
        self.read_stats()
        self.set_option(_lib.OPT_STATS, 1)
        try:
            self.smooth_batch_raw(arr, n, stream)
            return self.read_stats()
        finally:
            self.set_option(_lib.OPT_STATS, 0)

    def status(self, stream=None):
        """Synchronise the stream and raise if a device-side failure was recorded."""
        check(self.lib.hasf_status_of(self.h, _stream_handle(stream)), "hasf_status_of")

    def operator(self, op: int, X, r: int, C=None, D=None, conn: int = 8, out=None, stream=None):
        """One operator: _lib.OP_THIN (C = W), OP_THICK (C = V), OP_HC, OP_HF."""
        import torch
        if out is None:
            out = torch.empty_like(X)
        d = _desc(X, out, C, D, r, conn)
        check(self.lib.hasf_operator(self.h, op, ctypes.byref(d), _stream_handle(stream)),
              "hasf_operator")
        return out

    def edt(self, F, outside_is_feature: bool = False, stream=None):
        """Exact squared EDT (int32, -1 = no feature) of a uint8 device image."""
        import torch
        h, w = F.shape
        d = torch.empty((h, w), dtype=torch.int32, device=F.device)
        check(self.lib.hasf_edt(self.h, _ptr(F), w, h, F.stride(0), int(outside_is_feature),
                                _ptr(d), _stream_handle(stream)), "hasf_edt")
        return d

    def levels(self, F, r: int, mode: int = 0, stream=None):
        """Priority levels as the fused kernel derives them (r^2 + 1 = beyond r).
        mode 0: distance to F; 1: to F plus the outside; 2: to the complement
        of F plus the outside."""
        import torch
        h, w = F.shape
        d = torch.empty((h, w), dtype=torch.int32, device=F.device)
        check(self.lib.hasf_levels(self.h, _ptr(F), w, h, F.stride(0), mode,
                                   r, _ptr(d), _stream_handle(stream)), "hasf_levels")
        return d

    def simple_table(self, conn: int = 8):
        import numpy as np
        out = np.zeros(256, np.uint8)
        check(self.lib.hasf_simple_table(self.h, conn, out.ctypes.data_as(ctypes.c_void_p)),
              "hasf_simple_table")
        return out

    def simple3_table(self, stream=None):
        """The 3D simple-voxel table as a numpy uint32 array of 2^21 words."""
        import torch
        out = torch.empty(1 << 21, dtype=torch.int32, device=f"cuda:{self.device}")
        check(self.lib.hasf_simple3_table(self.h, _ptr(out), _stream_handle(stream)),
              "hasf_simple3_table")
        torch.cuda.synchronize(self.device)
        return out.cpu().numpy().view("uint32")

    # -- CUDA graphs and the autotuner --------------------------------------------
    def graph_create(self, images: list[Image]):
        """Capture one batched launch of `images` (buffers fixed) as a CUDA graph."""
        arr = self.batch_descriptors(images)
        g = ctypes.c_void_p()
        check(self.lib.hasf_graph_create(self.h, arr, len(images), ctypes.byref(g)),
              "hasf_graph_create")
        return g

    def graph_launch(self, graph, stream=None):
        check(self.lib.hasf_graph_launch(graph, _stream_handle(stream)), "hasf_graph_launch")

    def graph_destroy(self, graph):
        check(self.lib.hasf_graph_destroy(graph), "hasf_graph_destroy")

    def autotune(self, width: int, height: int, rmax: int, conn: int = 8) -> int:
        """Time the launch shapes for this size bucket; returns CTAs per image (0 = one CTA)."""
        c = ctypes.c_int32()
        check(self.lib.hasf_autotune(self.h, width, height, rmax, conn, ctypes.byref(c)),
              "hasf_autotune")
        return c.value

    def tuning_get(self, width: int, height: int, rmax: int):
        """(ctas, rows_per_group) recorded for the size bucket, or None."""
        c, g = ctypes.c_int32(), ctypes.c_int32()
        rc = self.lib.hasf_tuning_get(self.h, width, height, rmax, ctypes.byref(c), ctypes.byref(g))
        if rc == _lib.HASF_ENOTFOUND:
            return None
        check(rc, "hasf_tuning_get")
        return c.value, g.value

    def tuning_save(self, path: str):
        check(self.lib.hasf_tuning_save(self.h, path.encode()), "hasf_tuning_save")

    def tuning_load(self, path: str):
        check(self.lib.hasf_tuning_load(self.h, path.encode()), "hasf_tuning_load")

    # -- host-buffer entry point -----------------------------------------------
    def host_descriptors(self, jobs):
        """Descriptor array for hasf_smooth_host over host buffers, checked once,
        for callers that smooth new contents of the same buffers again and
        again (see smooth_host_raw).  jobs: list of (X numpy (h, w) uint8,
        rmax, C or None, D or None, conn, out numpy); the arrays of one job may
        be row-strided views (pixels adjacent in a row) sharing one row stride,
        the pitch.  The arrays must stay alive while the descriptors are used."""
        arr = (_lib.HasfImage * max(1, len(jobs)))()
        for i, (X, rmax, C, D, conn, out) in enumerate(jobs):
            h, w = X.shape
            pitch = X.strides[0]
            for a in (X, C, D, out):
                if a is not None:
                    if (a.dtype.itemsize != 1 or a.shape != (h, w) or a.strides[1] != 1
                            or a.strides[0] != pitch):
                        raise ValueError("host images: (h, w) uint8, one row stride per job")
            arr[i] = _lib.HasfImage(X.ctypes.data, out.ctypes.data,
                                    C.ctypes.data if C is not None else None,
                                    D.ctypes.data if D is not None else None,
                                    w, h, pitch, rmax, conn, 0)
        return arr

    def smooth_host_raw(self, arr, n: int):
        """hasf_smooth_host over a descriptor array from host_descriptors."""
        check(self.lib.hasf_smooth_host(self.h, arr, n), "hasf_smooth_host")

    def smooth_host(self, jobs):
        """HASF of host buffers (see host_descriptors for `jobs`); synchronous."""
        self.smooth_host_raw(self.host_descriptors(jobs), len(jobs))

    # -- serving ------------------------------------------------------------------
    def smooth3d(self, volumes, stream=None):
        """HASF of 3D volumes, (26, 6) adjacency.  volumes: list of
        (X, rmax, C, D) with X a contiguous (d, h, w) uint8 CUDA tensor (C, D of
        the same shape or None).  Returns the output tensors."""
        import torch
        arr = (_lib.HasfVolume * max(1, len(volumes)))()
        outs = []
        for i, (X, rmax, C, D) in enumerate(volumes):
            if X.dim() != 3 or not X.is_contiguous() or X.dtype != torch.uint8:
                raise ValueError("a volume is a contiguous (d, h, w) uint8 tensor")
            out = torch.empty_like(X)
            outs.append(out)
            d, h, w = X.shape
            arr[i] = _lib.HasfVolume(X.data_ptr(), out.data_ptr(),
                                     None if C is None else C.data_ptr(),
                                     None if D is None else D.data_ptr(), w, h, d, rmax, (0, 0))
        check(self.lib.hasf_smooth3d(self.h, arr, len(volumes), _stream_handle(stream)),
              "hasf_smooth3d")
        return outs

    def submit(self, X, rmax: int, out, C=None, D=None, conn: int = 8) -> int:
        d = _desc(X, out, C, D, rmax, conn)
        t = ctypes.c_uint64()
        check(self.lib.hasf_submit(self.h, ctypes.byref(d), ctypes.byref(t)), "hasf_submit")
        return t.value

    def poll(self, ticket: int):
        """(done, status) of a submitted job."""
        done, st = ctypes.c_int(), ctypes.c_int()
        check(self.lib.hasf_poll(self.h, ticket, ctypes.byref(done), ctypes.byref(st)),
              "hasf_poll")
        return bool(done.value), st.value

    def cancel(self, ticket: int) -> int:
        return self.lib.hasf_cancel(self.h, ticket)

    def drain(self):
        check(self.lib.hasf_drain(self.h), "hasf_drain")
