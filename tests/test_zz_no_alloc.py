"""The allocation-free entry point hasf_smooth_noalloc, for callers that cannot
allocate device memory (latency-critical loops that must not stall on
cudaMalloc, code inside a framework that owns the device memory).

It must give the same images as hasf_smooth, bit for bit, on consecutive
calls that reuse its fixed scratch array.  This file runs last so that a
failure here leaves every other test already run.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from paper_1603_09337_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09337_gb300 import Context, build
    build.build()
    torch.cuda.set_device(0)
    ctx = Context(0)
    yield ctx, _lib.load()
    ctx.close()


def _desc(X, out, C, D, rmax, conn, width=None):
    """Descriptor of device tensors that share one row pitch (their row
    stride); `width` (default: all columns) may be less than the pitch."""
    h, pitch = X.shape[0], X.stride(0)
    w = width if width is not None else X.shape[1]
    return _lib.HasfImage(X.data_ptr(), out.data_ptr(),
                          C.data_ptr() if C is not None else None,
                          D.data_ptr() if D is not None else None, w, h, pitch, rmax, conn, 0)


def _pitched(A, pitch, fill):
    """A (h, w) image in a device buffer whose rows are `pitch` bytes apart,
    the bytes past the width set to `fill`."""
    import torch
    h, w = A.shape
    buf = torch.full((h, pitch), fill, dtype=torch.uint8, device="cuda")
    buf[:, :w] = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    return buf


def test_noalloc_equals_hasf_smooth_on_two_calls(env):
    import torch
    ctx, lib = env
    jobs = synth.batch_512(2, first=500)
    Dm = synth.small_random(9, 512, 512, 20) & (1 - jobs[1].X)
    cases = [(jobs[0].X, jobs[0].C, None, 5, 8), (jobs[1].X, None, Dm, 4, 4)]
    stream = torch.cuda.current_stream()
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for X, C, D, rmax, conn in cases:          # two calls in a row, different images
        tX = torch.from_numpy(X).cuda()
        tC = torch.from_numpy(C).cuda() if C is not None else None
        tD = torch.from_numpy(np.ascontiguousarray(D)).cuda() if D is not None else None
        out = torch.zeros_like(tX)
        d = _desc(tX, out, tC, tD, rmax, conn)
        rc = lib.hasf_smooth_noalloc(ctypes.byref(d), ctypes.c_void_p(status.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
        assert rc == _lib.HASF_OK
        ref = ctx.smooth(tX, rmax, C=tC, D=tD, conn=conn)
        ctx.status()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_ragged_and_near_limit_equal_oracle(env):
    """Both kernels of the entry point -- the register kernel (images up to
    512 x 512, rmax <= 31) and the fused shared-memory kernel (larger images,
    larger rmax) -- on widths that are not a multiple of 32 (a partial last
    word), a row pitch above the width, C and D together, (4,8) adjacency, and
    an image near the shared-memory bound of the entry point (500 x 1130):
    equal to the oracle and to hasf_smooth, and the bytes past the width are
    left untouched."""
    import torch
    ctx, lib = env
    stream = torch.cuda.current_stream()
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    cases = []
    # register kernel: 300 x 317 with C and D, (4,8); 509 x 511 at its rmax bound
    X = synth.shapes_image(4141, 300, 317, 4, 8, 50, n_holes=2, jitter=2, noise_permille=40)
    cases.append((X, synth.constraint_points(5, X, 15),
                  synth.small_random(6, 300, 317, 30) & (1 - X), 3, 4, 352))
    X = synth.shapes_image(4040, 509, 511, 3, 20, 120, n_holes=3, jitter=2, noise_permille=20)
    cases.append((X, None, None, 31, 8, 512))
    # fused kernel: rmax above the register kernel's bound; width above 512
    X = synth.shapes_image(3939, 150, 200, 3, 10, 40, n_holes=2, jitter=2, noise_permille=30)
    cases.append((X, None, None, 33, 8, 208))
    X = synth.shapes_image(4242, 517, 300, 3, 10, 60, n_holes=2, jitter=2, noise_permille=40)
    C = synth.constraint_points(7, X, 20)
    Dm = synth.small_random(8, 517, 300, 30) & (1 - X)
    cases.append((X, C, Dm, 3, 4, 544))
    X2 = synth.shapes_image(4343, 500, 1130, 20, 10, 80, n_holes=6, jitter=2, noise_permille=50)
    cases.append((X2, synth.constraint_points(9, X2, 30), None, 4, 8, 512))
    for X, C, D, rmax, conn, pitch in cases:
        h, w = X.shape
        tX = _pitched(X, pitch, 1)
        tC = _pitched(C, pitch, 1) if C is not None else None
        tD = _pitched(D, pitch, 1) if D is not None else None
        out = torch.full_like(tX, 7)
        d = _desc(tX, out, tC, tD, rmax, conn, width=w)
        rc = lib.hasf_smooth_noalloc(ctypes.byref(d), ctypes.c_void_p(status.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
        assert rc == _lib.HASF_OK
        ref = torch.full_like(tX, 7)
        dr = _desc(tX, ref, tC, tD, rmax, conn, width=w)
        assert lib.hasf_smooth(ctx.h, ctypes.byref(dr), ctypes.c_void_p(stream.cuda_stream)) \
            == _lib.HASF_OK
        ctx.status()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        got = out.cpu().numpy()
        np.testing.assert_array_equal(got[:, :w], oracle.hasf(X, rmax, C=C, D=D, conn=conn),
                                      err_msg=f"{h}x{w}")
        np.testing.assert_array_equal(got, ref.cpu().numpy())
        assert (got[:, w:] == 7).all()


def test_noalloc_rejects_images_beyond_its_limit(env):
    import torch
    _, lib = env
    big = torch.zeros((2048, 2048), dtype=torch.uint8, device="cuda")
    d = _desc(big, big, None, None, 2, 8)
    assert lib.hasf_smooth_noalloc(ctypes.byref(d), None, None) == _lib.HASF_EBUDGET
    bad = _desc(big[:8, :8], big[:8, :8], None, None, 0, 8)
    assert lib.hasf_smooth_noalloc(ctypes.byref(bad), None, None) == _lib.HASF_EINVAL
