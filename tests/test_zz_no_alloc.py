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


def _desc(X, out, C, D, rmax, conn):
    h, w = X.shape
    return _lib.HasfImage(X.data_ptr(), out.data_ptr(),
                          C.data_ptr() if C is not None else None,
                          D.data_ptr() if D is not None else None, w, h, w, rmax, conn, 0)


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


def test_noalloc_rejects_images_beyond_its_limit(env):
    import torch
    _, lib = env
    big = torch.zeros((2048, 2048), dtype=torch.uint8, device="cuda")
    d = _desc(big, big, None, None, 2, 8)
    assert lib.hasf_smooth_noalloc(ctypes.byref(d), None, None) == _lib.HASF_EBUDGET
    bad = _desc(big[:8, :8], big[:8, :8], None, None, 0, 8)
    assert lib.hasf_smooth_noalloc(ctypes.byref(bad), None, None) == _lib.HASF_EINVAL
