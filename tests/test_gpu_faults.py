"""Failure detection without a GPU fault.

A gang of CTAs (one large image, or a volume) meets at a global-memory
barrier whose waits are bounded by a deadline.  The host-set fault option
makes CTA 0 of every gang leave its job before its first barrier, as a CTA
that died would: the other CTAs' waits run out at a short deadline,
the job reports HASF_ETIMEOUT through the status word, and the context keeps
working.  Allocation failures are injected on the host and must surface as
HASF_ENOMEM from the call that needed the memory, with the context usable
afterwards.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
from paper_1603_09337_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09337_gb300 import build
    build.build()
    return torch


def _expect_timeout(ctx, t0, limit_s):
    with pytest.raises(_lib.HasfError) as e:
        ctx.status()
    assert e.value.code == _lib.HASF_ETIMEOUT
    assert time.perf_counter() - t0 < limit_s


def test_gang_barrier_deadline_without_a_fault(torch_cuda):
    """Generic gang (planes in L2) and tiled gang: CTA 0 never arrives, the
    others give up after 200 ms, the job reports
    HASF_ETIMEOUT; then the same context smooths the image correctly."""
    torch = torch_cuda
    from paper_1603_09337_gb300 import Context
    X = synth.shapes_image(71, 130, 70, 6, 4, 20, n_holes=2, hole_lo=2, hole_hi=4,
                           noise_permille=50)
    big = synth.shapes_image(72, 700, 600, 20, 10, 80, n_holes=4, jitter=2, noise_permille=30)
    with Context(0) as ctx:
        ctx.set_option(_lib.OPT_WAIT_DEADLINE_MS, 200)
        cases = [
            ("generic gang", X, [(_lib.OPT_FORCE_GANG, 1), (_lib.OPT_GANG_CTAS, 4)]),
            ("tiled gang", big, [(_lib.OPT_TILES, 2)]),
        ]
        for name, img, opts in cases:
            for o, v in opts:
                ctx.set_option(o, v)
            t = torch.from_numpy(img).cuda()
            ctx.set_option(_lib.OPT_FAULT_GANG_SKIP, 1)
            t0 = time.perf_counter()
            ctx.smooth(t, 2)
            _expect_timeout(ctx, t0, 10.0)
            ctx.set_option(_lib.OPT_FAULT_GANG_SKIP, 0)
            got = ctx.smooth(t, 2)
            ctx.status()
            np.testing.assert_array_equal(got.cpu().numpy(), oracle.hasf(img, 2), err_msg=name)
            for o, _ in opts:
                ctx.set_option(o, 1 if o == _lib.OPT_TILES else 0)


def test_volume_gang_deadline_without_a_fault(torch_cuda):
    """The 3D gang (64^3 volume, four CTAs) under the same injected fault."""
    torch = torch_cuda
    from paper_1603_09337_gb300 import Context
    X = synth.volume(31, 64, 64, 64, 20, 3, 9, 30)
    with Context(0) as ctx:
        ctx.set_option(_lib.OPT_WAIT_DEADLINE_MS, 200)
        ctx.set_option(_lib.OPT_FAULT_GANG_SKIP, 1)
        t = torch.from_numpy(X).cuda()
        t0 = time.perf_counter()
        ctx.smooth3d([(t, 2, None, None)])
        _expect_timeout(ctx, t0, 10.0)
        ctx.set_option(_lib.OPT_FAULT_GANG_SKIP, 0)
        got = ctx.smooth3d([(t, 2, None, None)])[0]
        ctx.status()
        np.testing.assert_array_equal(got.cpu().numpy(), oracle.hasf3d(X, 2))


def test_allocation_failure_reports_enomem(torch_cuda):
    """The first allocation after the fault option fails: hasf_smooth (scratch
    arena), hasf_smooth_host (staging buffers) and the server (a batch's
    scratch) report HASF_ENOMEM; the next calls succeed and are correct."""
    torch = torch_cuda
    from paper_1603_09337_gb300 import Context
    X = synth.shapes_image(73, 200, 150, 6, 5, 30, n_holes=2, noise_permille=40)
    want = oracle.hasf(X, 3)
    with Context(0) as ctx:
        t = torch.from_numpy(X).cuda()
        ctx.set_option(_lib.OPT_FAULT_ALLOC, 1)
        with pytest.raises(_lib.HasfError) as e:
            ctx.smooth(t, 3)
        assert e.value.code == _lib.HASF_ENOMEM
        got = ctx.smooth(t, 3)
        ctx.status()
        np.testing.assert_array_equal(got.cpu().numpy(), want)
    with Context(0) as ctx:
        out = np.zeros_like(X)
        ctx.set_option(_lib.OPT_FAULT_ALLOC, 1)
        with pytest.raises(_lib.HasfError) as e:
            ctx.smooth_host([(X, 3, None, None, 8, out)])
        assert e.value.code == _lib.HASF_ENOMEM
        ctx.smooth_host([(X, 3, None, None, 8, out)])
        np.testing.assert_array_equal(out, want)
    with Context(0) as ctx:
        t = torch.from_numpy(X).cuda()
        o1, o2 = torch.zeros_like(t), torch.zeros_like(t)
        ctx.set_option(_lib.OPT_FAULT_ALLOC, 1)
        k1 = ctx.submit(t, 3, o1)
        ctx.drain()
        assert ctx.poll(k1) == (1, _lib.HASF_ENOMEM)
        k2 = ctx.submit(t, 3, o2)
        ctx.drain()
        assert ctx.poll(k2) == (1, _lib.HASF_OK)
        np.testing.assert_array_equal(o2.cpu().numpy(), want)


def test_fault_options_are_checked(torch_cuda):
    from paper_1603_09337_gb300 import Context
    with Context(0) as ctx:
        for opt, bad in ((_lib.OPT_WAIT_DEADLINE_MS, -1), (_lib.OPT_WAIT_DEADLINE_MS, 60001),
                         (_lib.OPT_FAULT_GANG_SKIP, -1), (_lib.OPT_FAULT_GANG_SKIP, 2),
                         (_lib.OPT_FAULT_ALLOC, -1)):
            with pytest.raises(_lib.HasfError) as e:
                ctx.set_option(opt, bad)
            assert e.value.code == _lib.HASF_EINVAL
