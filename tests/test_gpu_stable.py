"""The filter run to stability (rmax < 0): steps r = 1, 2, ... until one
leaves the image unchanged, on the generic kernels, against the oracle."""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
from paper_1603_09337_gb300 import Image, _lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09337_gb300 import Context, build
    build.build()
    c = Context(0)
    yield c
    c.close()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def img(seed, h, w, noise=40):
    n = max(1, (h * w) // 2500)
    return synth.shapes_image(seed, w, h, n, 4, max(6, min(h, w) // 5), n_holes=n // 2 + 1,
                              hole_lo=2, hole_hi=5, jitter=1, noise_permille=noise)


SIZES = [(1, 1), (3, 70), (40, 48), (61, 97), (80, 96), (128, 130), (33, 200)]


@pytest.mark.parametrize("conn", [8, 4])
def test_stable_batch_equals_oracle(ctx, conn):
    jobs, expect = [], []
    for i, (h, w) in enumerate(SIZES):
        X = img(1200 + i, h, w)
        C = synth.constraint_points(i, X, 5) if i % 2 else None
        Dm = (synth.small_random(1300 + i, w, h, 20) & (1 - X)) if i % 3 == 0 else None
        out, r = oracle.hasf_stable(X, 64, C=C, D=Dm, conn=conn)
        assert r >= 1
        jobs.append(Image(dev(X), _lib.RMAX_STABLE, C=None if C is None else dev(C),
                          D=None if Dm is None else dev(Dm), conn=conn))
        expect.append(out)
    outs = ctx.smooth_batch(jobs)
    ctx.status()
    for i, (o, e) in enumerate(zip(outs, expect)):
        np.testing.assert_array_equal(host(o), e, err_msg=f"image {i} {SIZES[i]}")


def test_stable_mixed_with_fixed_order(ctx):
    """Run-to-stability images and fixed-order images in one launch (the latter
    on the register kernel) each give their own result."""
    xs = [img(1400 + i, 90 + 7 * i, 110 - 5 * i) for i in range(6)]
    rm = [_lib.RMAX_STABLE if i % 2 == 0 else 1 + i % 4 for i in range(6)]
    outs = ctx.smooth_batch([Image(dev(x), r) for x, r in zip(xs, rm)])
    ctx.status()
    for x, r, o in zip(xs, rm, outs):
        e = oracle.hasf_stable(x, 64)[0] if r < 0 else oracle.hasf(x, r)
        np.testing.assert_array_equal(host(o), e)


def test_stable_in_gang_mode(ctx):
    ctx.set_option(_lib.OPT_FORCE_GANG, 1)
    ctx.set_option(_lib.OPT_GANG_CTAS, 3)
    try:
        X = img(1500, 150, 170)
        C = synth.constraint_points(3, X, 9)
        got = host(ctx.smooth(dev(X), -20, C=dev(C)))
        ctx.status()
        np.testing.assert_array_equal(got, oracle.hasf_stable(X, 20, C=C)[0])
    finally:
        ctx.set_option(_lib.OPT_FORCE_GANG, 0)
        ctx.set_option(_lib.OPT_GANG_CTAS, 0)


def test_stable_cap_reports_unstable(ctx):
    """A cap below the fixed point: HASF_EUNSTABLE, and the output is the filter
    of order cap."""
    X = img(1600, 80, 96)
    _, r = oracle.hasf_stable(X, 64)
    assert r >= 2
    got = host(ctx.smooth(dev(X), -(r - 1)))
    with pytest.raises(_lib.HasfError) as e:
        ctx.status()
    assert e.value.code == _lib.HASF_EUNSTABLE
    np.testing.assert_array_equal(got, oracle.hasf(X, r - 1))
    ctx.status()   # the status was cleared


def test_stable_served(ctx):
    import torch
    X = img(1700, 100, 120)
    out = torch.empty_like(dev(X))
    t = ctx.submit(dev(X), _lib.RMAX_STABLE, out)
    t0 = time.time()
    while True:
        done, st = ctx.poll(t)
        if done:
            break
        assert time.time() - t0 < 60
        time.sleep(0.001)
    assert st == _lib.HASF_OK
    np.testing.assert_array_equal(host(out), oracle.hasf_stable(X, 64)[0])


def test_stable_rejected_where_undefined(ctx):
    X = dev(img(1800, 40, 40))
    with pytest.raises(_lib.HasfError):
        ctx.smooth(X, -65)
    with pytest.raises(_lib.HasfError):
        ctx.smooth(X, 0)
    with pytest.raises(_lib.HasfError):
        ctx.operator(_lib.OP_THIN, X, -3)


@pytest.mark.parametrize("conn", [8, 4])
def test_stable_on_the_register_kernel(ctx, conn):
    """Caps of at most 31 steps on images of at most 512 x 512 run on the
    register kernel; the results equal the oracle's."""
    jobs, expect = [], []
    for i, (h, w) in enumerate([(40, 48), (80, 96), (128, 130), (300, 512), (512, 257)]):
        X = img(1900 + i, h, w)
        C = synth.constraint_points(i, X, 5) if i % 2 else None
        out, r = oracle.hasf_stable(X, 31, C=C, conn=conn)
        jobs.append(Image(dev(X), -31, C=None if C is None else dev(C), conn=conn))
        expect.append((out, r))
    outs = ctx.smooth_batch(jobs)
    if all(r > 0 for _, r in expect):
        ctx.status()
    else:
        with pytest.raises(_lib.HasfError):
            ctx.status()
    for o, (e, _) in zip(outs, expect):
        np.testing.assert_array_equal(host(o), e)
