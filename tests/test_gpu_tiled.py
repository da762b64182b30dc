"""The tiled register kernel (images larger than 512 x 512): thread-block
clusters of up to 16 tiles, and the gang form through global memory."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1603_09337_gb300 import _lib, synth

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


def img(seed, h, w, noise=50):
    n = max(1, (h * w) // 25000)
    return synth.shapes_image(seed, w, h, n, 6, max(8, min(h, w) // 5), n_holes=n // 2 + 1,
                              hole_lo=2, hole_hi=6, jitter=2, noise_permille=noise)


# tile grids 2x1, 1x2, 2x2, 3x2, 2x3 with ragged last tiles
SHAPES = [(100, 600), (600, 100), (700, 700), (900, 1100), (1300, 800), (513, 1025)]


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("conn", [8, 4])
def test_tiled_equals_oracle(ctx, mode, conn):
    ctx.set_option(_lib.OPT_TILES, mode)
    try:
        for i, (h, w) in enumerate(SHAPES):
            X = img(500 + i, h, w)
            C = synth.constraint_points(i, X, 7)
            Dm = synth.small_random(600 + i, w, h, 20) & (1 - X)
            r = 2 + i % 3
            got = host(ctx.smooth(dev(X), r, C=dev(C), D=dev(Dm), conn=conn))
            ctx.status()
            np.testing.assert_array_equal(got, oracle.hasf(X, r, C=C, D=Dm, conn=conn),
                                          err_msg=f"{h}x{w} r{r}")
    finally:
        ctx.set_option(_lib.OPT_TILES, 1)


def test_tiled_operators(ctx):
    X = img(77, 800, 900)
    W = synth.small_random(3, 900, 800, 30) & X
    for op, ref in [(_lib.OP_HC, lambda: oracle.hc(X, 3, C=W)), (_lib.OP_HF, lambda: oracle.hf(X, 3))]:
        got = host(ctx.operator(op, dev(X), 3, C=dev(W) if op == _lib.OP_HC else None))
        np.testing.assert_array_equal(got, ref())


def test_sixteen_tile_cluster(ctx):
    """2048 x 2048 = 4 x 4 tiles, the largest cluster."""
    X = img(9, 2048, 2048, noise=40)
    got = host(ctx.smooth(dev(X), 4))
    ctx.status()
    np.testing.assert_array_equal(got, oracle.hasf(X, 4))


def test_tiled_equals_generic(ctx):
    """The same bytes from the tiled, generic one-CTA/gang and forced-gang paths."""
    X = img(31, 1000, 1500)
    a = host(ctx.smooth(dev(X), 6))
    ctx.set_option(_lib.OPT_TILES, 0)
    try:
        b = host(ctx.smooth(dev(X), 6))
    finally:
        ctx.set_option(_lib.OPT_TILES, 1)
    ctx.status()
    np.testing.assert_array_equal(a, b)
