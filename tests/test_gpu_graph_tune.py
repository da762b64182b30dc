"""CUDA-graph replay of a batched launch, and the autotuner."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1603_09337_gb300 import synth

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


def test_graph_replays_new_contents(ctx):
    """One graph over a mixed batch (register, one-CTA and gang paths); new
    image bytes written into the same buffers give the new results."""
    import torch
    from paper_1603_09337_gb300 import Image
    sizes = [(512, 512, 5), (300, 200, 3), (700, 520, 4), (1100, 900, 2)]
    bufs = [torch.zeros((h, w), dtype=torch.uint8, device="cuda") for w, h, _ in sizes]
    imgs = [Image(b, r) for b, (w, h, r) in zip(bufs, sizes)]
    g = ctx.graph_create(imgs)
    try:
        for rep in range(2):
            X = [synth.shapes_image(100 * rep + i, w, h, max(1, w * h // 30000), 5, 40,
                                    n_holes=2, noise_permille=40)
                 for i, (w, h, _) in enumerate(sizes)]
            for b, x in zip(bufs, X):
                b.copy_(torch.from_numpy(x))
            ctx.graph_launch(g)
            ctx.status()
            for im, x, (w, h, r) in zip(imgs, X, sizes):
                got = im.out.cpu().numpy()
                if w * h <= 300 * 200:
                    np.testing.assert_array_equal(got, oracle.hasf(x, r))
                ref = ctx.smooth(torch.from_numpy(x).cuda(), r)
                ctx.status()
                np.testing.assert_array_equal(got, ref.cpu().numpy())
    finally:
        ctx.graph_destroy(g)


def test_autotune_choice_and_roundtrip(ctx, tmp_path):
    import torch
    c = ctx.autotune(800, 640, 3)
    assert c in (-1, 0) or (c & (c - 1)) == 0    # tiled, one CTA or a power of two
    assert ctx.autotune(400, 300, 3) == 0        # register kernel: nothing to tune
    X = synth.shapes_image(5, 800, 640, 20, 5, 60, n_holes=3, noise_permille=50)
    got = ctx.smooth(torch.from_numpy(X).cuda(), 3)
    ctx.status()
    np.testing.assert_array_equal(got.cpu().numpy(), oracle.hasf(X, 3))
    path = str(tmp_path / "tune.txt")
    ctx.tuning_save(path)
    text = open(path).read().split()
    assert text and len(text) % 4 == 0
    ctx.tuning_load(path)
