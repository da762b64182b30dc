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
    """The autotuner records a launch shape for a tiled-size bucket and a sweep
    schedule for a register-kernel bucket; later calls use them and still equal
    the oracle; the choices survive a save / load round trip."""
    import torch
    from paper_1603_09337_gb300 import Context
    c = ctx.autotune(800, 640, 3)
    assert c in (-1, 0) or (c & (c - 1)) == 0    # tiled, one CTA or a power of two
    assert ctx.tuning_get(800, 640, 3) == (c, 0)
    assert ctx.autotune(400, 300, 3) == 0        # register kernel: its sweep schedule is tuned
    ctas, group = ctx.tuning_get(400, 300, 3)
    assert ctas == 0 and group in (1, 2, 4)
    for w, h in ((800, 640), (400, 300)):
        X = synth.shapes_image(5, w, h, 20, 5, 60, n_holes=3, noise_permille=50)
        got = ctx.smooth(torch.from_numpy(X).cuda(), 3)
        ctx.status()
        np.testing.assert_array_equal(got.cpu().numpy(), oracle.hasf(X, 3))
    path = str(tmp_path / "tune.txt")
    ctx.tuning_save(path)
    rows = [l.split() for l in open(path) if l.strip()]
    assert rows and all(len(r) == 5 for r in rows)
    with Context(0) as fresh:
        assert fresh.tuning_get(400, 300, 3) is None
        fresh.tuning_load(path)
        assert fresh.tuning_get(400, 300, 3) == (0, group)
        assert fresh.tuning_get(800, 640, 3) == (c, 0)


@pytest.mark.parametrize("group", [1, 2, 4])
def test_every_sweep_schedule_equals_oracle(ctx, group):
    """The register kernel's three sweep schedules (rows of a parity tested
    together) give the oracle's images, for both adjacencies, with C and D."""
    import torch
    from paper_1603_09337_gb300 import _lib
    ctx.set_option(_lib.OPT_ROW_GROUP, group)
    try:
        for i, (w, h, r, conn) in enumerate([(512, 512, 5, 8), (300, 200, 3, 4), (97, 61, 2, 8),
                                             (511, 333, 4, 4)]):
            X = synth.shapes_image(40 + i, w, h, max(1, w * h // 20000), 5, 50, n_holes=3,
                                   jitter=2, noise_permille=60)
            C = synth.constraint_points(i, X, 20)
            Dm = synth.small_random(i + 3, w, h, 20) & (1 - X)
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            got = ctx.smooth(t(X), r, C=t(C), D=t(Dm), conn=conn)
            ctx.status()
            np.testing.assert_array_equal(got.cpu().numpy(),
                                          oracle.hasf(X, r, C=C, D=Dm, conn=conn),
                                          err_msg=f"{w}x{h} group {group}")
    finally:
        ctx.set_option(_lib.OPT_ROW_GROUP, 0)
