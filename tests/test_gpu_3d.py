"""The 3D filter ((26, 6) adjacency) through hasf_smooth3d against the 3D
oracle, bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1603_09337_gb300 import _lib

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


def balls(seed, d, h, w, n, rlo, rhi, noise):
    rng = np.random.default_rng(seed)
    Z, Y, Xc = np.indices((d, h, w))
    X = np.zeros((d, h, w), np.uint8)
    for _ in range(n):
        cz, cy, cx = rng.integers(0, d), rng.integers(0, h), rng.integers(0, w)
        rr = rng.integers(rlo, rhi + 1)
        X |= ((Z - cz) ** 2 + (Y - cy) ** 2 + (Xc - cx) ** 2 <= rr * rr).astype(np.uint8)
    return (X ^ (rng.random((d, h, w)) < noise)).astype(np.uint8)


SHAPES = [(1, 1, 1), (1, 9, 40), (5, 6, 7), (12, 13, 33), (16, 20, 64), (9, 31, 70)]


def test_simple3_table_equals_oracle(ctx):
    """The table the 3D kernel reads against the oracle's simple-voxel test on
    sampled neighbourhoods: uniform, sparse and dense ones, and every code
    whose only object neighbours are among the six face neighbours."""
    lut = ctx.simple3_table()
    assert lut.shape == (1 << 21,)
    rng = np.random.default_rng(2603)
    idx = [rng.integers(0, 1 << 26, 60000)]
    for p in (0.1, 0.25, 0.75, 0.9):
        bits = rng.random((30000, 26)) < p
        idx.append((bits * (1 << np.arange(26))).sum(axis=1))
    faces = [4, 10, 12, 14, 16, 22]             # positions of the six face neighbours
    for m in range(64):
        code = sum(1 << faces[k] for k in range(6) if (m >> k) & 1)
        idx.append(np.array([(code & 0x1FFF) | ((code >> 14) << 13)]))
    idx = np.unique(np.concatenate(idx).astype(np.int64))
    got = (lut[idx >> 5] >> (idx & 31).astype(np.uint32)) & 1
    codes = (idx & 0x1FFF) | ((idx >> 13) << 14)
    want = np.array([oracle.simple3d(int(c)) for c in codes], np.uint32)
    assert 0 < want.sum() < len(want)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("table", [1, 0])
@pytest.mark.parametrize("rmax", [1, 2, 3])
def test_volumes_equal_oracle(ctx, rmax, table):
    """Both simple-voxel tests: the table and the flood fills."""
    ctx.set_option(_lib.OPT_SIMPLE3_TABLE, table)
    vols, want = [], []
    for i, (d, h, w) in enumerate(SHAPES):
        X = balls(100 * rmax + i, d, h, w, max(1, d * h * w // 2000), 2, 5, 0.04)
        rng = np.random.default_rng(i)
        C = (X & (rng.random(X.shape) < 0.02)).astype(np.uint8) if i % 2 else None
        D = ((1 - X) & (rng.random(X.shape) < 0.03)).astype(np.uint8) if i % 3 == 1 else None
        vols.append((dev(X), rmax, None if C is None else dev(C), None if D is None else dev(D)))
        want.append(oracle.hasf3d(X, rmax, C=C, D=D))
    outs = ctx.smooth3d(vols)
    ctx.status()
    ctx.set_option(_lib.OPT_SIMPLE3_TABLE, 1)
    for i, (o, e) in enumerate(zip(outs, want)):
        np.testing.assert_array_equal(host(o), e, err_msg=f"volume {i} {SHAPES[i]}")


def test_gang_volume_equals_oracle(ctx):
    """A volume shared by a gang of several CTAs, with and without C and D."""
    X = balls(7, 40, 48, 70, 12, 3, 7, 0.03)
    rng = np.random.default_rng(17)
    C = (X & (rng.random(X.shape) < 0.02)).astype(np.uint8)
    D = ((1 - X) & (rng.random(X.shape) < 0.03)).astype(np.uint8)
    outs = ctx.smooth3d([(dev(X), 2, None, None), (dev(X), 2, dev(C), dev(D))])
    ctx.status()
    np.testing.assert_array_equal(host(outs[0]), oracle.hasf3d(X, 2))
    np.testing.assert_array_equal(host(outs[1]), oracle.hasf3d(X, 2, C=C, D=D))


def test_round_cap_reports_timeout(ctx):
    X = balls(8, 10, 12, 14, 3, 2, 4, 0.05)
    ctx.set_option(_lib.OPT_ROUND_CAP, 1)
    try:
        ctx.smooth3d([(dev(X), 2, None, None)])
        with pytest.raises(_lib.HasfError) as e:
            ctx.status()
        assert e.value.code == _lib.HASF_ETIMEOUT
    finally:
        ctx.set_option(_lib.OPT_ROUND_CAP, 0)
    ctx.smooth3d([(dev(X), 1, None, None)])
    ctx.status()


def test_bad_volumes_rejected(ctx):
    import torch
    X = dev(np.zeros((4, 4, 4), np.uint8))
    for r in (0, 13):
        with pytest.raises(_lib.HasfError) as e:
            ctx.smooth3d([(X, r, None, None)])
        assert e.value.code == _lib.HASF_EINVAL
    with pytest.raises(ValueError):
        ctx.smooth3d([(torch.zeros((4, 4), dtype=torch.uint8, device="cuda"), 1, None, None)])


def test_wide_rows_take_the_unfused_passes(ctx):
    """Rows longer than 32 words (width > 1024) run the eight separate subfield
    passes instead of the fused pairs."""
    X = balls(9, 4, 5, 1100, 30, 1, 3, 0.05)
    got = host(ctx.smooth3d([(dev(X), 2, None, None)])[0])
    ctx.status()
    np.testing.assert_array_equal(got, oracle.hasf3d(X, 2))
