"""Parity of the CUDA library (through its C ABI) with the CPU oracle.

All results are integers/bits: the bar is bit-exact equality.
"""
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


SIZES = [(1, 1), (1, 64), (64, 1), (31, 33), (33, 31), (37, 100), (32, 32), (65, 97), (130, 70)]


def case_image(seed, h, w, noise=50):
    n_shapes = max(1, (h * w) // 900)
    hi = max(3, min(h, w) // 3)
    lo = max(1, min(3, hi))
    return synth.shapes_image(seed, w, h, n_shapes, lo, hi, n_holes=n_shapes // 2, hole_lo=1,
                              hole_hi=max(1, hi // 3), jitter=1, noise_permille=noise)


# --- single steps ----------------------------------------------------------------

@pytest.mark.parametrize("conn", [8, 4])
def test_simple_table_matches_oracle(ctx, conn):
    np.testing.assert_array_equal(ctx.simple_table(conn), oracle.simple_lut(conn))


@pytest.mark.parametrize("h,w", SIZES + [(513, 511), (512, 512)])
@pytest.mark.parametrize("outside", [False, True])
def test_edt_matches_oracle(ctx, h, w, outside):
    for seed, dens in [(1, 30), (2, 500), (3, 0)]:
        F = synth.small_random(seed + h * 131 + w, w, h, dens)
        got = host(ctx.edt(dev(F), outside)).astype(np.int64)
        exp = oracle.edt(F, outside)
        exp[exp == oracle.INF] = -1
        np.testing.assert_array_equal(got, exp)


@pytest.mark.parametrize("r", [1, 2, 3, 5, 10, 33, 64])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_levels_equal_clamped_oracle_edt(ctx, r, mode):
    """The threshold walk of the fused kernel gives the clamped exact EDT."""
    for h, w in [(45, 77), (130, 33), (8, 300)]:
        F = synth.small_random(r * 7 + h + w, w, h, 8 if mode != 2 else 990)
        got = host(ctx.levels(dev(F), r, mode)).astype(np.int64)
        feat, outside = (1 - F, True) if mode == 2 else (F, mode == 1)
        exp = np.minimum(oracle.edt(feat, outside), r * r + 1)
        np.testing.assert_array_equal(got, exp)


def _thin_ref(Z, W, r, conn):
    prio = oracle.edt(1 - Z, outside_is_feature=True)
    return oracle.thin(Z, W | (prio > r * r).astype(np.uint8), prio, conn)


def _thick_ref(Y, V, r, conn):
    prio = oracle.edt(Y)
    return oracle.thicken(Y, V & (prio <= r * r).astype(np.uint8), prio, conn)


@pytest.mark.parametrize("conn", [8, 4])
@pytest.mark.parametrize("r", [1, 2, 4])
def test_thin_and_thicken_operators(ctx, conn, r):
    for i, (h, w) in enumerate(SIZES):
        Z = case_image(10 + i, h, w)
        W = synth.small_random(20 + i, w, h, 40) & Z
        got = host(ctx.operator(_lib.OP_THIN, dev(Z), r, C=dev(W), conn=conn))
        np.testing.assert_array_equal(got, _thin_ref(Z, W, r, conn), err_msg=f"thin {h}x{w}")
        V = synth.small_random(30 + i, w, h, 800)
        got = host(ctx.operator(_lib.OP_THICK, dev(Z), r, C=dev(V), conn=conn))
        np.testing.assert_array_equal(got, _thick_ref(Z, V, r, conn), err_msg=f"thick {h}x{w}")


@pytest.mark.parametrize("r", [1, 3])
def test_cutting_and_filling_operators(ctx, r):
    for i, (h, w) in enumerate(SIZES):
        X = case_image(40 + i, h, w)
        C = synth.constraint_points(i, X, 5)
        D = synth.small_random(50 + i, w, h, 30) & (1 - X)
        np.testing.assert_array_equal(host(ctx.operator(_lib.OP_HC, dev(X), r, C=dev(C))),
                                      oracle.hc(X, r, C=C))
        np.testing.assert_array_equal(host(ctx.operator(_lib.OP_HF, dev(X), r, D=dev(D))),
                                      oracle.hf(X, r, D=D))


# --- the whole filter ---------------------------------------------------------------

@pytest.mark.parametrize("conn", [8, 4])
@pytest.mark.parametrize("rmax", [1, 2, 3, 5])
def test_hasf_small_sizes(ctx, conn, rmax):
    for i, (h, w) in enumerate(SIZES):
        X = case_image(60 + i + rmax, h, w)
        got = host(ctx.smooth(dev(X), rmax, conn=conn))
        np.testing.assert_array_equal(got, oracle.hasf(X, rmax, conn=conn), err_msg=f"{h}x{w}")


def test_hasf_with_constraints(ctx):
    for i, (h, w) in enumerate(SIZES[3:]):
        X = case_image(80 + i, h, w)
        C = synth.constraint_points(i + 3, X, 8)
        D = synth.small_random(90 + i, w, h, 40) & (1 - X)
        got = host(ctx.smooth(dev(X), 3, C=dev(C), D=dev(D)))
        np.testing.assert_array_equal(got, oracle.hasf(X, 3, C=C, D=D))


def test_hasf_512_rmax3(ctx):
    job = synth.single_512()
    got = host(ctx.smooth(dev(job.X), job.rmax))
    np.testing.assert_array_equal(got, oracle.hasf(job.X, job.rmax))


def test_hasf_ragged_tile_edges(ctx):
    for h, w in [(513, 511), (511, 513), (257, 1025), (1000, 95)]:
        X = case_image(h * 3 + w, h, w)
        got = host(ctx.smooth(dev(X), 2))
        np.testing.assert_array_equal(got, oracle.hasf(X, 2), err_msg=f"{h}x{w}")


def test_degenerate_images(ctx):
    for h, w in [(1, 1), (1, 40), (40, 1), (2, 2), (7, 5)]:
        for X in (np.zeros((h, w), np.uint8), np.ones((h, w), np.uint8)):
            np.testing.assert_array_equal(host(ctx.smooth(dev(X), 4)), oracle.hasf(X, 4))


def test_nonbinary_input_and_pitch(ctx):
    import torch
    X = case_image(7, 60, 70)
    big = np.zeros((60, 96), np.uint8)
    big[:, :70] = X * 200                 # non-zero means object
    t = dev(big)
    view = t[:, :70]
    out = torch.zeros_like(t)[:, :70]
    ctx.smooth(view, 3, out=out)
    np.testing.assert_array_equal(host(out), oracle.hasf(X, 3))


def test_out_aliases_in(ctx):
    X = case_image(8, 90, 80)
    t = dev(X)
    ctx.smooth(t, 3, out=t)
    np.testing.assert_array_equal(host(t), oracle.hasf(X, 3))


# --- batch, gang mode, launch shapes --------------------------------------------------

def _mixed_jobs():
    jobs = []
    for i, (h, w) in enumerate(SIZES + [(200, 150), (513, 511)]):
        X = case_image(100 + i, h, w)
        C = synth.constraint_points(i, X, 6) if i % 2 else None
        jobs.append((X, 1 + i % 5, C, 8 if i % 3 else 4))
    return jobs


def test_batch_equals_oracle_per_image(ctx):
    from paper_1603_09337_gb300 import Image
    jobs = _mixed_jobs()
    imgs = [Image(dev(X), r, C=dev(C) if C is not None else None, conn=cn) for X, r, C, cn in jobs]
    outs = ctx.smooth_batch(imgs)
    ctx.status()
    for (X, r, C, cn), o in zip(jobs, outs):
        np.testing.assert_array_equal(host(o), oracle.hasf(X, r, C=C, conn=cn))


def test_batch_order_does_not_matter(ctx):
    from paper_1603_09337_gb300 import Image
    jobs = _mixed_jobs()
    perm = np.random.default_rng(3).permutation(len(jobs))
    a = ctx.smooth_batch([Image(dev(j[0]), j[1], conn=j[3]) for j in jobs])
    b = ctx.smooth_batch([Image(dev(jobs[k][0]), jobs[k][1], conn=jobs[k][3]) for k in perm])
    for pos, k in enumerate(perm):
        np.testing.assert_array_equal(host(a[k]), host(b[pos]))


@pytest.mark.parametrize("gang", [1, 3, 8])
def test_gang_mode_equals_oracle(ctx, gang):
    ctx.set_option(_lib.OPT_FORCE_GANG, 1)
    ctx.set_option(_lib.OPT_GANG_CTAS, gang)
    try:
        for i, (h, w) in enumerate([(31, 33), (130, 70), (257, 300)]):
            X = case_image(200 + i, h, w)
            C = synth.constraint_points(i, X, 4)
            got = host(ctx.smooth(dev(X), 3, C=dev(C), conn=8 if i % 2 == 0 else 4))
            ctx.status()
            np.testing.assert_array_equal(got, oracle.hasf(X, 3, C=C, conn=8 if i % 2 == 0 else 4))
    finally:
        ctx.set_option(_lib.OPT_FORCE_GANG, 0)
        ctx.set_option(_lib.OPT_GANG_CTAS, 0)


def test_full_batch_equals_oracle(ctx):
    """The benchmark's launch: 256 images of 512 x 512, rmax 5, 50 kept points
    each, one batched launch; every image equals the oracle."""
    from paper_1603_09337_gb300 import Image
    from tests._oracle_threads import hasf_many
    jobs = synth.batch_512(256)
    imgs = [Image(dev(j.X), j.rmax, C=dev(j.C)) for j in jobs]
    outs = ctx.smooth_batch(imgs)
    ctx.status()
    want = hasf_many([(j.X, j.rmax, j.C, None, 8) for j in jobs])
    for k, (o, w) in enumerate(zip(outs, want)):
        np.testing.assert_array_equal(host(o), w, err_msg=f"image {k}")


def test_single_image_workload_equals_oracle(ctx):
    """The single-image workload: one 512 x 512 image (12 shapes, 6 holes,
    5 % noise), rmax 3, no constraint set, one hasf_smooth launch."""
    job = synth.single_512()
    got = host(ctx.smooth(dev(job.X), job.rmax))
    ctx.status()
    np.testing.assert_array_equal(got, oracle.hasf(job.X, job.rmax))


# --- host-buffer path, errors ---------------------------------------------------------

def test_host_buffers(ctx):
    jobs = _mixed_jobs()[:6]
    outs = [np.zeros_like(X) for X, *_ in jobs]
    ctx.smooth_host([(X, r, C, None, cn, o) for (X, r, C, cn), o in zip(jobs, outs)])
    for (X, r, C, cn), o in zip(jobs, outs):
        np.testing.assert_array_equal(o, oracle.hasf(X, r, C=C, conn=cn))


def test_host_buffers_pinned_mapped_and_staged(ctx):
    """Pinned host buffers, some with padded rows, one job pageable: read and
    written by the kernels in place (direct access, the default), moved by
    the library's copy kernel over the mapping, or by one copy per buffer;
    the results equal the oracle and the row padding is left untouched."""
    import torch
    jobs = _mixed_jobs()[:6]
    for mapped in (2, 1, 0):
        ctx.set_option(_lib.OPT_HOST_MAPPED, mapped)
        specs, pads = [], []
        for k, (X, r, C, cn) in enumerate(jobs):
            h, w = X.shape
            pitch = w + 16 * (k % 3)
            def buf(fill):
                b = torch.full((h, pitch), fill, dtype=torch.uint8)
                return (b.pin_memory() if k != 5 else b).numpy()
            bx, bo = buf(0), buf(7)
            bx[:, :w] = X
            bc = None
            if C is not None:
                bc = buf(0)
                bc[:, :w] = C
            specs.append((bx[:, :w], r, None if bc is None else bc[:, :w], None, cn, bo[:, :w]))
            pads.append(bo)
        ctx.smooth_host(specs)
        for (X, r, C, cn), bo in zip(jobs, pads):
            w = X.shape[1]
            np.testing.assert_array_equal(bo[:, :w], oracle.hasf(X, r, C=C, conn=cn))
            assert (bo[:, w:] == 7).all()
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    wide = [case_image(400 + i, 96 + 64 * i, 512 - 128 * i) for i in range(3)]
    xs = [case_image(300 + i, 40 + i, 70 - i) for i in range(40)]
    for mapped in (1, 2):
        ctx.set_option(_lib.OPT_HOST_MAPPED, mapped)
        # rows of whole 16-byte chunks: the copy kernel's vector path
        hw = [pin(x) for x in wide]
        hwo = [pin(np.zeros_like(x)) for x in wide]
        ctx.smooth_host([(x, 2, None, None, 8, o) for x, o in zip(hw, hwo)])
        for x, o in zip(wide, hwo):
            np.testing.assert_array_equal(o, oracle.hasf(x, 2))
        # forty pinned images in one call
        hx = [pin(x) for x in xs]
        ho = [pin(np.zeros_like(x)) for x in xs]
        ctx.smooth_host([(x, 1 + i % 3, None, None, 8, o) for i, (x, o) in enumerate(zip(hx, ho))])
        for i, (x, o) in enumerate(zip(xs, ho)):
            np.testing.assert_array_equal(o, oracle.hasf(x, 1 + i % 3), err_msg=f"image {i}")


def test_invalid_arguments(ctx):
    import ctypes
    X = dev(np.zeros((8, 8), np.uint8))
    lib = ctx.lib
    for kw in [dict(width=0), dict(height=70000), dict(pitch=4), dict(rmax=0), dict(rmax=65),
               dict(connectivity=6), dict(reserved=1)]:
        d = _lib.HasfImage(X.data_ptr(), X.data_ptr(), None, None, 8, 8, 8, 2, 8, 0)
        for k, v in kw.items():
            setattr(d, k, v)
        assert lib.hasf_smooth(ctx.h, ctypes.byref(d), None) == _lib.HASF_EINVAL, kw
    d = _lib.HasfImage(None, X.data_ptr(), None, None, 8, 8, 8, 2, 8, 0)
    assert lib.hasf_smooth(ctx.h, ctypes.byref(d), None) == _lib.HASF_EINVAL


def test_round_cap_reports_timeout(ctx):
    """A device iteration cap of one round per level must surface as
    HASF_ETIMEOUT on the host (no GPU fault involved)."""
    X = synth.single_512().X
    ctx.set_option(_lib.OPT_ROUND_CAP, 1)
    try:
        ctx.smooth(dev(X), 3)
        with pytest.raises(_lib.HasfError) as e:
            ctx.status()
        assert e.value.code == _lib.HASF_ETIMEOUT
    finally:
        ctx.set_option(_lib.OPT_ROUND_CAP, 0)
    got = host(ctx.smooth(dev(X), 1))   # the context stays usable
    ctx.status()
    np.testing.assert_array_equal(got, oracle.hasf(X, 1))


def test_budget_too_small(ctx):
    from paper_1603_09337_gb300 import Context
    small = Context(0, budget_bytes=4096)
    try:
        X = dev(np.zeros((512, 512), np.uint8))
        with pytest.raises(_lib.HasfError) as e:
            small.smooth(X, 2)
        assert e.value.code == _lib.HASF_EBUDGET
    finally:
        small.close()


# --- large images (gang mode) and ragged batches ---------------------------------------

def test_large_image_exact_2048(ctx):
    """A 2048 x 2048 image of the large-image workload's kind (discs and
    ellipses of semi-axes 5-200, 3 % noise), rmax 10: sixteen tiles, one
    thread-block cluster; equal to the oracle."""
    X = synth.shapes_image(synth.image_seed(2, 2048), 2048, 2048, 250, 5, 200, n_holes=0,
                           jitter=0, noise_permille=30)
    got = host(ctx.smooth(dev(X), 10))
    ctx.status()
    np.testing.assert_array_equal(got, oracle.hasf(X, 10))


def test_extreme_aspect_ratios(ctx):
    """Images at the width and height limits of the tiled paths: one row of
    65,536 pixels (128 tiles, a tiled gang), 3 x 40,000 and 40,000 x 3."""
    for h, w in [(1, 65536), (3, 40000), (40000, 3)]:
        X = synth.small_random(h * 7 + w, w, h, 550)
        got = host(ctx.smooth(dev(X), 2))
        ctx.status()
        np.testing.assert_array_equal(got, oracle.hasf(X, 2), err_msg=f"{h}x{w}")


@pytest.mark.parametrize("side", [4096, 8192])
def test_large_image_equals_stored_oracle(ctx, side):
    """The 4096^2 / 8192^2 workloads at rmax 10 (tiled gangs of 64 / 256
    CTAs), pixel by pixel against the oracle's result, which takes the oracle
    minutes and is therefore stored under tests/golden by
    make_large_golden.py; a second run gives the same bytes."""
    from tests.golden.make_large_golden import expected
    job = synth.large_image(side)
    want = expected(side)
    t = dev(job.X)
    a = host(ctx.smooth(t, job.rmax))
    b = host(ctx.smooth(t, job.rmax))
    ctx.status()
    diff = np.argwhere(a != want)
    assert len(diff) == 0, f"{len(diff)} pixels differ, first (y, x): {diff[:5].tolist()}"
    np.testing.assert_array_equal(a, b)


def test_ragged_batch_equals_oracle(ctx):
    """A ragged batch of the mixed-size workload (sides 128-2048, rmax 1-8):
    64 images in one call, every image against the oracle."""
    from paper_1603_09337_gb300 import Image
    from tests._oracle_threads import hasf_many
    jobs = synth.ragged_batch(64)
    imgs = [Image(dev(j.X), j.rmax) for j in jobs]
    outs = ctx.smooth_batch(imgs)
    ctx.status()
    want = hasf_many([(j.X, j.rmax, None, None, 8) for j in jobs])
    for k, (o, w) in enumerate(zip(outs, want)):
        np.testing.assert_array_equal(host(o), w, err_msg=f"image {k} {jobs[k].X.shape}")
