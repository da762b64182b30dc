"""The continuous-batching server (hasf_submit / hasf_poll / hasf_cancel).

Requests arrive while others run; the server admits them by the byte budget,
batches them into launches on several streams, and each result must be the
same bytes as hasf_smooth on that image alone.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

from paper_1603_09337_gb300 import _lib, synth
from tests._oracle_threads import hasf_many

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_09337_gb300 import build
    build.build()
    return torch


def _stream_jobs(n, seed=11):
    rng = synth.SplitMix64(seed)
    jobs = []
    for i in range(n):
        w, h = rng.randint(40, 700), rng.randint(40, 700)
        X = synth.shapes_image(seed * 1000 + i, w, h, max(1, w * h // 20000), 4,
                               max(5, min(w, h) // 4), n_holes=1, hole_lo=2, hole_hi=5,
                               jitter=1, noise_permille=rng.randint(20, 100))
        jobs.append((X, rng.randint(1, 6)))
    return jobs


def _wait(ctx, tickets, timeout=120.0):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets):
        for t in tickets:
            if t in done:
                continue
            d, st = ctx.poll(t)
            if d:
                done[t] = st
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.001)
    return done


def test_served_results_equal_solo_results(torch_cuda):
    torch = torch_cuda
    from paper_1603_09337_gb300 import Context
    jobs = _stream_jobs(40)
    with Context(0) as ctx:
        ins = [torch.from_numpy(X).cuda() for X, _ in jobs]
        solo = []
        for t, (X, r) in zip(ins, jobs):
            solo.append(ctx.smooth(t, r))
        ctx.status()
        outs = [torch.zeros_like(t) for t in ins]
        tickets = []
        for k, ((X, r), t, o) in enumerate(zip(jobs, ins, outs)):
            tickets.append(ctx.submit(t, r, o))
            if k % 7 == 3:
                time.sleep(0.002)       # arrivals spread while batches run
        st = _wait(ctx, tickets)
        assert all(v == _lib.HASF_OK for v in st.values())
        torch.cuda.synchronize()
        for o, s in zip(outs, solo):
            np.testing.assert_array_equal(o.cpu().numpy(), s.cpu().numpy())
        want = hasf_many([(X, r, None, None, 8) for X, r in jobs])
        for i, w in enumerate(want):
            np.testing.assert_array_equal(outs[i].cpu().numpy(), w, err_msg=f"job {i}")


def test_poll_cancel_and_errors(torch_cuda):
    torch = torch_cuda
    from paper_1603_09337_gb300 import Context
    with Context(0) as ctx:
        ctx.set_option(_lib.OPT_SERVE_STREAMS, 1)
        ctx.set_option(_lib.OPT_SERVE_BATCH, 1)
        X = torch.from_numpy(synth.large_image(2048).X[:1024, :1024].copy()).cuda()
        outs = [torch.zeros_like(X) for _ in range(6)]
        tickets = [ctx.submit(X, 8, o) for o in outs]
        # the last one is still queued behind five slow jobs on one stream
        assert ctx.cancel(tickets[-1]) in (_lib.HASF_OK, _lib.HASF_EPENDING)
        st = _wait(ctx, tickets)
        assert st[tickets[-1]] in (_lib.HASF_ECANCELLED, _lib.HASF_OK)
        assert all(st[t] == _lib.HASF_OK for t in tickets[:-1])
        with pytest.raises(_lib.HasfError) as e:
            ctx.poll(tickets[0])               # already reported
        assert e.value.code == _lib.HASF_ENOTFOUND
        assert ctx.cancel(123456789) == _lib.HASF_ENOTFOUND
    with Context(0, budget_bytes=1 << 16) as small:
        big = torch.zeros((2048, 2048), dtype=torch.uint8, device="cuda")
        with pytest.raises(_lib.HasfError) as e:
            small.submit(big, 3, torch.zeros_like(big))
        assert e.value.code == _lib.HASF_EBUDGET


def test_drain_and_destroy_with_work_in_flight(torch_cuda):
    torch = torch_cuda
    from paper_1603_09337_gb300 import Context
    jobs = _stream_jobs(12, seed=5)
    ctx = Context(0)
    ins = [torch.from_numpy(X).cuda() for X, _ in jobs]
    outs = [torch.zeros_like(t) for t in ins]
    tickets = [ctx.submit(t, r, o) for (X, r), t, o in zip(jobs, ins, outs)]
    ctx.drain()
    for t in tickets:
        d, st = ctx.poll(t)
        assert d and st == _lib.HASF_OK
    more = [ctx.submit(t, r, o) for (X, r), t, o in zip(jobs, ins, outs)]
    assert more
    ctx.close()                                 # cancels or finishes, never hangs
