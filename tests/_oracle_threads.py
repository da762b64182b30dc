"""Run the CPU oracle on many images at once, one thread per host core.

The oracle's C functions keep no global state, and ctypes releases the GIL
while a foreign call runs, so plain threads use every core.  Threads (rather
than processes) also keep this safe to use after the CUDA runtime has started
in the test process.  Test infrastructure only.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle


def hasf_many(jobs, threads: int | None = None) -> list[np.ndarray]:
    """oracle.hasf on every (X, rmax, C, D, conn) of `jobs`, in order; the
    largest images are started first so that the cores finish together."""
    order = sorted(range(len(jobs)), key=lambda i: -jobs[i][0].size * max(1, abs(jobs[i][1])))
    out: list = [None] * len(jobs)

    def run(i):
        X, rmax, C, D, conn = jobs[i]
        out[i] = oracle.hasf(X, rmax, C=C, D=D, conn=conn)

    with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
        list(ex.map(run, order))
    return out
