#!/usr/bin/env python3
"""Write the oracle's result for the large single-image workloads.

The large workloads are one 4096 x 4096 or 8192 x 8192 image of 2,000 seeded
discs and ellipses (semi-axes 5-200) with 3 % salt-and-pepper noise, filtered
by HASF with rmax = 10, (8,4) adjacency and no constraint sets.  The CPU oracle
takes minutes on such an image, too long for a GPU test to recompute, so this
script runs it once and stores the result next to itself:

  large_<side>_r10.xz    the pixels the filter changed (oracle output XOR
                         input), np.packbits row-major, lzma-compressed; the
                         test regenerates the input from its seed and applies
                         the XOR to get the expected image;
  large_<side>_r10.json  seed, size, rmax, the number of changed pixels, the
                         SHA-256 of np.packbits(expected) and this command.

Only ``oracle`` (the plain CPU restatement of the method) and the input
generator ``synth`` are called; nothing here comes from the CUDA library.

  python tests/golden/make_large_golden.py 4096 [8192 ...]
"""
from __future__ import annotations

import hashlib
import json
import lzma
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1603_09337_gb300 import synth  # noqa: E402

RMAX = 10


def paths(side: int) -> tuple[str, str]:
    base = os.path.join(HERE, f"large_{side}_r{RMAX}")
    return base + ".xz", base + ".json"


def expected(side: int) -> np.ndarray:
    """The stored oracle result of the large workload of this side (uint8 0/1)."""
    xz, meta_path = paths(side)
    meta = json.load(open(meta_path))
    job = synth.large_image(side)
    assert job.meta["seed"] == meta["seed"] and job.rmax == meta["rmax"]
    X = (job.X != 0).astype(np.uint8)
    diff = np.unpackbits(np.frombuffer(lzma.decompress(open(xz, "rb").read()), np.uint8),
                         count=side * side).reshape(side, side)
    out = X ^ diff
    if hashlib.sha256(np.packbits(out).tobytes()).hexdigest() != meta["sha256_packbits"]:
        raise ValueError(f"{xz}: stored result does not match its checksum")
    return out


def make(side: int) -> dict:
    job = synth.large_image(side)
    assert job.rmax == RMAX and job.C is None
    X = (job.X != 0).astype(np.uint8)
    t0 = time.perf_counter()
    out = oracle.hasf(X, RMAX)
    dt = time.perf_counter() - t0
    diff = out ^ X
    xz, meta_path = paths(side)
    with open(xz, "wb") as f:
        f.write(lzma.compress(np.packbits(diff).tobytes(), preset=9 | lzma.PRESET_EXTREME))
    meta = {
        "workload": f"{side}x{side}, 2,000 discs/ellipses (semi-axes 5-200), 3% noise, "
                    f"rmax={RMAX}, (8,4) adjacency, C = D = empty",
        "generator": f"paper_1603_09337_gb300.synth.large_image({side})",
        "seed": job.meta["seed"], "width": side, "height": side, "rmax": RMAX, "conn": 8,
        "changed_pixels": int(diff.sum()), "object_pixels_in": int(X.sum()),
        "object_pixels_out": int(out.sum()),
        "sha256_packbits": hashlib.sha256(np.packbits(out).tobytes()).hexdigest(),
        "oracle_seconds": round(dt, 1),
        "command": f"python tests/golden/make_large_golden.py {side}",
    }
    with open(meta_path, "w") as f:
        json.dump(meta, f, indent=1)
        f.write("\n")
    return meta


if __name__ == "__main__":
    for s in sys.argv[1:] or ["4096"]:
        print(json.dumps(make(int(s))), flush=True)
