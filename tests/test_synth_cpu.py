"""The seeded input generators are part of the workload definitions: the same
seed gives the same bytes on every machine (integer SplitMix64, exact integer
shape tests).  These digests pin that; a change to a generator must change
them on purpose."""
from __future__ import annotations

import hashlib

from paper_1603_09337_gb300 import synth


def digest(a) -> str:
    return hashlib.sha256(a.tobytes()).hexdigest()[:16]


def test_workload_generators_are_reproducible():
    assert digest(synth.single_512(0).X) == "1a3149952a5a7b52"
    b = synth.batch_512(2)
    assert digest(b[1].X) == "6c4f1c7245a909a6"
    assert digest(b[1].C) == "cf397bafaa9ff185"
    r = synth.ragged_batch(2)
    assert r[0].X.shape == (523, 1708) and r[0].rmax == 2
    assert digest(r[0].X) == "e37b37c7e5046236"
    assert r[1].X.shape == (1364, 1627) and r[1].rmax == 5
    assert digest(synth.volume(11, 12, 13, 40, 3, 2, 5, 40)) == "55993b7704d24608"
    assert digest(synth.small_random(5, 33, 17, 300)) == "051b23b747f922e9"


def test_generators_make_binary_images():
    j = synth.single_512(3)
    assert j.X.dtype.name == "uint8" and set(j.X.ravel().tolist()) <= {0, 1}
    assert 0.05 < j.X.mean() < 0.95
