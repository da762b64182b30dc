"""The stored oracle results of the large single-image workloads
(tests/golden/large_<side>_r10.*, written by make_large_golden.py from the
oracle alone) decode, match their checksums, and have the properties the
filter guarantees: the numbers of 8-components of the object and of
4-components of the background (outside included) are those of the input."""
from __future__ import annotations

import json

import numpy as np
import pytest

from paper_1603_09337_gb300 import synth
from tests import _brute as B
from tests.golden.make_large_golden import expected, paths


@pytest.mark.parametrize("side", [4096, 8192])
def test_stored_large_result(side):
    meta = json.load(open(paths(side)[1]))
    out = expected(side)                     # raises if the checksum does not match
    X = synth.large_image(side).X
    assert int((out != X).sum()) == meta["changed_pixels"]
    assert int(out.sum()) == meta["object_pixels_out"]
    assert set(np.unique(out)) <= {0, 1}
    assert B.component_counts(out) == B.component_counts(X)
