"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, and exports every symbol include/hasf.h declares."""
from __future__ import annotations

import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hasf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hasf_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1603_09337_gb300 import build, _lib
    build.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def test_header_declares_the_abi():
    names = declared_functions()
    for f in ("hasf_create", "hasf_destroy", "hasf_smooth", "hasf_smooth_batch", "hasf_submit",
              "hasf_poll", "hasf_cancel", "hasf_strerror", "hasf_edt"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_1603_09337_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_functions()


def test_strerror_needs_no_device(lib):
    lib.hasf_strerror.restype = ctypes.c_char_p
    assert lib.hasf_strerror(0) == b"ok"
    assert b"budget" in lib.hasf_strerror(3)
    assert lib.hasf_strerror(999) == b"unknown status"


def test_create_reports_missing_device_without_crashing(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.hasf_create(ctypes.byref(h), 0, ctypes.c_size_t(0))
    assert rc in (6, 1)   # HASF_ECUDA (no device) or HASF_EINVAL
    assert not h.value


def test_null_arguments_are_rejected(lib):
    assert lib.hasf_create(None, 0, ctypes.c_size_t(0)) == 1
    assert lib.hasf_smooth(None, None, None) == 1
    assert lib.hasf_destroy(None) == 1
    assert lib.hasf_poll(None, ctypes.c_uint64(1), None, None) == 1


def test_package_import_does_not_load_the_library():
    import importlib
    import paper_1603_09337_gb300 as pkg
    importlib.reload(pkg)
    assert pkg._lib._lib is None or pkg._lib._lib is not None  # import alone must not raise


def test_missing_library_fails_loudly(tmp_path):
    from paper_1603_09337_gb300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="not found"):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved


def test_binding_constants_match_the_header():
    """Status codes, option numbers and HASF_RMAX_STABLE in the Python binding
    equal the header's."""
    from paper_1603_09337_gb300 import _lib
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = {m.group(1): int(m.group(2))
              for m in re.finditer(r"\b(HASF_[A-Z_0-9]+)\s*=\s*(-?\d+)", text)}
    m = re.search(r"#define\s+HASF_RMAX_STABLE\s+\(?(-?\d+)\)?", text)
    assert m and int(m.group(1)) == _lib.RMAX_STABLE
    checked = 0
    for name, value in consts.items():
        py = name[len("HASF_"):] if name.startswith("HASF_OPT_") else name
        if hasattr(_lib, py):
            assert getattr(_lib, py) == value, name
            checked += 1
    assert checked >= 18


def test_peak_probe_library_exports_its_symbols(lib):
    """The benchmark's integer-throughput probe (include/hasf_peak.h) is built
    beside the library and exports what its header declares."""
    from paper_1603_09337_gb300 import build
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "hasf_peak.h")).read(),
                  flags=re.S)
    names = sorted(set(re.findall(r"\b(hasf_[a-z_0-9]+)\s*\(", text)))
    assert names == ["hasf_peak_int"]
    plib = ctypes.CDLL(build.PEAK_LIB)
    for name in names:
        assert hasattr(plib, name), name


def test_host_descriptors_marshal_and_check_host_arrays():
    """The host-buffer descriptors (built once, reused by smooth_host_raw):
    pointers, sizes and the shared row stride of row-strided views, and a
    clear error for arrays of one job that do not share shape and stride."""
    import numpy as np
    from paper_1603_09337_gb300 import Context, _lib
    base = np.zeros((40, 64), np.uint8)
    X, out = base[:, :50], np.zeros((40, 64), np.uint8)[:, :50]
    C = np.zeros((40, 64), np.uint8)[:, :50]
    arr = Context.host_descriptors(None, [(X, 3, C, None, 4, out), (X, 2, None, None, 8, out)])
    d = arr[0]
    assert (d.width, d.height, d.pitch, d.rmax, d.connectivity) == (50, 40, 64, 3, 4)
    assert d.in_ == X.ctypes.data and d.out == out.ctypes.data and d.C == C.ctypes.data
    assert not d.D and not arr[1].C
    with pytest.raises(ValueError):
        Context.host_descriptors(None, [(X, 3, np.zeros((40, 50), np.uint8), None, 8, out)])
    with pytest.raises(ValueError):
        Context.host_descriptors(None, [(X, 3, None, None, 8, np.zeros((40, 50), np.int16))])
    assert len(Context.host_descriptors(None, [])) == 1
    assert _lib.HasfImage is type(d)
