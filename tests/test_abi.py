"""The C-ABI library builds, loads and exports every entry point include/c8r.h
declares (no GPU needed); argument validation answers before any device work."""
import ctypes
import os
import re
import subprocess

import pytest

from _util import built_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "c8r.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(c8r_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = built_lib()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (c8r_[a-z_0-9]+)$", out, flags=re.M))
    names = declared()
    assert len(names) >= 20
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    built_lib()
    from paper_2309_03717_gb300 import c8r
    lib = c8r.load()
    assert sorted(c8r.exported_names()) == declared()
    for n in declared():
        assert hasattr(lib, n)


def test_host_side_validation_without_device_work():
    built_lib()
    from paper_2309_03717_gb300 import c8r
    lib = c8r.load()
    h = ctypes.c_void_p()
    assert lib.c8r_create(ctypes.byref(h), 100000) == c8r.C8R_EINVAL
    assert h.value is None
    assert b"no CUDA device" in lib.c8r_last_error(None)
    assert lib.c8r_create(None, 0) == c8r.C8R_EINVAL
    assert lib.c8r_set_medium(None, 0, 1.0, 1.0) == c8r.C8R_EINVAL
    assert lib.c8r_push_tracks(None, None, 0, None) == c8r.C8R_EINVAL
    assert lib.c8r_measure_peaks(0, None) == c8r.C8R_EINVAL
    assert lib.c8r_set_deposit(None, c8r.C8R_DEPOSIT_LINEAR) == c8r.C8R_EINVAL
    # the generator validates its arguments before any launch
    out = c8r.c8r_tracks(c8r.C8R_F32, *([None] * 12))
    assert lib.c8r_generate_tracks(1, 0, 10, 0.0, None, None) == c8r.C8R_EINVAL
    assert lib.c8r_generate_tracks(1, 0, 10, 0.0, ctypes.byref(out), None) == c8r.C8R_EINVAL  # NULL arrays
    assert lib.c8r_generate_tracks(1, -1, 10, 0.0, ctypes.byref(out), None) == c8r.C8R_EINVAL
    assert lib.c8r_generate_tracks(1, 0, -1, 0.0, ctypes.byref(out), None) == c8r.C8R_EINVAL
    assert lib.c8r_generate_tracks(1, 0, 10, float("nan"), ctypes.byref(out), None) == c8r.C8R_EINVAL
    lib.c8r_destroy(None)  # accepted
    assert lib.c8r_batch_create(None, 0, None, 0, 1.0, 1.0) == c8r.C8R_EINVAL


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2309_03717_gb300 import c8r
    saved = c8r._lib
    c8r._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            c8r.load(str(tmp_path / "missing.so"))
    finally:
        c8r._lib = saved
