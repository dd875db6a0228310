"""The C-ABI library builds (nvcc, sm_103a only), loads, and exports every entry point include/lsd.h declares
(no compute calls: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lsd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsd_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_02455_b300 import build
    path = build.build()
    from paper_2606_02455_b300 import lsd
    return path, lsd.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lsd_init", "lsd_draft_window", "lsd_verify_window", "lsd_step", "lsd_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    path, L = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lsd_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        getattr(L, n)


def test_binding_covers_every_symbol():
    from paper_2606_02455_b300 import lsd
    assert sorted(lsd.SYMBOLS) == _declared()


def test_strerror_names_codes(lib):
    _, L = lib
    assert L.lsd_strerror(0) == b"ok"
    assert b"neighbour" in L.lsd_strerror(-7)
    assert L.lsd_strerror(-999) == b"unknown error"


def test_init_rejects_bad_arguments_without_a_gpu(lib):
    """Argument validation happens before any CUDA call: a NULL system is LSD_EINVAL."""
    import ctypes
    _, L = lib
    h = ctypes.c_void_p()
    assert L.lsd_init(None, None, None, 0.01, 1.0, 300.0, 8, ctypes.byref(h)) == -1
    assert L.lsd_init(None, None, None, 0.01, 1.0, 300.0, 8, None) == -1
