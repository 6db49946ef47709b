"""Host-side checks of the C ABI that need no GPU: the library loads, exports every entry point
include/seg.h declares, the binding covers them all, and argument errors are reported before any
device work."""
import ctypes
import os
import re

import pytest

from paper_1912_11494_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(seg_\w+)\s*\(", text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1912_11494_gb300 import build
    build.build()
    return binding.lib()


def test_header_declares_entry_points():
    names = declared()
    for must in ("seg_create_atlas", "seg_destroy_atlas", "seg_label", "seg_label_batch",
                 "seg_grad", "seg_status_string", "seg_sync_status", "seg_apply_affine"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), f"libseg.so does not export {name}"


def test_binding_covers_every_declared_symbol():
    assert {n for n, _, _ in binding.SIGNATURES} == declared()


def test_status_strings(lib):
    for code, name in binding.STATUS_NAMES.items():
        assert lib.seg_status_string(code).decode() == name


def test_argument_errors_before_device_work(lib):
    h = ctypes.c_void_p()
    assert lib.seg_create_atlas(None, None, None, 10, 2, 21, None, ctypes.byref(h)) == 1
    assert b"NULL" in lib.seg_last_error()
    assert lib.seg_create_atlas(1, 1, 1, 0, 2, 21, None, ctypes.byref(h)) == 1
    assert lib.seg_create_atlas(1, 1, 1, 10, 2, 20, None, ctypes.byref(h)) == 1
    assert lib.seg_create_atlas(1, 1, 1, 10, 2, 21, None, None) == 1
    assert lib.seg_label(None, None, 0, 0, None, None, None, None, None) == 1
    assert lib.seg_label_batch(None, 0, None, None, 0, None, None, None) == 1
    assert lib.seg_label_host(None, None, 0, 0, None, None, None) == 1
    assert lib.seg_set_gemm_record_cap(None, 0) == 1
    assert lib.seg_grad(None, None, 0, None, None, None, None, None, None, None) == 1
    assert lib.seg_sync_status(None, None) == 1
    assert lib.seg_destroy_atlas(None) == 0
    assert lib.seg_apply_affine(None, -1, None, None, None) == 1
    assert lib.seg_apply_affine(None, 0, None, None, None) == 1
    assert lib.seg_gemm_stats(None, None, None, None, None, None) == 1
    assert lib.seg_resample(None, None, -1, None, None) == 1
    assert lib.seg_resample(None, None, 0, None, None) == 0
    assert lib.seg_resample(None, None, 5, None, None) == 1
    assert lib.seg_label_streamlines(None, None, None, 0, 0, None, None, None, None, None) == 1
    assert lib.seg_set_classification(None, 0) == 1
    # a float buffer that is not 4-byte aligned is refused before it is touched
    aff = (ctypes.c_double * 12)()
    assert lib.seg_apply_affine(ctypes.c_void_p(0x1002), 1, aff, ctypes.c_void_p(0x2000),
                                None) == 1
    assert b"aligned" in lib.seg_last_error()


def test_modes_match_the_header(lib):
    """binding.MODES names every seg_mode the header declares, with its value; every mode has at
    least one tile configuration and an unknown mode has none (host-side query)."""
    text = open(os.path.join(ROOT, "include", "seg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    enum = {m.group(1).lower(): int(m.group(2))
            for m in re.finditer(r"SEG_MODE_(\w+)\s*=\s*(\d+)", text)}
    assert enum == binding.MODES
    for name, value in enum.items():
        n = lib.seg_num_configs(value)
        assert n >= 1, name
        if name in ("plain_culled", "culled_fused"):
            assert n == 1
    assert lib.seg_num_configs(max(enum.values()) + 1) == 0
