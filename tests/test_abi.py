"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/epic_interp.h (no GPU needed: nothing is computed)."""

import ctypes
import os
import re

import pytest

from paper_1501_02565_gb300 import build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "epic_interp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(epic_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return native.load()


def test_header_declares_the_documented_entry_points():
    names = declared_functions()
    assert set(names) == set(native.EXPORTED)
    for core in ("epic_interp_create", "epic_interp_run", "epic_interp_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_status_codes_match_header():
    text = open(HEADER).read()
    for name, val in re.findall(r"(EPIC_\w+)\s*=\s*(\d+)", text):
        assert getattr(native, name) == int(val)


def test_config_struct_layout_matches_defaults(lib):
    cfg = native.epic_config_default()
    assert cfg.max_W == 1024 and cfg.max_H == 436
    assert cfg.weight_squared == 1 and cfg.max_degree == 32
    assert abs(cfg.fallback_eps - 1e-10) < 1e-16
    assert cfg.apron == -1 and cfg.max_passes == 4096


def test_null_handle_is_rejected_without_a_gpu(lib):
    assert lib.epic_interp_sync(None) == native.EPIC_ERR_INVALID
    assert lib.epic_interp_last_error(None) == b"null handle"
    out = ctypes.c_void_p()
    # create with a null output pointer is an argument error, not a CUDA call
    assert lib.epic_interp_create(None, 0, None) == native.EPIC_ERR_INVALID


def test_library_is_built_for_sm_103a_only():
    src = open(os.path.join(ROOT, "paper_1501_02565_gb300", "build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in src
