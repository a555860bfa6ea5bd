"""The C-ABI library builds for sm_103a, loads, and exports every symbol of include/topomag.h (no GPU needed)."""

import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1707_09898_gb300 import _lib

    return _lib


def test_exports_every_declared_function(lib):
    names = lib.header_functions()
    assert len(names) >= 14
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing
    assert set(lib._SIGS) == set(names), "binding signatures out of sync with the header"


def test_version_string(lib):
    assert lib.lib().tm_version().decode().startswith("topomag")


def test_null_handles_are_rejected(lib):
    L = lib.lib()
    assert L.tm_create(None, 0) == -1
    assert L.tm_set_grid(None, lib.c_int3(8, 8, 8), 8, lib.c_double3(1, 1, 1)) == -1
    assert L.tm_last_error(None) == b"null context"
