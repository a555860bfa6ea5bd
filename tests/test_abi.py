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


def test_fault_injection_hook_without_a_gpu(lib):
    """The nth call of the armed entry point fails with TM_ERR_INJECTED before any work;
    the calls around it behave as without the hook (here: a null context, TM_ERR_ARG)."""
    L = lib.lib()
    assert L.tm_inject_fault(b"tm_set_penalty", 2) == 0
    codes = [L.tm_set_penalty(None, 3.0) for _ in range(4)]
    assert codes == [-1, -7, -1, -1]
    L.tm_inject_fault(b"tm_set_penalty", 1)
    assert L.tm_set_fused(None, 1) == -1  # another entry point: not armed
    assert L.tm_set_penalty(None, 3.0) == -7
    L.tm_inject_fault(b"tm_set_penalty", 3)
    L.tm_inject_fault(None, 0)  # disarmed
    assert [L.tm_set_penalty(None, 3.0) for _ in range(4)] == [-1] * 4


def test_fault_injection_from_the_environment(lib):
    """TM_FAULT_INJECT=<call>:<nth> arms the hook when the library loads (a fresh process)."""
    import os
    import subprocess
    import sys

    code = ("import ctypes, sys; L = ctypes.CDLL(sys.argv[1]); "
            "L.tm_set_penalty.argtypes = [ctypes.c_void_p, ctypes.c_double]; "
            "print([L.tm_set_penalty(None, 3.0) for _ in range(3)])")
    env = dict(os.environ, TM_FAULT_INJECT="tm_set_penalty:3")
    out = subprocess.run([sys.executable, "-c", code, lib.LIB_PATH], env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "[-1, -1, -7]"


def test_default_padding_without_a_gpu(lib):
    """tm_set_grid's padded length per axis: the smallest supported even 2^a 3^b >= 2 n,
    with 288 and 384 replaced by 512 (any L >= 2 n is the same linear convolution); the
    cuFFT comparison pipeline keeps the smallest length itself."""
    from paper_1707_09898_gb300.cufft_pipeline import plain_length

    L = lib.lib()
    want = {1: 8, 4: 8, 5: 12, 10: 24, 17: 36, 60: 128, 100: 256, 128: 256, 129: 512, 144: 512,
            150: 512, 192: 512, 200: 512, 256: 512, 257: 576, 288: 576}
    for n, Lx in want.items():
        assert L.tm_default_fft_length(n) == Lx, n
        assert Lx >= 2 * n
    assert L.tm_default_fft_length(0) == 0 and L.tm_default_fft_length(289) == 0
    assert [plain_length(n) for n in (5, 17, 129, 150, 192, 256)] == [12, 36, 288, 384, 384, 512]
