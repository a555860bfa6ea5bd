"""The allocation-free projected-gradient step gives the same rho as tm_optimize_step.

tm_optimize_step_noalloc serves callers that must not allocate device memory
when they call in (a caching allocator that has reserved the device, or a
time-critical loop that cannot absorb cudaMalloc's implicit synchronisation).
Its scratch is a static device array shared by every call, so this checks two
calls in a row (the second with fewer elements, over the first call's leftover
scratch contents), the unnormalised form, a zero gradient, and the size limit.
One case also goes straight to the float64 oracle's projected-gradient step.
This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
MAX_N = 33_554_432


@pytest.fixture(scope="module")
def env():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1707_09898_gb300 import Magnet, _lib

    return Magnet, _lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)


def test_noalloc_step_matches_context_step(env):
    Magnet, _lib = env
    L = _lib.lib()
    rng = np.random.default_rng(12)
    # larger grid first, then a smaller one: the second call reads only the scratch slots it wrote
    for n_out, nzd, alpha, normalize in [((64, 48, 40), 36, 0.1, True), ((20, 12, 10), 7, 0.05, True),
                                         ((20, 12, 10), 7, 0.02, False)]:
        m = Magnet(n_out, nzd, tensor=False)
        shape = m.design_shape
        rho = torch.from_numpy(rng.random(shape, dtype=np.float64).astype(np.float32)).to(DEV)
        G = torch.from_numpy(rng.normal(size=shape).astype(np.float32)).to(DEV)
        ref = rho.clone()
        m.optimize_step(ref, G, alpha, normalize)
        new = rho.clone()
        rc = L.tm_optimize_step_noalloc(_p(new), _p(G), new.numel(), alpha, int(normalize), _stream())
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.equal(new, ref), float((new - ref).abs().max())
        m.close()


def test_noalloc_step_matches_oracle(env):
    """The step against oracle.optimizer.projected_gradient_step on the same float32 inputs:
    the float32 step alpha / max|G| and one rounding per update, so within a few float32
    ulps of rho (<= 1) of the float64 result; the clip to [0, 1] is exact on both sides."""
    from oracle import optimizer as P

    _, _lib = env
    L = _lib.lib()
    rng = np.random.default_rng(21)
    for n, alpha, normalize in [(70_001, 0.1, True), (70_001, 0.05, False), (3, 0.3, True)]:
        rho_np = rng.random(n, dtype=np.float64).astype(np.float32)
        G_np = (rng.normal(size=n) * (0.2 if not normalize else 1e11)).astype(np.float32)
        rho, G = torch.from_numpy(rho_np).to(DEV), torch.from_numpy(G_np).to(DEV)
        for _ in range(2):  # two calls in a row over the scratch the first one left
            out = rho.clone()
            assert L.tm_optimize_step_noalloc(_p(out), _p(G), n, alpha, int(normalize), _stream()) == 0
            torch.cuda.synchronize()
        ref = P.projected_gradient_step(rho_np, G_np, alpha, normalize)
        err = np.abs(out.cpu().numpy().astype(np.float64) - ref).max()
        assert err <= 4 * 2.0**-24, (n, normalize, err)
        assert ((out >= 0) & (out <= 1)).all()


def test_noalloc_zero_gradient_and_size_limit(env):
    _, _lib = env
    L = _lib.lib()
    rho = torch.rand(1000, device=DEV)
    keep = rho.clone()
    G = torch.zeros_like(rho)
    assert L.tm_optimize_step_noalloc(_p(rho), _p(G), rho.numel(), 0.1, 1, _stream()) == 0
    torch.cuda.synchronize()
    assert torch.equal(rho, keep)
    # beyond the static scratch: rejected before any launch
    assert L.tm_optimize_step_noalloc(_p(rho), _p(G), MAX_N + 1, 0.1, 1, _stream()) == -2
    assert L.tm_optimize_step_noalloc(None, _p(G), 10, 0.1, 1, _stream()) == -1
