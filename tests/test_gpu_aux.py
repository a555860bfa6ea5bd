"""Failure detection, fault injection, input validation, logging and checkpoint/resume
on the GPU, with no GPU fault: a bounded wait that runs out on purpose, an injected
host-side failure, a rejected density, and a resumed run compared bit for bit."""

import json

import numpy as np
import pytest
import torch

from paper_1707_09898_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


def prepared(wl):
    from paper_1707_09898_gb300 import Magnet

    m = Magnet(wl.n_out, wl.nzd, wl.cellsize, M0=wl.M0_const(), p=wl.p, device=0)
    m.set_target(torch.from_numpy(wl.mask()).to(DEV), Ht_const=tuple(float(v) for v in wl.Ht_const_vec()), w=wl.w)
    return m


def test_bounded_wait_runs_out_and_is_reported():
    from paper_1707_09898_gb300 import _lib

    wl = W.config1()
    m = prepared(wl)
    rho = torch.from_numpy(wl.rho()).to(DEV)
    J0, G0 = m.evaluate(rho)
    # a wait on an mbarrier phase that nothing completes: it gives up after 300 polls
    assert m.selftest_wait_timeout(300) == -6
    assert "bounded wait" in _lib.lib().tm_last_error(m.h).decode()
    # the status word was cleared and the context still works
    J1, G1 = m.evaluate(rho)
    assert J1 == J0 and torch.equal(G1, G0)
    assert m.selftest_wait_timeout(0) == -1


def test_injected_failure_leaves_the_context_usable():
    from paper_1707_09898_gb300 import _lib

    L = _lib.lib()
    wl = W.config1()
    m = prepared(wl)
    rho = torch.from_numpy(wl.rho()).to(DEV)
    J0, G0 = m.evaluate(rho)
    L.tm_inject_fault(b"tm_evaluate", 2)
    J1, _ = m.evaluate(rho)
    with pytest.raises(_lib.TopomagError) as e:
        m.evaluate(rho)
    assert e.value.code == -7
    J2, G2 = m.evaluate(rho)
    assert J0 == J1 == J2 and torch.equal(G2, G0)
    # a call made inside another entry point does not count: tm_evaluate_step runs
    # tm_evaluate internally, and only the caller's own tm_evaluate calls fail
    L.tm_inject_fault(b"tm_evaluate", 1)
    G = G0.clone()
    r = rho.clone()
    m.evaluate_step(r, G, 0.1)
    with pytest.raises(_lib.TopomagError):
        m.evaluate(rho)
    L.tm_inject_fault(None, 0)


def test_invalid_density_is_rejected():
    from paper_1707_09898_gb300 import _lib

    wl = W.config1()
    m = prepared(wl)
    rho = torch.from_numpy(wl.rho()).to(DEV)
    assert m.check_design(rho) == 0
    for bad in (float("nan"), -0.01, 1.5):
        r = rho.clone()
        r[3, 4, 5] = bad
        with pytest.raises(_lib.TopomagError) as e:
            m.check_design(r)
        assert e.value.code == -1 and "1 of 4096" in str(e.value)


def test_log_and_bitwise_resume(tmp_path):
    from paper_1707_09898_gb300 import optimize

    wl = W.config2()
    cfg = {"workload": wl.name, "alpha": wl.alpha}
    k, extra = 7, 6
    a = optimize.Run(prepared(wl), wl.rho(), wl.alpha, cfg, log=str(tmp_path / "a.jsonl"))
    a.step(k + extra)
    b = optimize.Run(prepared(wl), wl.rho(), wl.alpha, cfg)
    b.step(k)
    b.save(str(tmp_path / "ck.npz"))
    c = optimize.Run.resume(prepared(wl), str(tmp_path / "ck.npz"), config=cfg)
    assert c.k == k
    c.step(extra)
    assert torch.equal(c.rho, a.rho)
    assert c.history == a.history
    with pytest.raises(ValueError):
        optimize.Run.resume(prepared(wl), str(tmp_path / "ck.npz"), config={"workload": "another"})
    # the log: one line per evaluation, the quantities of the final density
    lines = [json.loads(x) for x in open(tmp_path / "a.jsonl")]
    assert [x["k"] for x in lines] == list(range(k + extra + 1))
    assert [x["J"] for x in lines] == a.history
    r = a.rho.cpu().numpy()
    assert abs(lines[-1]["volume_fraction"] - r.astype(np.float64).mean()) <= 1e-12
    assert lines[-1]["intermediate_fraction"] == np.mean((r > np.float32(0.1)) & (r < np.float32(0.9)))
    assert lines[-1]["grad_max"] == float(a.G.abs().max())


def test_chosen_fft_lengths_are_checked():
    """tm_set_grid_lengths: a length that is not supported or below 2 n is refused and the
    grid stays as it was; 0 keeps the default of that axis."""
    from paper_1707_09898_gb300 import Magnet, _lib

    lib = _lib.lib()
    m = Magnet((20, 24, 10), 6, device=0, tensor=False)
    assert m.fft_lengths() == (48, 48, 24)  # the smallest supported L >= 2 n
    cell = _lib.c_double3(1e-3, 1e-3, 1e-3)
    for L in ((50, 48, 24), (36, 48, 24), (48, 48, 576 * 2)):
        assert lib.tm_set_grid_lengths(m.h, _lib.c_int3(20, 24, 10), 6, cell, _lib.c_int3(*L)) == -2, L
        assert m.fft_lengths() == (48, 48, 24)
    assert lib.tm_set_grid_lengths(m.h, _lib.c_int3(20, 24, 10), 6, cell, _lib.c_int3(64, 0, 32)) == 0
    assert m.fft_lengths() == (64, 48, 32)
    # the default for 2 n in (256, 512) is 512
    m2 = Magnet((130, 150, 192), 8, device=0, tensor=False)
    assert m2.fft_lengths() == (512, 512, 512)
