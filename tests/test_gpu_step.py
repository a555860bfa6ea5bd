"""tm_evaluate_step: one projected-gradient iteration per call (the step on the gradient
of the previous evaluation, then the evaluation at the new rho). It must give the same
rho, dJ/drho and J, bit for bit, as tm_optimize_step followed by tm_evaluate, both where
the step runs inside the x forward pass (512-point x transforms of one spectrum) and
where it runs as its own pass (other lengths, varying M0)."""

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


def magnet(wl):
    from paper_1707_09898_gb300 import Magnet

    M0 = torch.from_numpy(wl.M0_field()).to(DEV) if wl.m0_kind != "const" else wl.M0_const()
    m = Magnet(wl.n_out, wl.nzd, wl.cellsize, M0=M0, p=wl.p, device=0)
    m.set_target(torch.from_numpy(wl.mask()).to(DEV), Ht_const=tuple(float(v) for v in wl.Ht_const_vec()), w=wl.w)
    return m


CASES = {
    "x512_fused": lambda: W.small((230, 14, 10), 9, seed=81),
    "x512_ragged_rows": lambda: W.small((200, 11, 7), 5, seed=82),
    "x48_separate_step": lambda: W.small((20, 230, 7), 6, seed=83),
    "vmf_separate_step": lambda: W.small((14, 11, 13), 9, seed=84, m0_kind="vmf"),
    "throughput_256": lambda: W.config4(256),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("mode", ["reuse_max", "recompute_max", "plain"])
def test_evaluate_step_equals_step_then_evaluate(case, mode):
    if case == "throughput_256" and mode != "reuse_max":
        pytest.skip("one mode at full size")
    wl = CASES[case]()
    m = magnet(wl)
    normalize, reuse = {"reuse_max": (True, True), "recompute_max": (True, False), "plain": (False, False)}[mode]
    rho0 = torch.from_numpy(wl.rho()).to(DEV)

    rho1 = rho0.clone()
    G1 = torch.empty_like(rho1)
    J1, _ = m.evaluate(rho1, G=G1)
    alpha = 0.1 if normalize else 0.1 / float(G1.abs().max())
    Js1 = []
    for _ in range(3):
        m.optimize_step(rho1, G1, alpha, normalize, reuse_max=reuse)
        J1, _ = m.evaluate(rho1, G=G1)
        Js1.append(J1)

    rho2 = rho0.clone()
    G2 = torch.empty_like(rho2)
    m.evaluate(rho2, G=G2)
    Js2 = []
    for _ in range(3):
        J2, _ = m.evaluate_step(rho2, G2, alpha, normalize, reuse_max=reuse)
        Js2.append(J2)

    assert not torch.equal(rho2, rho0)  # the steps moved rho
    assert torch.equal(rho1, rho2)
    assert torch.equal(G1, G2)
    assert Js1 == Js2


def test_zero_gradient_leaves_rho():
    """max|G| = 0 with normalisation: no step (as tm_optimize_step), then the evaluation."""
    wl = CASES["x512_fused"]()
    m = magnet(wl)
    rho = torch.from_numpy(wl.rho()).to(DEV)
    r0 = rho.clone()
    G = torch.zeros_like(rho)
    J, _ = m.evaluate_step(rho, G, 0.1, True, reuse_max=False)
    assert torch.equal(rho, r0)
    J_ref, G_ref = m.evaluate(r0)
    assert J == J_ref and torch.equal(G, G_ref)


def test_non_contiguous_arrays_are_refused():
    wl = CASES["x512_fused"]()
    m = magnet(wl)
    nzd, ny, nx = wl.design_shape
    big = torch.zeros((nzd, ny, 2 * nx), dtype=torch.float32, device=DEV)
    rho = big[:, :, :nx]
    with pytest.raises(ValueError):
        m.evaluate_step(rho, torch.zeros((nzd, ny, nx), dtype=torch.float32, device=DEV), 0.1)
