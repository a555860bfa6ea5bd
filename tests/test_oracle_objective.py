"""Pins of the oracle's objective, adjoint gradient and update (Sec. "Methodology").

The adjoint gradient is compared with central finite differences of J(rho)
(which also fixes its sign, see the reading of the operator form of the
gradient), and the projected step with hand-worked values.
"""

import numpy as np
import pytest

from oracle import convolution as C
from oracle import objective as O
from oracle import optimizer as P
from paper_1707_09898_gb300 import workloads as W


@pytest.mark.parametrize("m0_kind,w,ht", [("const", (0.0, 0.0, 1.0), "const"), ("vmf", (1.0, 1.0, 1.0), "normal"),
                                          ("vmf", (0.5, 0.0, 2.0), "const")])
@pytest.mark.parametrize("p", [3.0, 1.5])
def test_gradient_matches_central_differences(m0_kind, w, ht, p):
    wl = W.small((6, 5, 8), 5, cellsize=(1e-3, 0.7e-3, 1.2e-3), m0_kind=m0_kind, w=w, ht_kind=ht)
    g = C.Geometry(wl.n_out, wl.nzd, wl.cellsize)
    op = C.FFTOperator(g)
    rho = wl.rho().astype(np.float64) * 0.8 + 0.1
    M0 = wl.M0_field().astype(np.float64)
    Ht = wl.Ht_field().astype(np.float64)
    mask = wl.mask()
    J, G, _ = O.objective_and_gradient(op, rho, M0, p, mask, Ht, w)
    rng = np.random.default_rng(5)
    flat = rng.choice(rho.size, size=12, replace=False)
    h = 1e-4
    for f in flat:
        idx = np.unravel_index(f, rho.shape)
        rp, rm = rho.copy(), rho.copy()
        rp[idx] += h
        rm[idx] -= h
        Jp = O.objective(op.forward(O.magnetization(rp, M0, p)), mask, Ht, w)
        Jm = O.objective(op.forward(O.magnetization(rm, M0, p)), mask, Ht, w)
        fd = (Jp - Jm) / (2 * h)
        assert G[idx] == pytest.approx(fd, rel=1e-6, abs=1e-8 * np.abs(G).max())


def test_objective_and_dJdH_on_a_hand_case():
    H = np.zeros((3, 1, 1, 2))
    H[:, 0, 0, 0] = [1.0, 2.0, 3.0]
    H[:, 0, 0, 1] = [5.0, 5.0, 5.0]
    mask = np.array([[[1, 0]]], dtype=np.uint8)
    Ht = np.array([0.5, 0.0, 1.0])
    w = (2.0, 0.0, 1.0)
    assert O.objective(H, mask, Ht, w) == pytest.approx(2 * 0.25 + 0 + 4.0)
    g = O.dJ_dH(H, mask, Ht, w)
    np.testing.assert_allclose(g[:, 0, 0, 0], [2.0, 0.0, 4.0])
    np.testing.assert_allclose(g[:, 0, 0, 1], 0.0)


def test_projected_gradient_step_hand_case():
    rho = np.array([0.5, 0.95, 0.02, 0.3])
    G = np.array([-2.0, -4.0, 1.0, 0.0])
    out = P.projected_gradient_step(rho, G, 0.1, normalize=True)
    np.testing.assert_allclose(out, [0.55, 1.0, 0.0, 0.3])
    out = P.projected_gradient_step(rho, G, 0.01, normalize=False)
    np.testing.assert_allclose(out, [0.52, 0.99, 0.01, 0.3])
    np.testing.assert_array_equal(P.projected_gradient_step(rho, np.zeros(4), 0.1), rho)


def test_optimizer_reduces_objective():
    wl = W.small((8, 8, 10), 8)
    g = C.Geometry(wl.n_out, wl.nzd, wl.cellsize)
    op = C.FFTOperator(g)
    rho0 = np.full(wl.design_shape, 0.5)
    _, hist = P.optimize(op, rho0, wl.M0_const(), 3.0, wl.mask(), wl.Ht_const_vec(), wl.w, iters=15, alpha=0.05)
    assert hist[-1] < 0.5 * hist[0]
