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


# ---- quadratic stencil objectives (Sec. "Optimization of field and gradient") ----

def _fd_check(obj, H, picks, h=1e-6):
    J, g = obj(H)
    for idx in picks:
        Hp, Hm = H.copy(), H.copy()
        Hp[idx] += h
        Hm[idx] -= h
        fd = (obj(Hp)[0] - obj(Hm)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(g[idx])), idx
    return J, g


def test_stencil_objective_gradient_by_central_differences():
    from oracle.objective import stencil_objective

    rng = np.random.default_rng(40)
    H = rng.normal(size=(3, 4, 5, 6))
    rows = []
    for k in range(12):
        ents = [(int(rng.integers(3)), int(rng.integers(4)), int(rng.integers(5)), int(rng.integers(6)),
                 float(rng.normal())) for _ in range(int(rng.integers(1, 4)))]
        rows.append((float(rng.normal()), ents))
    rows.append((0.7, [(2, 1, 1, 1, 1.0), (2, 1, 1, 1, 2.0)]))  # a cell twice in one row
    picks = [(e[0], e[1], e[2], e[3]) for _, ents in rows for e in ents]
    J, g = _fd_check(lambda X: stencil_objective(X, rows), H, picks)
    # J is the quadratic form: J(2H) = 4 J(H); g is linear in H
    J2, g2 = stencil_objective(2 * H, rows)
    assert np.isclose(J2, 4 * J) and np.allclose(g2, 2 * g)


def _fg_setup():
    field = np.zeros((12, 12), bool)
    field[3:8, 4:9] = True
    strip = [(y, 3, 1, -1) for y in range(3, 8)] + [(y, 9, 1, 1) for y in range(3, 8)] + \
            [(8, x, 0, 1) for x in range(4, 9)]
    return field, strip


def test_field_gradient_objective_closed_forms_and_differences():
    from oracle.objective import field_gradient_objective

    field, strip = _fg_setup()
    nz, plane, h, beta = 4, 2, 0.5, 1e3
    yy, xx = np.meshgrid(np.arange(12), np.arange(12), indexing="ij")
    # H_z = a + bx x + by y on the plane: dH/dn = sign * slope exactly
    a, bx, by = 0.3, 0.02, -0.05
    H = np.zeros((3, nz, 12, 12))
    H[2, plane] = a + bx * xx * h + by * yy * h
    H[0] = 5.0  # other components play no part
    J, _ = field_gradient_objective(H, plane, field, strip, h, beta)
    n_x = sum(1 for s in strip if s[2] == 1)
    n_y = sum(1 for s in strip if s[2] == 0)
    J_ref = -0.5 * np.sum(H[2, plane][field] ** 2) - 0.5 * beta * (n_x * bx ** 2 + n_y * by ** 2)
    assert np.isclose(J, J_ref, rtol=1e-12)
    # constant field: only the field term
    Hc = np.zeros_like(H)
    Hc[2, plane] = 0.7
    J, _ = field_gradient_objective(Hc, plane, field, strip, h, beta)
    assert np.isclose(J, -0.5 * 0.49 * field.sum())
    # the gradient by central differences at field, strip-neighbour and unrelated cells
    rng = np.random.default_rng(41)
    Hr = rng.normal(size=H.shape)
    picks = [(2, plane, 4, 5), (2, plane, 5, 2), (2, plane, 5, 3), (2, plane, 5, 4), (2, plane, 9, 6),
             (2, plane, 7, 6), (2, plane, 5, 10), (2, plane - 1, 5, 5), (0, plane, 5, 5)]
    _, g = _fd_check(lambda X: field_gradient_objective(X, plane, field, strip, h, beta), Hr, picks)
    assert g[2, plane - 1, 5, 5] == 0 and g[0, plane, 5, 5] == 0


def test_field_gradient_objective_is_a_stencil_objective():
    from oracle.objective import field_gradient_objective, stencil_objective

    field, strip = _fg_setup()
    plane, h, beta = 1, 1.0, 1e5
    rows = [(-0.5, [(2, plane, y, x, 1.0)]) for y, x in zip(*np.nonzero(field))]
    for y, x, axis, sgn in strip:
        dy, dx = (sgn, 0) if axis == 0 else (0, sgn)
        rows.append((-0.5 * beta, [(2, plane, y + dy, x + dx, 1 / (2 * h)), (2, plane, y - dy, x - dx, -1 / (2 * h))]))
    H = np.random.default_rng(42).normal(size=(3, 3, 12, 12))
    J1, g1 = field_gradient_objective(H, plane, field, strip, h, beta)
    J2, g2 = stencil_objective(H, rows)
    assert np.isclose(J1, J2, rtol=1e-13) and np.allclose(g1, g2, rtol=1e-13, atol=1e-9)
