"""Pins of the oracle's stray-field operator and adjoint (Sec. "Discretization", Eq. (convolution)).

The FFT route is compared with plain O(N^2) direct sums (which it must equal:
the FFT only accelerates the same convolution); the field of a single cell is
compared with the physical point-dipole field (sign of H = -N m); the mean
field of a uniformly magnetized box is compared with Aharoni's closed form;
the adjoint is checked by the dot-product identity.
"""

import numpy as np
import pytest

from oracle import convolution as C
from oracle import tensor as T
from tests.test_oracle_tensor import aharoni_z

GEOMS = [
    ((5, 4, 6), 3, (1.0, 1.0, 1.0)),
    ((4, 6, 5), 5, (1e-3, 0.6e-3, 1.4e-3)),
    ((7, 3, 4), 2, (2.0, 1.0, 1.0)),
    ((6, 5, 19), 2, (1.0, 1.0, 1.0)),  # far-field offsets (|dz| > 16) included
]


@pytest.mark.parametrize("n_out,nzd,d", GEOMS)
def test_fft_equals_direct_sum(n_out, nzd, d):
    g = C.Geometry(n_out, nzd, d)
    rng = np.random.default_rng(0)
    M = rng.normal(size=(3,) + g.design_shape)
    gH = rng.normal(size=(3,) + g.out_shape)
    f = C.FFTOperator(g)
    dsum = C.DirectOperator(g, f.octant)
    H1, H2 = f.forward(M), dsum.forward(M)
    assert np.linalg.norm(H1 - H2) <= 1e-12 * np.linalg.norm(H2)
    A1, A2 = f.adjoint(gH), dsum.adjoint(gH)
    assert np.linalg.norm(A1 - A2) <= 1e-12 * np.linalg.norm(A2)


@pytest.mark.parametrize("n_out,nzd,d", GEOMS)
def test_adjoint_dot_product_identity(n_out, nzd, d):
    g = C.Geometry(n_out, nzd, d)
    rng = np.random.default_rng(1)
    m = rng.normal(size=(3,) + g.design_shape)
    q = rng.normal(size=(3,) + g.out_shape)
    f = C.FFTOperator(g)
    lhs = np.sum(q * f.forward(m))
    rhs = np.sum(f.adjoint(q) * m)
    assert abs(lhs - rhs) <= 1e-13 * (np.linalg.norm(q) * np.linalg.norm(f.forward(m)))


def test_single_cell_field_is_a_dipole_field():
    """A single cell magnetized along z: H on the axis is +2m/(4 pi r^3), in the plane -m/(4 pi r^3)."""
    d = 1e-3
    g = C.Geometry((1, 1, 60), 1, (d, d, d))
    M = np.zeros((3,) + g.design_shape)
    Ms = 8e5
    M[2] = Ms
    H = C.FFTOperator(g).forward(M)
    m = Ms * d ** 3
    for k in (30, 45, 59):
        r = k * d
        assert H[2, k, 0, 0] == pytest.approx(2 * m / (4 * np.pi * r ** 3), rel=3e-6)  # cell-averaged vs point dipole: O((d/r)^4)
        assert abs(H[0, k, 0, 0]) < 1e-9 * abs(H[2, k, 0, 0])
    g2 = C.Geometry((60, 1, 1), 1, (d, d, d))
    M2 = np.zeros((3,) + g2.design_shape)
    M2[2, 0, 0, 0] = Ms
    H2 = C.FFTOperator(g2).forward(M2)
    for i in (30, 59):
        r = i * d
        assert H2[2, 0, 0, i] == pytest.approx(-m / (4 * np.pi * r ** 3), rel=3e-6)  # cell-averaged vs point dipole: O((d/r)^4)


@pytest.mark.parametrize("n,d", [((4, 3, 5), (1.0, 1.0, 1.0)), ((6, 4, 2), (1.0, 0.5, 2.0))])
def test_uniform_box_mean_field(n, d):
    """rho = 1, constant M0: the mean of H over the magnet is -N_box M0 (box identity)."""
    g = C.Geometry(n, n[2], d)
    M0 = np.array([0.3, -0.5, 1.0]) * 7e5
    M = np.broadcast_to(M0[:, None, None, None], (3,) + g.design_shape)
    H = C.FFTOperator(g).forward(M)
    a, b, c = n[0] * d[0] / 2, n[1] * d[1] / 2, n[2] * d[2] / 2
    Nbox = np.array([aharoni_z(b, c, a), aharoni_z(c, a, b), aharoni_z(a, b, c)])
    np.testing.assert_allclose(H.mean(axis=(1, 2, 3)), -Nbox * M0, rtol=1e-10)


def test_cellsize_scale_invariance():
    rng = np.random.default_rng(2)
    g1 = C.Geometry((5, 5, 6), 4, (1e-3, 1.5e-3, 1e-3))
    g2 = C.Geometry((5, 5, 6), 4, (1.0, 1.5, 1.0))
    M = rng.normal(size=(3,) + g1.design_shape)
    H1 = C.FFTOperator(g1).forward(M)
    H2 = C.FFTOperator(g2).forward(M)
    assert np.linalg.norm(H1 - H2) <= 1e-12 * np.linalg.norm(H2)


def test_pointwise_sums_match_fft():
    g = C.Geometry((6, 5, 8), 5, (1.0, 1.2, 0.9))
    rng = np.random.default_rng(3)
    M = rng.normal(size=(3,) + g.design_shape)
    q = np.zeros((3,) + g.out_shape)
    support = np.array([(7, 1, 2), (7, 2, 3), (6, 4, 0)])
    for (z, y, x) in support:
        q[:, z, y, x] = rng.normal(size=3)
    f = C.FFTOperator(g)
    H = f.forward(M)
    cells = np.array([(0, 0, 0), (7, 4, 5), (3, 2, 1)])
    got = C.field_at(g, f.octant, M, cells)
    np.testing.assert_allclose(got, H[:, cells[:, 0], cells[:, 1], cells[:, 2]].T, rtol=1e-11, atol=1e-12 * np.abs(H).max())
    A = f.adjoint(q)
    dcells = np.array([(0, 0, 0), (4, 4, 5), (2, 1, 3)])
    got = C.adjoint_at(g, f.octant, q, dcells, support)
    np.testing.assert_allclose(got, A[:, dcells[:, 0], dcells[:, 1], dcells[:, 2]].T, rtol=1e-11, atol=1e-12 * np.abs(A).max())
