"""Pins of the oracle's demagnetization tensor (Sec. "Discretization", Eq. (demag_tensor)).

None of these re-types the oracle's formulas: each compares against an
independent fact -- a closed form (cube 1/3, Aharoni's prism formula), an
identity of the six-fold integral (trace, parity, additivity over cells), a
separately coded Gauss-Legendre quadrature of the defining integral, or the
point-dipole limit.
"""

import numpy as np
import pytest
from scipy.special import roots_legendre

from oracle import tensor as T


def aharoni_z(a, b, c):
    """Demagnetizing factor along z of a 2a x 2b x 2c prism (Aharoni, J. Appl. Phys. 83, 3432 (1998))."""
    r = np.sqrt(a * a + b * b + c * c)
    ab, bc, ac = np.sqrt(a * a + b * b), np.sqrt(b * b + c * c), np.sqrt(a * a + c * c)
    t = ((b * b - c * c) / (2 * b * c) * np.log((r - a) / (r + a))
         + (a * a - c * c) / (2 * a * c) * np.log((r - b) / (r + b))
         + b / (2 * c) * np.log((ab + a) / (ab - a)) + a / (2 * c) * np.log((ab + b) / (ab - b))
         + c / (2 * a) * np.log((bc - b) / (bc + b)) + c / (2 * b) * np.log((ac - a) / (ac + a))
         + 2 * np.arctan(a * b / (c * r)) + (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r + c / (a * b) * (ac + bc)
         - (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c))
    return t / np.pi


def tent_rule(d, n):
    """Gauss-Legendre nodes/weights for E[h(w)], w with density (d-|w|)/d^2 on [-d, d]."""
    x, wt = roots_legendre(n)
    w = d * (1 + x) / 2
    ww = wt * d / 2 * (d - w) / d ** 2
    return np.concatenate([w, -w]), np.concatenate([ww, ww])


def quadrature_tensor(R, d, n=24):
    """N(R) = V E[K(R + w)] by brute-force tensor-product quadrature of the definition."""
    nx, wx = tent_rule(d[0], n)
    ny, wy = tent_rule(d[1], n)
    nz, wz = tent_rule(d[2], n)
    X = R[0] + nx[:, None, None]
    Y = R[1] + ny[None, :, None]
    Z = R[2] + nz[None, None, :]
    r2 = X * X + Y * Y + Z * Z
    r = np.sqrt(r2)
    W = wx[:, None, None] * wy[None, :, None] * wz[None, None, :]
    base = 1.0 / (4 * np.pi)
    comp = {
        "xx": 1 / r ** 3 - 3 * X * X / r ** 5, "yy": 1 / r ** 3 - 3 * Y * Y / r ** 5,
        "zz": 1 / r ** 3 - 3 * Z * Z / r ** 5, "xy": -3 * X * Y / r ** 5,
        "xz": -3 * X * Z / r ** 5, "yz": -3 * Y * Z / r ** 5,
    }
    V = d[0] * d[1] * d[2]
    return np.array([base * V * np.sum(comp[c] * W) for c in T.COMPONENTS])


def test_cube_self_term_is_one_third():
    N = T.demag_tensor(0, 0, 0, (1e-3, 1e-3, 1e-3))
    np.testing.assert_allclose(N[:3], 1.0 / 3.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(N[3:], 0.0, atol=1e-15)


@pytest.mark.parametrize("d", [(1.0, 2.0, 3.0), (0.3, 0.3, 1.0), (2.0, 1.0, 0.25)])
def test_prism_self_term_matches_aharoni(d):
    N = T.newell_tensor(0.0, 0.0, 0.0, d)
    a, b, c = d[0] / 2, d[1] / 2, d[2] / 2
    ref = np.array([aharoni_z(b, c, a), aharoni_z(c, a, b), aharoni_z(a, b, c)])
    np.testing.assert_allclose(N[:3], ref, rtol=1e-12)
    assert abs(N[:3].sum() - 1.0) < 1e-13
    np.testing.assert_allclose(N[3:], 0.0, atol=1e-15)


@pytest.mark.parametrize("ijk", [(1, 0, 0), (1, 1, 0), (3, 2, 1), (0, 5, 7), (16, 3, 2), (17, 3, 2), (40, 9, 1)])
@pytest.mark.parametrize("d", [(1.0, 1.0, 1.0), (1.0, 0.5, 2.0)])
def test_trace_vanishes_off_origin(ijk, d):
    N = T.demag_tensor(*ijk, d)
    # FP64 second differences lose digits with distance (about 5e-9 at 28 small-cell edges)
    assert abs(N[:3].sum()) < 2e-8 * np.abs(N).max()


def test_parity_under_reflection():
    d = (1.0, 0.7, 1.3)
    base = T.demag_tensor(3, 2, 5, d)
    for sx in (1, -1):
        for sy in (1, -1):
            for sz in (1, -1):
                N = T.demag_tensor(3 * sx, 2 * sy, 5 * sz, d)
                for c, name in enumerate(T.COMPONENTS):
                    ox, oy, oz = T.ODD[name]
                    s = (sx if ox else 1) * (sy if oy else 1) * (sz if oz else 1)
                    assert N[c] == pytest.approx(s * base[c], rel=0, abs=1e-9 * np.abs(base).max())


@pytest.mark.parametrize("R", [(2, 0, 0), (2, 1, 1), (3, 2, 1), (0, 2, 3), (5, -3, 2), (-4, 4, -2)])
@pytest.mark.parametrize("d", [(1.0, 1.0, 1.0), (1.0, 0.5, 2.0)])
def test_newell_matches_independent_quadrature(R, d):
    dn = T.normalized_cellsize(d)
    Rp = np.array(R) * dn
    q = quadrature_tensor(Rp, dn)
    N = T.demag_tensor(*R, d)
    np.testing.assert_allclose(N, q, rtol=0, atol=1e-10 * np.abs(q).max())


@pytest.mark.parametrize("R", [(17, 0, 0), (17, 3, 2), (20, 10, 5), (30, -7, 1), (64, 20, 33)])
def test_far_rule_matches_quadrature(R):
    d = (1.0, 1.0, 1.0)
    q = quadrature_tensor(np.array(R, float), d, n=16)
    N = T.demag_tensor(*R, d)
    np.testing.assert_allclose(N, q, rtol=0, atol=1e-8 * np.abs(q).max())


def test_near_far_switch_is_continuous():
    d = (1.0, 1.0, 1.0)
    for R in [(16, 0, 0), (16, 5, 3), (16, 16, 16)]:
        near = T.newell_tensor(*np.array(R, float), d)
        far = T.far_tensor(*np.array(R, float), d)
        np.testing.assert_allclose(far, near, rtol=0, atol=5e-7 * np.abs(near).max())


def test_point_dipole_limit():
    d = (1.0, 1.0, 1.0)
    R = np.array([150.0, -80.0, 60.0])
    N = T.demag_tensor(150, -80, 60, d)
    r = np.linalg.norm(R)
    K = (np.eye(3) / r ** 3 - 3 * np.outer(R, R) / r ** 5) / (4 * np.pi)
    ref = np.array([K[0, 0], K[1, 1], K[2, 2], K[0, 1], K[0, 2], K[1, 2]])
    np.testing.assert_allclose(N, ref, rtol=0, atol=1e-8 * np.abs(ref).max())


@pytest.mark.parametrize("n,d", [((2, 2, 2), (1.0, 1.0, 1.0)), ((3, 2, 1), (1.0, 2.0, 1.5)), ((4, 3, 5), (1.0, 1.0, 0.5))])
def test_box_identity(n, d):
    """(1/|G|) sum_i sum_j N(i - j) equals the self-term of the whole box (additivity of the integral)."""
    nx, ny, nz = n
    idx = np.array([(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)])
    D = idx[:, None, :] - idx[None, :, :]
    N = T.demag_tensor(D[..., 0], D[..., 1], D[..., 2], d).sum(axis=(1, 2)) / len(idx)
    a, b, c = nx * d[0] / 2, ny * d[1] / 2, nz * d[2] / 2
    ref = np.array([aharoni_z(b, c, a), aharoni_z(c, a, b), aharoni_z(a, b, c)])
    np.testing.assert_allclose(N[:3], ref, rtol=1e-11)
    np.testing.assert_allclose(N[3:], 0.0, atol=1e-13)


def test_scale_invariance():
    a = T.demag_tensor(np.arange(-3, 20), 2, 1, (1e-3, 2e-3, 1.5e-3))
    b = T.demag_tensor(np.arange(-3, 20), 2, 1, (1.0, 2.0, 1.5))
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-18)


def test_fft_length():
    got = {n: T.fft_length(n) for n in (1, 4, 8, 16, 17, 18, 32, 64, 66, 72, 128, 192, 256)}
    assert got == {1: 2, 4: 8, 8: 16, 16: 32, 17: 36, 18: 36, 32: 64, 64: 128, 66: 144, 72: 144,
                   128: 256, 192: 384, 256: 512}


def test_padded_tensor_spectrum_is_real():
    n_out, L = (5, 4, 6), (12, 8, 12)
    pad = T.padded_tensor(n_out, L, (1.0, 0.8, 1.2))
    for c in range(6):
        F = np.fft.fftn(pad[c])
        assert np.abs(F.imag).max() < 1e-13 * np.abs(F.real).max()
