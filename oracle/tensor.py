"""Oracle: the discrete demagnetization tensor (float64, numpy).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

The paper (Sec. "Discretization", Eq. (demag_tensor)) defines the tensor as
the six-fold cell-cell integral of the second derivatives of 1/|x - x'|,
normalised by the cell volume, depending only on the index difference i - j.
It leaves the evaluation to the micromagnetic literature it cites. This module
uses the conventional sign (positive self-term; a cube gives 1/3 on the
diagonal) so that the field is H = -sum_j N(i-j) m_j; the paper writes the
same operator with the minus folded into N.

Evaluation rule (identical in meaning on the CUDA side, implemented twice):

* near field, integer offset with max(|i|,|j|,|k|) <= R_NEAR: the exact
  closed form of Newell, Williams and Dunlop (1993) -- second differences of
  the functions f (diagonal) and g (off-diagonal) with weights
  (-1, 2, -1) per axis, divided by 4*pi*V;
* far field: the cell-cell average of the point-dipole kernel
  K(r) = (delta/|r|^3 - 3 r r^T/|r|^5) / (4 pi), times V, by a 3-node
  tensor-product rule on the triangular (tent) distribution of the
  centre-to-centre separation. The rule reproduces the tent's moments of
  order 0..5 exactly, so its error is O((d/|R|)^6).

Components are ordered (xx, yy, zz, xy, xz, yz). Their parities under
reflection of one axis: the diagonal is even in x, y and z; xy is odd in x and
y; xz odd in x and z; yz odd in y and z. Hence N(-R) = N(R).
"""

import numpy as np

COMPONENTS = ("xx", "yy", "zz", "xy", "xz", "yz")
# odd[c] = (odd in x, odd in y, odd in z)
ODD = {
    "xx": (False, False, False),
    "yy": (False, False, False),
    "zz": (False, False, False),
    "xy": (True, True, False),
    "xz": (True, False, True),
    "yz": (False, True, True),
}
# (row, col) of each component in the symmetric 3x3 tensor
INDEX = {"xx": (0, 0), "yy": (1, 1), "zz": (2, 2), "xy": (0, 1), "xz": (0, 2), "yz": (1, 2)}

R_NEAR = 16

# 3-node rule for E[phi(w)] with w tent-distributed on [-d, d]:
# nodes 0 and +-sqrt(2/5) d, weights 7/12 and 5/24 (moments 1, d^2/6, d^4/15).
_TENT_NODE = np.sqrt(0.4)
_TENT_W = (5.0 / 24.0, 7.0 / 12.0, 5.0 / 24.0)


def _arr(*a):
    return [np.asarray(v, dtype=np.float64) for v in np.broadcast_arrays(*a)]


def _flat(*a):
    """Broadcast to a common shape and return (shape, 1-D float64 copies)."""
    b = _arr(*a)
    return b[0].shape, [v.reshape(-1).copy() for v in b]


def newell_f(x, y, z):
    """Newell's f(x, y, z): even in every argument (Newell et al. 1993, Eq. 27)."""
    shape, (x, y, z) = _flat(x, y, z)
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    out = (2.0 * x2 - y2 - z2) * R / 6.0
    rxz = np.sqrt(x2 + z2)
    rxy = np.sqrt(x2 + y2)
    m = (y > 0) & (rxz > 0)
    out[m] += 0.5 * y[m] * (z2[m] - x2[m]) * np.arcsinh(y[m] / rxz[m])
    m = (z > 0) & (rxy > 0)
    out[m] += 0.5 * z[m] * (y2[m] - x2[m]) * np.arcsinh(z[m] / rxy[m])
    m = (x > 0) & (y > 0) & (z > 0)
    out[m] -= x[m] * y[m] * z[m] * np.arctan(y[m] * z[m] / (x[m] * R[m]))
    return out.reshape(shape)


def newell_g(x, y, z):
    """Newell's g(x, y, z): odd in x and in y, even in z (Newell et al. 1993, Eq. 32)."""
    shape, (x, y, z) = _flat(x, y, z)
    sgn = np.sign(x) * np.sign(y)
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    out = -x * y * R / 3.0
    nz = (x > 0) & (y > 0)  # g vanishes identically when x = 0 or y = 0
    rxy = np.sqrt(x2 + y2)
    ryz = np.sqrt(y2 + z2)
    rxz = np.sqrt(x2 + z2)
    m = nz
    out[m] += x[m] * y[m] * z[m] * np.arcsinh(z[m] / rxy[m])
    out[m] += y[m] / 6.0 * (3.0 * z2[m] - y2[m]) * np.arcsinh(x[m] / ryz[m])
    out[m] += x[m] / 6.0 * (3.0 * z2[m] - x2[m]) * np.arcsinh(y[m] / rxz[m])
    m = nz & (z > 0)
    out[m] -= z2[m] * z[m] / 6.0 * np.arctan(x[m] * y[m] / (z[m] * R[m]))
    out[m] -= z[m] * y2[m] / 2.0 * np.arctan(x[m] * z[m] / (y[m] * R[m]))
    out[m] -= z[m] * x2[m] / 2.0 * np.arctan(y[m] * z[m] / (x[m] * R[m]))
    return (sgn * out).reshape(shape)


_SD_W = {-1: -1.0, 0: 2.0, 1: -1.0}


def _second_difference(fun, a, b, c, da, db, dc):
    acc = np.zeros(np.broadcast(a, b, c).shape)
    for ea in (-1, 0, 1):
        for eb in (-1, 0, 1):
            for ec in (-1, 0, 1):
                w = _SD_W[ea] * _SD_W[eb] * _SD_W[ec]
                acc += w * fun(a + ea * da, b + eb * db, c + ec * dc)
    return acc


def newell_tensor(X, Y, Z, cellsize):
    """Exact cell-averaged tensor at physical offsets (X, Y, Z): shape (6, ...)."""
    dx, dy, dz = (float(v) for v in cellsize)
    X, Y, Z = _arr(X, Y, Z)
    k = 1.0 / (4.0 * np.pi * dx * dy * dz)
    return np.stack([
        k * _second_difference(newell_f, X, Y, Z, dx, dy, dz),  # xx
        k * _second_difference(newell_f, Y, X, Z, dy, dx, dz),  # yy
        k * _second_difference(newell_f, Z, Y, X, dz, dy, dx),  # zz
        k * _second_difference(newell_g, X, Y, Z, dx, dy, dz),  # xy
        k * _second_difference(newell_g, X, Z, Y, dx, dz, dy),  # xz
        k * _second_difference(newell_g, Y, Z, X, dy, dz, dx),  # yz
    ])


def dipole_kernel(X, Y, Z):
    """Point-dipole kernel K(r) = (delta/r^3 - 3 r r^T / r^5)/(4 pi): shape (6, ...)."""
    X, Y, Z = _arr(X, Y, Z)
    r2 = X * X + Y * Y + Z * Z
    r = np.sqrt(r2)
    i3 = 1.0 / (r2 * r)
    i5 = 3.0 * i3 / r2
    c = 1.0 / (4.0 * np.pi)
    return c * np.stack([
        i3 - i5 * X * X,
        i3 - i5 * Y * Y,
        i3 - i5 * Z * Z,
        -i5 * X * Y,
        -i5 * X * Z,
        -i5 * Y * Z,
    ])


def far_tensor(X, Y, Z, cellsize):
    """Tent-averaged dipole kernel times V (far-field rule): shape (6, ...)."""
    dx, dy, dz = (float(v) for v in cellsize)
    X, Y, Z = _arr(X, Y, Z)
    acc = np.zeros((6,) + X.shape)
    for a, wa in zip((-1, 0, 1), _TENT_W):
        for b, wb in zip((-1, 0, 1), _TENT_W):
            for c, wc in zip((-1, 0, 1), _TENT_W):
                acc += (wa * wb * wc) * dipole_kernel(
                    X + a * _TENT_NODE * dx, Y + b * _TENT_NODE * dy, Z + c * _TENT_NODE * dz)
    return acc * (dx * dy * dz)


def normalized_cellsize(cellsize):
    """The tensor is invariant under uniform scaling; evaluate with max(d) = 1."""
    d = np.asarray(cellsize, dtype=np.float64)
    return d / d.max()


def demag_tensor(i, j, k, cellsize):
    """N at integer cell offsets (i, j, k), near/far switch at R_NEAR: shape (6, ...)."""
    d = normalized_cellsize(cellsize)
    i, j, k = (np.asarray(v, dtype=np.int64) for v in np.broadcast_arrays(i, j, k))
    out = np.zeros((6,) + i.shape)
    near = np.maximum(np.maximum(np.abs(i), np.abs(j)), np.abs(k)) <= R_NEAR
    if near.any():
        out[:, near] = newell_tensor(i[near] * d[0], j[near] * d[1], k[near] * d[2], d)
    far = ~near
    if far.any():
        out[:, far] = far_tensor(i[far] * d[0], j[far] * d[1], k[far] * d[2], d)
    return out


def tensor_octant(n, cellsize, chunk=1 << 22):
    """N at every offset of the non-negative octant [0,nx) x [0,ny) x [0,nz).

    Returns float64 array (6, nz, ny, nx); the other octants follow from ODD.
    """
    nx, ny, nz = (int(v) for v in n)
    out = np.empty((6, nz, ny, nx))
    plane = nx * ny
    zs_per = max(1, chunk // max(plane, 1))
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for z0 in range(0, nz, zs_per):
        z1 = min(nz, z0 + zs_per)
        zz = np.arange(z0, z1)[:, None, None] + np.zeros((1, ny, nx), dtype=np.int64)
        out[:, z0:z1] = demag_tensor(np.broadcast_to(xx, zz.shape), np.broadcast_to(yy, zz.shape), zz, cellsize)
    return out


def tensor_lookup(octant, di, dj, dk):
    """N(di, dj, dk) for arbitrary-sign integer offsets from an octant table: (6, ...)."""
    di, dj, dk = (np.asarray(v, dtype=np.int64) for v in np.broadcast_arrays(di, dj, dk))
    vals = octant[:, np.abs(dk), np.abs(dj), np.abs(di)]
    sx, sy, sz = np.where(di < 0, -1.0, 1.0), np.where(dj < 0, -1.0, 1.0), np.where(dk < 0, -1.0, 1.0)
    for c, name in enumerate(COMPONENTS):
        ox, oy, oz = ODD[name]
        s = 1.0
        if ox:
            s = s * sx
        if oy:
            s = s * sy
        if oz:
            s = s * sz
        if not np.isscalar(s):
            vals[c] = vals[c] * s
    return vals


def fft_length(n):
    """Padded FFT length per axis: the smallest 2^a 3^b >= 2 n (zero padding to 2n)."""
    target = 2 * int(n)
    best = None
    p2 = 1
    while p2 < 4 * target:
        v = p2
        while v < target:
            v *= 3
        if best is None or v < best:
            best = v
        p2 *= 2
    return best


def padded_tensor(n_out, L, cellsize, octant=None):
    """The L-periodic real arrays holding N at offsets |R_a| <= n_a - 1, zeros elsewhere.

    Returns float64 (6, Lz, Ly, Lx). Requires L_a >= 2 n_a - 1 per axis.
    """
    nx, ny, nz = (int(v) for v in n_out)
    Lx, Ly, Lz = (int(v) for v in L)
    assert Lx >= 2 * nx - 1 and Ly >= 2 * ny - 1 and Lz >= 2 * nz - 1
    if octant is None:
        octant = tensor_octant((nx, ny, nz), cellsize)
    out = np.zeros((6, Lz, Ly, Lx))

    def slots(n, Lax):
        # slot s holds offset o(s): s for s < n, s - L for s > L - n
        s = np.concatenate([np.arange(n), np.arange(Lax - n + 1, Lax)])
        o = np.concatenate([np.arange(n), np.arange(-(n - 1), 0)])
        return s, o

    sx, ox = slots(nx, Lx)
    sy, oy = slots(ny, Ly)
    sz, oz = slots(nz, Lz)
    OZ, OY, OX = np.meshgrid(oz, oy, ox, indexing="ij")
    vals = tensor_lookup(octant, OX, OY, OZ)
    out[np.ix_(np.arange(6), sz, sy, sx)] = vals
    return out
