"""Oracle: the stray-field operator D and its adjoint (float64, numpy/scipy).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Geometry. The output grid has n_out = (nx, ny, nz) cells; the design box is
its bottom slab z in [0, nzd) with the same nx, ny. rho (and so M) lives on the
design box and is zero outside it; H is wanted on the whole output grid.

Forward (Sec. "Discretization", Eq. (convolution), with the conventional sign):
    H_i = - sum_{j in design} N(i - j) m_j,   i in the output grid.
Adjoint (the same operator with input and output regions exchanged; D is
self-adjoint because N(-R) = N(R) and every N(R) is a symmetric matrix):
    (D^T g)_j = - sum_{i in output} N(j - i) g_i,   j in the design box.

Two independent evaluations are given: a zero-padded float64 FFT (the paper's
O(N log N) route, Sec. "Discretization") and plain O(N^2) direct sums.
"""

import numpy as np
import scipy.fft as sfft

from . import tensor as _t


class Geometry:
    """Grid sizes, cell size and padded FFT lengths (L = smallest 2^a 3^b >= 2 n)."""

    def __init__(self, n_out, nzd, cellsize):
        self.n_out = tuple(int(v) for v in n_out)
        self.nzd = int(nzd)
        assert 1 <= self.nzd <= self.n_out[2]
        self.cellsize = tuple(float(v) for v in cellsize)
        self.L = tuple(_t.fft_length(n) for n in self.n_out)

    @property
    def design_shape(self):
        nx, ny, _ = self.n_out
        return (self.nzd, ny, nx)

    @property
    def out_shape(self):
        nx, ny, nz = self.n_out
        return (nz, ny, nx)


class FFTOperator:
    """D by zero-padded float64 FFT: rfftn of the six padded tensor components."""

    def __init__(self, geom, octant=None, workers=None):
        self.g = geom
        self.workers = workers
        Lx, Ly, Lz = geom.L
        self.octant = octant if octant is not None else _t.tensor_octant(geom.n_out, geom.cellsize)
        pad = _t.padded_tensor(geom.n_out, geom.L, geom.cellsize, self.octant)
        # Nhat[a][b] (symmetric), complex half spectra of shape (Lz, Ly, Lx//2+1)
        self.Nhat = {}
        for c, name in enumerate(_t.COMPONENTS):
            self.Nhat[_t.INDEX[name]] = sfft.rfftn(pad[c], s=(Lz, Ly, Lx), workers=workers)
        del pad

    def _N(self, a, b):
        return self.Nhat[(min(a, b), max(a, b))]

    def _convolve(self, src, out_nz):
        """-(N * src) for src (3, sz, ny, nx) placed at z in [0, sz); crop to out_nz planes."""
        Lx, Ly, Lz = self.g.L
        nx, ny = self.g.n_out[0], self.g.n_out[1]
        S = [sfft.rfftn(src[b], s=(Lz, Ly, Lx), workers=self.workers) for b in range(3)]
        out = np.empty((3, out_nz, ny, nx))
        for a in range(3):
            acc = self._N(a, 0) * S[0] + self._N(a, 1) * S[1] + self._N(a, 2) * S[2]
            full = sfft.irfftn(-acc, s=(Lz, Ly, Lx), workers=self.workers)
            out[a] = full[:out_nz, :ny, :nx]
        return out

    def forward(self, M):
        """H on the output grid for M (3, nzd, ny, nx) on the design box."""
        M = np.asarray(M, dtype=np.float64)
        assert M.shape == (3,) + self.g.design_shape
        return self._convolve(M, self.g.n_out[2])

    def adjoint(self, gH):
        """D^T gH on the design box for gH (3, nz, ny, nx) on the output grid."""
        gH = np.asarray(gH, dtype=np.float64)
        assert gH.shape == (3,) + self.g.out_shape
        return self._convolve(gH, self.g.nzd)


def _full_matrix_blocks(geom, octant):
    """Dense blocks N(i - j) for every output i and design j: (3, 3, n_out_cells, n_design_cells)."""
    nx, ny, nz = geom.n_out
    zi, yi, xi = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    zj, yj, xj = np.meshgrid(np.arange(geom.nzd), np.arange(ny), np.arange(nx), indexing="ij")
    di = xi.ravel()[:, None] - xj.ravel()[None, :]
    dj = yi.ravel()[:, None] - yj.ravel()[None, :]
    dk = zi.ravel()[:, None] - zj.ravel()[None, :]
    vals = _t.tensor_lookup(octant, di, dj, dk)
    blocks = np.empty((3, 3) + di.shape)
    for c, name in enumerate(_t.COMPONENTS):
        a, b = _t.INDEX[name]
        blocks[a, b] = vals[c]
        blocks[b, a] = vals[c]
    return blocks


class DirectOperator:
    """D by explicit O(N_out * N_design) double sums (tiny grids only)."""

    def __init__(self, geom, octant=None):
        self.g = geom
        self.octant = octant if octant is not None else _t.tensor_octant(geom.n_out, geom.cellsize)
        nout = np.prod(geom.out_shape)
        ndes = np.prod(geom.design_shape)
        assert nout * ndes <= 40_000_000, "direct sums are for tiny grids"
        self.blocks = _full_matrix_blocks(geom, self.octant)

    def forward(self, M):
        M = np.asarray(M, dtype=np.float64).reshape(3, -1)
        H = -np.einsum("abij,bj->ai", self.blocks, M)
        return H.reshape((3,) + self.g.out_shape)

    def adjoint(self, gH):
        gH = np.asarray(gH, dtype=np.float64).reshape(3, -1)
        # (D^T g)_j = -sum_i N(j - i) g_i = -sum_i N(i - j) g_i   (N even, symmetric)
        out = -np.einsum("abij,ai->bj", self.blocks, gH)
        return out.reshape((3,) + self.g.design_shape)


def field_at(geom, octant, M, cells):
    """H at selected output cells (k, j, i) by direct sums over the whole design box.

    cells: integer array (m, 3) of (z, y, x). Returns (m, 3). Memory O(N_design).
    """
    M = np.asarray(M, dtype=np.float64)
    nx, ny, _ = geom.n_out
    zj, yj, xj = np.meshgrid(np.arange(geom.nzd), np.arange(ny), np.arange(nx), indexing="ij")
    Mf = M.reshape(3, -1)
    out = np.empty((len(cells), 3))
    for n, (z, y, x) in enumerate(np.asarray(cells)):
        vals = _t.tensor_lookup(octant, x - xj.ravel(), y - yj.ravel(), z - zj.ravel())
        H = np.zeros(3)
        for c, name in enumerate(_t.COMPONENTS):
            a, b = _t.INDEX[name]
            H[a] -= vals[c] @ Mf[b]
            if a != b:
                H[b] -= vals[c] @ Mf[a]
        out[n] = H
    return out


def adjoint_at(geom, octant, gH, cells, support=None):
    """(D^T gH) at selected design cells (z, y, x) by direct sums over the support of gH.

    support: optional integer array (s, 3) of (z, y, x) output cells where gH may be
    non-zero (default: all). Returns (m, 3).
    """
    gH = np.asarray(gH, dtype=np.float64)
    if support is None:
        nx, ny, nz = geom.n_out
        zi, yi, xi = (v.ravel() for v in np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij"))
    else:
        support = np.asarray(support)
        zi, yi, xi = support[:, 0], support[:, 1], support[:, 2]
    gs = gH[:, zi, yi, xi]
    out = np.empty((len(cells), 3))
    for n, (z, y, x) in enumerate(np.asarray(cells)):
        vals = _t.tensor_lookup(octant, x - xi, y - yi, z - zi)
        r = np.zeros(3)
        for c, name in enumerate(_t.COMPONENTS):
            a, b = _t.INDEX[name]
            r[a] -= vals[c] @ gs[b]
            if a != b:
                r[b] -= vals[c] @ gs[a]
        out[n] = r
    return out
