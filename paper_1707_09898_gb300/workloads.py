"""Seeded synthetic workloads for the magnet topology optimizer.

This module only generates inputs (sizes, densities, magnetizations, target
masks and target fields) from fixed seeds. It contains none of the method's
arithmetic, so both the CUDA path and the float64 oracle can be fed from it.

Every workload is synthetic. The paper's own benchmark geometry (a unit cube
magnetized along z with a small target box above it, Sec. "Validation and
Benchmarks") is only shown in a figure; the shapes below follow it: a design
box at the bottom of the grid, magnetization along +z, and a target region a
few cells above the top face or on the top layer.
"""

from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

MU0 = 4e-7 * np.pi
MS = 1.0 / MU0  # 1 T / mu0 in A/m


@dataclass(frozen=True)
class Workload:
    name: str
    n_out: Tuple[int, int, int]          # (nx, ny, nz) output grid
    nzd: int                             # design box is z in [0, nzd)
    cellsize: Tuple[float, float, float] = (1e-3, 1e-3, 1e-3)
    p: float = 3.0
    rho_kind: str = "uniform"            # "uniform" (U[0,1]) or "const"
    rho_const: float = 0.5
    rho_seed: int = 0
    m0_kind: str = "const"               # "const" or "vmf"
    m0_dir: Tuple[float, float, float] = (0.0, 0.0, 1.0)
    m0_seed: int = 0
    vmf_kappa: float = 10.0
    mask_z: int = 0                      # target plane z index (the first of mask_nz planes)
    mask_nz: int = 1                     # number of target planes
    ms: float = MS                       # magnetization magnitude of M0 (A/m)
    mask_xy: Tuple[int, int, int, int] = (0, 0, 0, 0)  # x0, x1, y0, y1 (half-open)
    ht_kind: str = "const"               # "const" or "normal"
    ht_const: Tuple[float, float, float] = (0.0, 0.0, 0.0)  # in units of ms
    ht_sigma: float = 0.05               # in units of ms (normal)
    ht_seed: int = 0
    w: Tuple[float, float, float] = (0.0, 0.0, 1.0)
    iters: int = 0
    alpha: float = 0.1

    @property
    def design_shape(self):
        return (self.nzd, self.n_out[1], self.n_out[0])

    @property
    def out_shape(self):
        return (self.n_out[2], self.n_out[1], self.n_out[0])

    @property
    def design_cells(self):
        return self.nzd * self.n_out[1] * self.n_out[0]

    # -- generators -------------------------------------------------------
    def rho(self):
        if self.rho_kind == "const":
            return np.full(self.design_shape, self.rho_const, dtype=np.float32)
        rng = np.random.default_rng(self.rho_seed)
        return rng.random(self.design_shape, dtype=np.float64).astype(np.float32)

    def M0_const(self):
        """(3,) float64 constant magnetization in A/m, or None when spatially varying."""
        if self.m0_kind != "const":
            return None
        d = np.asarray(self.m0_dir, dtype=np.float64)
        return self.ms * d

    def M0_field(self):
        """(3, nzd, ny, nx) float32 magnetization in A/m (constant or von Mises-Fisher)."""
        if self.m0_kind == "const":
            c = self.M0_const().astype(np.float32)
            return np.broadcast_to(c[:, None, None, None], (3,) + self.design_shape).copy()
        rng = np.random.default_rng(self.m0_seed)
        shape = self.design_shape
        u = rng.random(shape)
        phi = 2.0 * np.pi * rng.random(shape)
        k = self.vmf_kappa
        wz = 1.0 + np.log(u + (1.0 - u) * np.exp(-2.0 * k)) / k  # vMF inverse CDF about +z
        s = np.sqrt(np.maximum(0.0, 1.0 - wz * wz))
        return (self.ms * np.stack([s * np.cos(phi), s * np.sin(phi), wz])).astype(np.float32)

    def mask(self):
        m = np.zeros(self.out_shape, dtype=np.uint8)
        x0, x1, y0, y1 = self.mask_xy
        m[self.mask_z:self.mask_z + self.mask_nz, y0:y1, x0:x1] = 1
        return m

    def Ht_const_vec(self):
        """(3,) float32 constant target field in A/m, or None when a full field is used."""
        if self.ht_kind != "const":
            return None
        return (self.ms * np.asarray(self.ht_const, dtype=np.float64)).astype(np.float32)

    def Ht_field(self):
        """(3, nz, ny, nx) float32 target field (zero off the mask for the random kind)."""
        if self.ht_kind == "const":
            c = self.Ht_const_vec()
            return np.broadcast_to(c[:, None, None, None], (3,) + self.out_shape).copy()
        rng = np.random.default_rng(self.ht_seed)
        out = np.zeros((3,) + self.out_shape, dtype=np.float32)
        m = self.mask().astype(bool)
        vals = rng.normal(0.0, self.ht_sigma * self.ms, size=(3, int(m.sum())))
        out[:, m] = vals.astype(np.float32)
        return out


def _centered(n, width):
    a = (n - width) // 2
    return a, a + width


def config1():
    """16^3 design of 1 mm cubes, one layer of target cells above (n_out z = 17)."""
    return Workload(
        name="c1_16cube", n_out=(16, 16, 17), nzd=16, rho_seed=1,
        mask_z=16, mask_xy=(6, 10, 6, 10), ht_const=(0.0, 0.0, 0.1))


def config2():
    """64^3 design, target plane 16x16 two cells above the top face, rho = 0.5, 200 steps."""
    x0, x1 = _centered(64, 16)
    return Workload(
        name="c2_64cube_opt", n_out=(64, 64, 72), nzd=64, rho_kind="const", rho_const=0.5,
        mask_z=65, mask_xy=(x0, x1, x0, x1), ht_const=(0.0, 0.0, 0.2), iters=200, alpha=0.1)


def config3():
    """128x128x64 design, vMF(kappa=10) magnetization, random 3-component target on a 32x32 plane."""
    x0, x1 = _centered(128, 32)
    return Workload(
        name="c3_128x128x64_vmf", n_out=(128, 128, 66), nzd=64, rho_seed=3,
        m0_kind="vmf", m0_seed=4, mask_z=65, mask_xy=(x0, x1, x0, x1),
        ht_kind="normal", ht_seed=5, w=(1.0, 1.0, 1.0))


def config4(n, m0="const"):
    """Throughput workload: n^3 design = output grid, n/4 x n/4 target patch on the top layer.
    m0 = "vmf": a spatially varying magnetization (von Mises-Fisher about +z, kappa = 10, seed 8)."""
    x0, x1 = _centered(n, n // 4)
    return Workload(
        name=f"c4_{n}cube" + ("" if m0 == "const" else "_" + m0), n_out=(n, n, n), nzd=n, rho_seed=7,
        m0_kind=m0, m0_seed=8, mask_z=n - 1, mask_xy=(x0, x1, x0, x1), ht_const=(0.0, 0.0, 0.2))


def small(n_out, nzd, cellsize=(1e-3, 1e-3, 1e-3), seed=11, m0_kind="const", w=(0.0, 0.0, 1.0),
          mask_z=None, mask_xy=None, ht_kind="const"):
    """Small ragged test grids: arbitrary n_out / nzd, mask on the top output layer."""
    nx, ny, nz = n_out
    if mask_z is None:
        mask_z = nz - 1
    if mask_xy is None:
        mask_xy = (nx // 4, nx - nx // 4, ny // 4, ny - ny // 4)
    return Workload(
        name=f"small_{nx}x{ny}x{nz}_{nzd}", n_out=tuple(n_out), nzd=nzd, cellsize=tuple(cellsize),
        rho_seed=seed, m0_kind=m0_kind, m0_seed=seed + 1, mask_z=mask_z, mask_xy=mask_xy,
        ht_kind=ht_kind, ht_seed=seed + 2, ht_const=(0.0, 0.0, 0.1), w=tuple(w))


def paper_problem(box=5):
    """The paper's validation problem (Sec. "Validation and Benchmarks"): a unit cube of
    39^3 cells magnetized along +z (M0 = (0, 0, 1)) with two layers of cells above it
    (39 x 39 x 41 = 62,361 cells, the size of its finite-difference mesh), rho = 1 at the
    start; maximise the z field on a centred box x box area of those two layers:
    J = -1/2 sum_box H_z^2 (w_z = -1/2, H_t = 0)."""
    x0, x1 = _centered(39, box)
    return Workload(
        name=f"paper_39cube_box{box}", n_out=(39, 39, 41), nzd=39, cellsize=(1.0 / 39,) * 3,
        rho_kind="const", rho_const=1.0, ms=1.0, mask_z=39, mask_nz=2, mask_xy=(x0, x1, x0, x1),
        ht_const=(0.0, 0.0, 0.0), w=(0.0, 0.0, -0.5))


def paper_field_gradient(beta=1e5):
    """The paper's field-and-gradient problem (Sec. "Optimization of field and gradient"):
    a 40 x 40 x 20 design of cubic cells of edge 30 (in the length unit of beta) magnetized
    along +z (M0 = (0, 0, 1), rho = 1 at the start), the target plane two cells above its
    top face (z = 21 of a 40 x 40 x 22 grid),
    a centred 20 x 20 field region on it and a one-cell strip along three of its sides
    (x = 9 and x = 30 with outward normals -x and +x, y = 30 with normal +y).
    Returns (workload, field mask [ny][nx] bool, strip [(y, x, axis, sign)], beta); axis
    0 = y, 1 = x."""
    wl = Workload(
        name="paper_field_gradient", n_out=(40, 40, 22), nzd=20, cellsize=(30.0, 30.0, 30.0), rho_kind="const",
        rho_const=1.0, ms=1.0, mask_z=21, mask_xy=(10, 30, 10, 30), ht_const=(0.0, 0.0, 0.0), w=(0.0, 0.0, -0.5))
    field = wl.mask()[21].astype(bool)
    strip = ([(y, 9, 1, -1) for y in range(10, 30)] + [(y, 30, 1, 1) for y in range(10, 30)] +
             [(30, x, 0, 1) for x in range(10, 30)])
    return wl, field, strip, beta


# Warm-start specifications: the target of each optimisation drawn from a seed.
CONFIG5_TRAIN_SEEDS = range(10000, 12000)
CONFIG5_HELDOUT_SEEDS = range(20000, 20200)


def config5(seed):
    """64^3 design on a 64 x 64 x 72 grid, rho = 0.5, 200 steps of 0.1; the target is a
    centred square of width U{8..32} on the plane z = 63 + h, h ~ U{1..8} cells above the
    top face, with H_t,z ~ U[0.05, 0.3] Ms on it."""
    rng = np.random.default_rng(seed)
    h = int(rng.integers(1, 9))
    width = int(rng.integers(8, 33))
    ht = float(rng.uniform(0.05, 0.3))
    x0, x1 = _centered(64, width)
    return Workload(
        name=f"c5_spec{seed}", n_out=(64, 64, 72), nzd=64, rho_kind="const", rho_const=0.5,
        mask_z=63 + h, mask_xy=(x0, x1, x0, x1), ht_const=(0.0, 0.0, ht), iters=200, alpha=0.1)


def config5_spec(wl):
    """(footprint [ny][nx] uint8, H_t,z / Ms, height above the top face in cells) of a config5 workload."""
    return wl.mask()[wl.mask_z], float(wl.ht_const[2]), wl.mask_z - (wl.nzd - 1)
