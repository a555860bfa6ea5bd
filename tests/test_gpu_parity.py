"""Parity of the CUDA path (through the C ABI) with the float64 oracle.

Tolerances: relative L2 error <= 1e-5 for H, <= 1e-4 for dJ/drho and <= 1e-5
for J (float32 FFTs and products, float64 tensor setup and reductions). Inputs
are the same float32 arrays for both sides, promoted to float64 by the oracle.
Geometries span several 16-column tiles, ragged row counts, every radix (2, 3,
4, 8, 16, 32), anisotropic cells and design slabs thinner than the grid.
"""

import numpy as np
import pytest
import torch

from oracle import convolution as C
from oracle import objective as O
from oracle import optimizer as P
from oracle import tensor as T
from paper_1707_09898_gb300 import workloads as W

from errlog import record

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


def magnet(wl, **kw):
    from paper_1707_09898_gb300 import Magnet

    M0 = torch.from_numpy(wl.M0_field()).to(DEV) if wl.m0_kind != "const" else wl.M0_const()
    return Magnet(wl.n_out, wl.nzd, wl.cellsize, M0=M0, p=wl.p, device=0, **kw)


def oracle_op(wl):
    return C.FFTOperator(C.Geometry(wl.n_out, wl.nzd, wl.cellsize))


GEOMS = [
    # n_out, nzd, cellsize
    ((16, 16, 17), 16, (1e-3, 1e-3, 1e-3)),      # config 1 grid: L = 32, 32, 36
    ((40, 23, 30), 19, (1e-3, 0.8e-3, 1.3e-3)),  # L = 96 (radix 32x3), 48, 64; ragged rows
    ((33, 50, 12), 7, (2e-3, 1e-3, 1e-3)),       # L = 72 (8x3x3), 128, 24
    ((9, 6, 20), 5, (1e-3, 1e-3, 0.5e-3)),       # L = 18 (2x3x3), 12, 48
    ((70, 36, 44), 40, (1e-3, 1e-3, 1e-3)),      # L = 144 (16x3x3), 72, 96
    ((140, 12, 10), 6, (1e-3, 1e-3, 1e-3)),      # L = 288 (32x3x3), 24, 24
]


@pytest.mark.parametrize("n_out,nzd,d", GEOMS)
@pytest.mark.parametrize("m0", ["const", "vmf"])
def test_stray_field_and_adjoint(n_out, nzd, d, m0):
    wl = W.small(n_out, nzd, cellsize=d, m0_kind=m0, w=(1.0, 0.5, 2.0), ht_kind="normal")
    m = magnet(wl)
    rho = wl.rho()
    H = m.stray_field(torch.from_numpy(rho).to(DEV)).cpu().numpy()
    op = oracle_op(wl)
    M0 = wl.M0_field().astype(np.float64)
    Hr = op.forward(O.magnetization(rho, M0, wl.p))
    assert rel_l2(H, Hr) <= 1e-5
    gH = np.random.default_rng(3).normal(size=(3,) + wl.out_shape).astype(np.float32)
    G = m.stray_field_adjoint(torch.from_numpy(rho).to(DEV), torch.from_numpy(gH).to(DEV)).cpu().numpy()
    Gr = O.chain_rule(rho, M0, wl.p, op.adjoint(gH))
    assert rel_l2(G, Gr) <= 1e-4


@pytest.mark.parametrize("n_out,nzd,d", GEOMS[:4])
@pytest.mark.parametrize("ht", ["const", "normal"])
def test_objective_and_gradient(n_out, nzd, d, ht):
    wl = W.small(n_out, nzd, cellsize=d, m0_kind="vmf", w=(0.7, 1.0, 1.5), ht_kind=ht)
    m = magnet(wl)
    rho, mask, Htf = wl.rho(), wl.mask(), wl.Ht_field()
    Hout = torch.empty((3,) + wl.out_shape, device=DEV)
    J, G = m.objective_and_gradient(torch.from_numpy(rho).to(DEV), torch.from_numpy(mask).to(DEV),
                                    Ht=torch.from_numpy(Htf).to(DEV), w=wl.w, H_out=Hout)
    op = oracle_op(wl)
    Jr, Gr, Hr = O.objective_and_gradient(op, rho, wl.M0_field(), wl.p, mask, Htf, wl.w)
    assert abs(J - Jr) <= 1e-5 * abs(Jr)
    assert rel_l2(G.cpu().numpy(), Gr) <= 1e-4
    assert rel_l2(Hout.cpu().numpy(), Hr) <= 1e-5


def test_config1_against_oracle_and_direct_sum():
    wl = W.config1()
    m = magnet(wl)
    rho, mask = wl.rho(), wl.mask()
    J, G = m.objective_and_gradient(torch.from_numpy(rho).to(DEV), torch.from_numpy(mask).to(DEV),
                                    Ht_const=wl.Ht_const_vec(), w=wl.w)
    H = m.stray_field(torch.from_numpy(rho).to(DEV)).cpu().numpy()
    g = C.Geometry(wl.n_out, wl.nzd, wl.cellsize)
    fft, direct = C.FFTOperator(g), None
    direct = C.DirectOperator(g, fft.octant)
    Jr, Gr, Hr = O.objective_and_gradient(fft, rho, wl.M0_const(), wl.p, mask, wl.Ht_const_vec(), wl.w)
    Jd, Gd, Hd = O.objective_and_gradient(direct, rho, wl.M0_const(), wl.p, mask, wl.Ht_const_vec(), wl.w)
    assert rel_l2(Hr, Hd) <= 1e-12 and rel_l2(Gr, Gd) <= 1e-12
    record("c1 16x16x17", H=rel_l2(H, Hr), J=abs(J - Jr) / abs(Jr), G=rel_l2(G.cpu().numpy(), Gr))
    assert rel_l2(H, Hr) <= 1e-5
    assert rel_l2(G.cpu().numpy(), Gr) <= 1e-4
    assert abs(J - Jr) <= 1e-5 * abs(Jr)


def test_tensor_octant_matches_oracle():
    wl = W.small((20, 18, 24), 10, cellsize=(1e-3, 0.7e-3, 1.2e-3))
    m = magnet(wl, tensor=False)
    oct_gpu = m.tensor_octant()
    oct_ref = T.tensor_octant(wl.n_out, wl.cellsize)
    assert np.abs(oct_gpu - oct_ref).max() <= 1e-11 * np.abs(oct_ref).max()


def test_tensor_spectrum_matches_oracle():
    wl = W.small((12, 10, 14), 8, cellsize=(1e-3, 1.1e-3, 0.9e-3))
    m = magnet(wl)
    Lx, Ly, Lz = m.fft_lengths()
    spec = m.tensor_spectrum()
    pad = T.padded_tensor(wl.n_out, (Lx, Ly, Lz), wl.cellsize)
    for c in range(6):
        F = np.fft.rfftn(pad[c])
        assert np.abs(F.imag).max() <= 1e-12 * np.abs(F.real).max()
        ref = -F.real[: Lz // 2 + 1, : Ly // 2 + 1, :] / (Lx * Ly * Lz)
        assert np.abs(spec[c] - ref).max() <= 2e-7 * np.abs(ref).max()


def test_optimize_step_matches_oracle():
    wl = W.small((20, 12, 10), 8)
    m = magnet(wl)
    rng = np.random.default_rng(9)
    rho = rng.random(wl.design_shape).astype(np.float32)
    G = rng.normal(size=wl.design_shape).astype(np.float32)
    for normalize, alpha in [(True, 0.1), (False, 0.05)]:
        r = torch.from_numpy(rho).to(DEV)
        m.optimize_step(r, torch.from_numpy(G).to(DEV), alpha, normalize)
        ref = P.projected_gradient_step(rho, G, alpha, normalize)
        np.testing.assert_allclose(r.cpu().numpy(), ref, rtol=0, atol=2e-7)
    r = torch.from_numpy(rho).to(DEV)
    m.optimize_step(r, torch.zeros_like(r), 0.1, True)
    np.testing.assert_array_equal(r.cpu().numpy(), rho)


def test_autograd_functions():
    from paper_1707_09898_gb300 import StrayField, TopoObjective

    wl = W.small((24, 20, 18), 12, m0_kind="vmf", w=(1.0, 1.0, 1.0), ht_kind="normal")
    m = magnet(wl)
    rho = torch.from_numpy(wl.rho()).to(DEV).requires_grad_(True)
    c = torch.from_numpy(np.random.default_rng(4).normal(size=(3,) + wl.out_shape).astype(np.float32)).to(DEV)
    (StrayField.apply(rho, m) * c).sum().backward()
    op = oracle_op(wl)
    ref = O.chain_rule(wl.rho(), wl.M0_field(), wl.p, op.adjoint(c.cpu().numpy()))
    assert rel_l2(rho.grad.cpu().numpy(), ref) <= 1e-4
    rho.grad = None
    mask = torch.from_numpy(wl.mask()).to(DEV)
    Ht = torch.from_numpy(wl.Ht_field()).to(DEV)
    J = TopoObjective.apply(rho, m, mask, Ht, (0, 0, 0), wl.w)
    (2.0 * J).backward()
    _, Gr, _ = O.objective_and_gradient(op, wl.rho(), wl.M0_field(), wl.p, wl.mask(), wl.Ht_field(), wl.w)
    assert rel_l2(rho.grad.cpu().numpy(), 2.0 * Gr) <= 1e-4


def test_gradient_matches_central_differences_on_gpu():
    """Config-3 style (vMF M0, random 3-component target): GPU gradient vs central differences of J (float64)."""
    wl = W.small((32, 32, 18), 16, m0_kind="vmf", w=(1.0, 1.0, 1.0), ht_kind="normal")
    m = magnet(wl)
    rho = torch.from_numpy(wl.rho()).to(DEV)
    mask = torch.from_numpy(wl.mask()).to(DEV)
    Ht = torch.from_numpy(wl.Ht_field()).to(DEV)
    _, G = m.objective_and_gradient(rho, mask, Ht=Ht, w=wl.w)
    G = G.cpu().numpy()
    op = oracle_op(wl)
    rng = np.random.default_rng(6)
    big = np.flatnonzero(np.abs(G) > 1e-3 * np.abs(G).max())
    cells = rng.choice(big, size=16, replace=False)
    h = 1e-3
    r64 = wl.rho().astype(np.float64)
    M0 = wl.M0_field().astype(np.float64)
    for f in cells:
        idx = np.unravel_index(f, wl.design_shape)
        rp, rm = r64.copy(), r64.copy()
        rp[idx] += h
        rm[idx] -= h
        Jp = O.objective(op.forward(O.magnetization(rp, M0, wl.p)), wl.mask(), wl.Ht_field(), wl.w)
        Jm = O.objective(op.forward(O.magnetization(rm, M0, wl.p)), wl.mask(), wl.Ht_field(), wl.w)
        fd = (Jp - Jm) / (2 * h)
        assert abs(G[idx] - fd) <= 1e-3 * abs(fd) + 1e-5 * np.abs(G).max()


def test_errors_are_reported():
    from paper_1707_09898_gb300 import Magnet
    from paper_1707_09898_gb300._lib import TopomagError

    with pytest.raises(TopomagError, match="TM_ERR_SIZE"):
        Magnet((3, 8, 8), 4)
    with pytest.raises(TopomagError, match="TM_ERR_SIZE"):
        Magnet((300, 8, 8), 4)
    with pytest.raises(TopomagError, match="TM_ERR_ARG"):
        Magnet((8, 8, 8), 9)
    m = Magnet((8, 8, 8), 8, tensor=False)
    with pytest.raises(TopomagError, match="TM_ERR_STATE"):
        m.stray_field(torch.zeros(m.design_shape, device=DEV))
    with pytest.raises(TopomagError, match="TM_ERR_ARG"):
        m._ck(m.L.tm_set_penalty(m.h, 0.5))


@pytest.mark.parametrize("n_out,nzd,d,planes,m0", [
    ((16, 16, 17), 16, (1e-3, 1e-3, 1e-3), (16,), "const"),          # config 1 layout, one plane above
    ((40, 23, 30), 19, (1e-3, 0.8e-3, 1.3e-3), (22, 24, 25), "vmf"),  # three planes, gap, varying M0
    ((33, 50, 12), 7, (2e-3, 1e-3, 1e-3), (3, 9), "const"),          # a plane inside the design box
    ((24, 20, 26), 14, (1e-3, 1e-3, 1e-3), tuple(range(14, 24)), "const"),  # 10 planes: full pipeline
])
@pytest.mark.parametrize("w", [(0.0, 0.0, 1.0), (1.0, 0.5, 2.0)])
def test_prepared_target_matches_oracle(n_out, nzd, d, planes, m0, w):
    """tm_set_target + tm_evaluate (direct z sums for <= 8 target planes) against the oracle."""
    wl = W.small(n_out, nzd, cellsize=d, m0_kind=m0, w=w, ht_kind="normal")
    m = magnet(wl)
    mask = np.zeros(wl.out_shape, dtype=np.uint8)
    rng = np.random.default_rng(21)
    for z in planes:
        mask[z] = rng.random(wl.out_shape[1:]) < 0.3
    Htf = wl.Ht_field()
    m.set_target(torch.from_numpy(mask).to(DEV), Ht=torch.from_numpy(Htf).to(DEV), w=w)
    rho = torch.from_numpy(wl.rho()).to(DEV)
    for _ in range(2):  # repeated evaluations reuse the prepared target
        J, G = m.evaluate(rho)
    op = oracle_op(wl)
    Jr, Gr, _ = O.objective_and_gradient(op, wl.rho(), wl.M0_field(), wl.p, mask, Htf, w)
    assert abs(J - Jr) <= 1e-5 * abs(Jr)
    assert rel_l2(G.cpu().numpy(), Gr) <= 1e-4
    # the one-shot call agrees with the prepared one
    J2, G2 = m.objective_and_gradient(rho, torch.from_numpy(mask).to(DEV), Ht=torch.from_numpy(Htf).to(DEV), w=w)
    assert abs(J2 - Jr) <= 1e-5 * abs(Jr)
    assert rel_l2(G2.cpu().numpy(), Gr) <= 1e-4


def test_prepared_target_empty_mask_gives_zero():
    wl = W.small((16, 12, 10), 8)
    m = magnet(wl)
    m.set_target(torch.zeros(wl.out_shape, dtype=torch.uint8, device=DEV), Ht_const=(0, 0, 1e5))
    J, G = m.evaluate(torch.from_numpy(wl.rho()).to(DEV))
    assert J == 0.0 and float(G.abs().max()) == 0.0


def test_cufft_comparison_pipeline_matches_oracle():
    """The plain cuFFT comparison pipeline computes the same J and gradient (so its timing is comparable)."""
    from paper_1707_09898_gb300.cufft_pipeline import CufftMagnet

    wl = W.small((20, 18, 22), 16)
    b = CufftMagnet(wl.n_out, wl.nzd, wl.cellsize, M0=wl.M0_const(), p=wl.p)
    rho, mask = wl.rho(), wl.mask()
    J, G = b.objective_and_gradient(torch.from_numpy(rho).to(DEV), torch.from_numpy(mask).to(DEV),
                                    Ht_const=tuple(wl.Ht_const_vec()), w=wl.w)
    op = oracle_op(wl)
    Jr, Gr, _ = O.objective_and_gradient(op, rho, wl.M0_const(), wl.p, mask, wl.Ht_const_vec(), wl.w)
    assert abs(J - Jr) <= 1e-5 * abs(Jr)
    assert rel_l2(G.cpu().numpy(), Gr) <= 1e-4


def test_optimize_step_reuses_the_evaluated_max_only_for_that_array():
    from paper_1707_09898_gb300 import Magnet

    wl = W.config1()
    m = Magnet(wl.n_out, wl.nzd, wl.cellsize, M0=wl.M0_const(), p=wl.p, device=0)
    m.set_target(torch.from_numpy(wl.mask()).to(DEV), Ht_const=tuple(float(v) for v in wl.Ht_const_vec()), w=wl.w)
    rho = torch.from_numpy(wl.rho()).to(DEV)
    G = torch.empty_like(rho)
    m.evaluate(rho, G=G)
    r1 = m.optimize_step(rho.clone(), G, 0.1, True, reuse_max=True)
    r2 = m.optimize_step(rho.clone(), G, 0.1, True)
    assert torch.equal(r1, r2)
    G2 = G * 0.5  # another array: its own max is computed, so the step is the same
    r3 = m.optimize_step(rho.clone(), G2, 0.1, True, reuse_max=True)
    assert torch.allclose(r3, r2, atol=1e-6)
    assert not torch.equal(r2, rho)


@pytest.mark.parametrize("case", ["c1", "ragged", "vmf", "three_components", "two_planes"])
def test_fused_and_separate_yz_passes_agree(case):
    """The prepared path with the y transform fused into the direct z sum (default) and with
    separate passes: the same convolution, float32 rounding apart; both against the oracle.
    c1 / ragged: both directions fused; vmf, three_components: forward separate (three field
    components), adjoint fused with three spectra; two_planes: forward separate, adjoint
    fused from two source planes."""
    from paper_1707_09898_gb300 import Magnet

    if case == "c1":
        wl = W.config1()
    elif case == "vmf":
        wl = W.small((14, 11, 13), 9, seed=61, m0_kind="vmf", w=(1.0, 1.0, 1.0), ht_kind="normal")
    elif case == "three_components":
        wl = W.small((18, 10, 12), 8, seed=62, w=(0.5, 1.0, 2.0), ht_kind="normal")
    else:
        wl = W.small((20, 12, 15), 9, seed=63)
    mask = wl.mask()
    if case == "two_planes":
        mask[-2] = mask[-1]
    M0 = wl.M0_field() if wl.m0_kind != "const" else wl.M0_const()
    m = Magnet(wl.n_out, wl.nzd, wl.cellsize, M0=torch.from_numpy(M0).to(DEV) if wl.m0_kind != "const" else M0,
               p=wl.p, device=0)
    Ht = wl.Ht_field()
    m.set_target(torch.from_numpy(mask).to(DEV), Ht=torch.from_numpy(Ht).to(DEV), w=wl.w)
    rho = torch.from_numpy(wl.rho()).to(DEV)
    out = {}
    for fused in (True, False):
        m.set_fused(fused)
        J, G = m.evaluate(rho)
        out[fused] = (J, G.cpu().numpy())
    (Jf, Gf), (Js, Gs) = out[True], out[False]
    assert abs(Jf - Js) <= 1e-6 * abs(Js)
    assert np.linalg.norm(Gf - Gs) <= 1e-5 * np.linalg.norm(Gs)
    op = C.FFTOperator(C.Geometry(wl.n_out, wl.nzd, wl.cellsize))
    Jr, Gr, _ = O.objective_and_gradient(op, wl.rho(), M0, wl.p, mask, Ht, wl.w)
    for J, G in out.values():
        assert abs(J - Jr) <= 1e-5 * abs(Jr)
        assert np.linalg.norm(G - Gr) <= 1e-4 * np.linalg.norm(Gr)


@pytest.mark.parametrize("shape", [(230, 14, 10, 9), (20, 230, 7, 6), (18, 220, 92, 90)])
def test_length_512_fast_paths(shape):
    """Grids whose padded x or y length is 512 take the x passes with one frequency per
    thread and the warp-specialized y/z kernels (flattened over (column block, plane)
    items, the target plane's inverse y transform in the forward kernel's tail): ragged
    row counts, x and y extents below L/2, and (last case) blocks whose items span two
    column blocks. Fused and separate passes, the one-shot call and the field against the
    oracle; a second density checks that the item counters re-arm between launches."""
    nx, ny, nz, nzd = shape
    wl = W.small((nx, ny, nz), nzd, seed=71)
    mask = wl.mask()
    m = magnet(wl)
    Htc = tuple(float(v) for v in wl.Ht_const_vec())
    tmask = torch.from_numpy(mask).to(DEV)
    m.set_target(tmask, Ht_const=Htc, w=wl.w)
    op = C.FFTOperator(C.Geometry(wl.n_out, wl.nzd, wl.cellsize))
    rng = np.random.default_rng(72)
    for rho in (wl.rho(), rng.random(wl.design_shape).astype(np.float32)):
        rho_t = torch.from_numpy(rho).to(DEV)
        out = []
        for fused in (True, False):
            m.set_fused(fused)
            out.append(m.evaluate(rho_t))
        out.append(m.objective_and_gradient(rho_t, tmask, Ht_const=Htc, w=wl.w))
        Jr, Gr, _ = O.objective_and_gradient(op, rho, wl.M0_const(), wl.p, mask, wl.Ht_const_vec(), wl.w)
        for J, G in out:
            assert abs(J - Jr) <= 1e-5 * abs(Jr)
            assert rel_l2(G.cpu().numpy(), Gr) <= 1e-4
        (Jf, Gf), (Js, Gs) = out[0], out[1]
        assert abs(Jf - Js) <= 1e-6 * abs(Js)
        assert rel_l2(Gf.cpu().numpy(), Gs.cpu().numpy().astype(np.float64)) <= 1e-5
    m.set_fused(True)
    H = m.stray_field(rho_t).cpu().numpy()
    Hr = op.forward(O.magnetization(rho, wl.M0_const(), wl.p))
    assert rel_l2(H, Hr) <= 1e-5


@pytest.mark.parametrize("planes", [tuple(range(140, 150)), (143, 147)])
@pytest.mark.parametrize("w", [(0.0, 0.0, 1.0), (1.0, 0.0, 2.0)])
def test_length_512_z_pass(planes, w):
    """nz = 150 pads z to 512, the one-input z pass that transforms each column tile once
    for all outputs: the full field (every plane), the prepared target on 10 planes (the
    whole-grid route: output and input planes restricted to the device range) and on 2
    (few planes: the direct transforms of those planes), with one or two weighted field
    components (one or two outputs per column tile), and the one-shot call."""
    wl = W.small((24, 20, 150), 140, seed=81, w=w, ht_kind="normal")
    m = magnet(wl)
    assert m.fft_lengths()[2] == 512
    mask = np.zeros(wl.out_shape, dtype=np.uint8)
    rng = np.random.default_rng(82)
    for z in planes:
        mask[z] = rng.random(wl.out_shape[1:]) < 0.4
    Htf = wl.Ht_field()
    rho = wl.rho()
    rho_t = torch.from_numpy(rho).to(DEV)
    m.set_target(torch.from_numpy(mask).to(DEV), Ht=torch.from_numpy(Htf).to(DEV), w=w)
    J1, G1 = m.evaluate(rho_t)
    J2, G2 = m.objective_and_gradient(rho_t, torch.from_numpy(mask).to(DEV), Ht=torch.from_numpy(Htf).to(DEV), w=w)
    op = oracle_op(wl)
    Jr, Gr, _ = O.objective_and_gradient(op, rho, wl.M0_const(), wl.p, mask, Htf, w)
    for J, G in ((J1, G1), (J2, G2)):
        assert abs(J - Jr) <= 1e-5 * abs(Jr)
        assert rel_l2(G.cpu().numpy(), Gr) <= 1e-4
    H = m.stray_field(rho_t).cpu().numpy()
    Hr = op.forward(O.magnetization(rho, wl.M0_const(), wl.p))
    assert rel_l2(H, Hr) <= 1e-5


@pytest.mark.parametrize("shape,axis", [((140, 18, 12, 9), 0), ((150, 33, 10, 10), 0), ((20, 16, 140, 130), 2)])
def test_length_512_varying_magnetization(shape, axis):
    """A varying M0 on grids padded to 512 along x or z: three magnetization spectra in and
    out; along x the chain rule that sums the three components' inverse x transforms (the
    32 x 16 form forms only the kept half of each row), along z the cluster z pass of three
    inputs (half-zero forward stage, kept-half inverse); prepared and one-shot calls and
    the field against the oracle."""
    nx, ny, nz, nzd = shape
    wl = W.small((nx, ny, nz), nzd, seed=91, m0_kind="vmf", w=(1.0, 0.0, 2.0))
    m = magnet(wl)
    assert m.fft_lengths()[axis] == 512
    mask = wl.mask()
    Htc = tuple(float(v) for v in wl.Ht_const_vec())
    tmask = torch.from_numpy(mask).to(DEV)
    m.set_target(tmask, Ht_const=Htc, w=wl.w)
    rho = wl.rho()
    rho_t = torch.from_numpy(rho).to(DEV)
    out = [m.evaluate(rho_t), m.objective_and_gradient(rho_t, tmask, Ht_const=Htc, w=wl.w)]
    op = oracle_op(wl)
    Jr, Gr, _ = O.objective_and_gradient(op, rho, wl.M0_field(), wl.p, mask, wl.Ht_const_vec(), wl.w)
    for J, G in out:
        assert abs(J - Jr) <= 1e-5 * abs(Jr)
        assert rel_l2(G.cpu().numpy(), Gr) <= 1e-4
    H = m.stray_field(rho_t).cpu().numpy()
    Hr = op.forward(O.magnetization(rho, wl.M0_field(), wl.p))
    assert rel_l2(H, Hr) <= 1e-5
