"""Warm-start network kernels through the C ABI against the float64 oracle.

Per kernel, inputs are rounded to bfloat16 on the host first, so both sides
multiply the same numbers and only the kernel's own float32 accumulation and
output rounding remain:
* a bfloat16 output carries one rounding, |err| <= 2^-8 |ref| (the unit
  roundoff is 2^-9; one more for the float32 sum before it);
* a float32 sum of K products carries |err| <= K 2^-24 sum|terms|, bounded
  here by 1e-5 sum|terms| for the K <= 27 * 96 * 2 of these sizes.
The whole network is compared on an 8^3 grid (batch 2) against the oracle with
the same storage roundings (bfloat16 activations after each conv and pool, a
bfloat16 gradient entering each data- and weight-gradient product), so only float32
summation order differs; and, loosely, against the all-float64 oracle (a
weight gradient sums ~1e3 voxel terms of either sign, so bfloat16 storage
errors, relative to sum|terms|, reach sqrt(1e3) * 2^-9 ~ 6e-2 of the sum).
Sizes are ragged (N * D * H * W not a multiple of the 128-voxel block).
"""

import ctypes

import numpy as np
import pytest
import torch

from oracle import unet as U

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


@pytest.fixture(scope="module")
def L():
    from paper_1707_09898_gb300 import _lib

    return _lib.lib()


def p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def S():
    return ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)


def bf16_round(a):
    """Round-to-nearest-even to bfloat16, returned as float64 (no NaN/inf inputs)."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def to_bf16_dev(a):
    t = torch.from_numpy(np.ascontiguousarray(bf16_round(a), np.float32)).to(DEV)
    return t.to(torch.bfloat16)  # exact: the values are bfloat16 already


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(DEV)


def wf_wb(L, W):
    """Packed bfloat16 weight copies (forward, backward data) of W [27][cin][cout], made by
    the library's packing kernel."""
    cin, cout = W.shape[1], W.shape[2]
    wf = torch.empty(27 * cin * cout, dtype=torch.bfloat16, device=DEV)
    wb = torch.empty_like(wf)
    assert L.tmn_pack_conv_weights(p(f32(W)), p(wf), p(wb), cin, cout, S()) == 0
    return wf, wb


def net_status(L):
    st = ctypes.c_uint(1)
    assert L.tmn_status(ctypes.byref(st)) == 0
    return st.value


DIMS = (2, 5, 6, 7)  # N, D, H, W: 420 voxels


@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 32), (32, 64), (48, 16), (96, 32), (64, 64)])
def test_conv_forward(L, cin, cout):
    rng = np.random.default_rng(cin * 100 + cout)
    x = bf16_round(rng.normal(size=DIMS + (cin,)))
    W = bf16_round(rng.normal(0, 0.1, size=(27, cin, cout)))
    b = rng.normal(0, 0.1, size=cout).astype(np.float32).astype(np.float64)
    out = torch.empty(DIMS + (cout,), dtype=torch.bfloat16, device=DEV)
    for relu in (0, 1):
        Wf, _ = wf_wb(L, W)
        assert L.tmn_conv3d_forward(p(to_bf16_dev(x)), p(Wf), p(f32(b)), p(out), *DIMS, cin, cout, relu, S()) == 0
        got = out.float().cpu().numpy()
        ref = U.conv(x, W, b)
        if relu:
            ref = np.maximum(ref, 0)
        bound = U.conv(np.abs(x), np.abs(W), np.abs(b))
        assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * bound)
    assert net_status(L) == 0


@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 32), (32, 64), (48, 16), (96, 32), (64, 64)])
def test_conv_backward_data_and_weight(L, cin, cout):
    rng = np.random.default_rng(7 + cin * 100 + cout)
    x = bf16_round(rng.normal(size=DIMS + (cin,)))
    W = bf16_round(rng.normal(0, 0.1, size=(27, cin, cout)))
    g = bf16_round(rng.normal(size=DIMS + (cout,)))  # the data gradient rounds dout to bfloat16
    dx_ref, dW_ref, db_ref = U.conv_backward(x, W, g)
    _, Wb = wf_wb(L, W)
    gd = f32(g)
    din = torch.full(DIMS + (cin,), 0.5, dtype=torch.float32, device=DEV)
    assert L.tmn_conv3d_backward_data(p(gd), p(Wb), p(din), *DIMS, cin, cout, 0, S()) == 0
    bound = U.conv_backward(np.abs(x), np.abs(W), np.abs(g))[0]
    assert np.all(np.abs(din.cpu().numpy() - dx_ref) <= 1e-5 * bound + 1e-30)
    assert L.tmn_conv3d_backward_data(p(gd), p(Wb), p(din), *DIMS, cin, cout, 1, S()) == 0  # accumulate
    assert np.all(np.abs(din.cpu().numpy() - 2 * dx_ref) <= 2e-5 * bound + 1e-30)
    assert net_status(L) == 0
    # weight gradient: float32 sums of bfloat16 products (dout rounded to bfloat16, as the
    # kernel does; the bias gradient sums the float32 values)
    g32 = bf16_round(rng.normal(size=DIMS + (cout,)))
    _, dW_ref, db_ref = U.conv_backward(x, W, g32)
    _, dWb, dbb = U.conv_backward(np.abs(x), W, np.abs(g32))
    dW = torch.empty(27, cin, cout, device=DEV)
    db = torch.empty(cout, device=DEV)
    nvox = int(np.prod(DIMS))
    base = L.tmn_conv3d_backward_weight_work(nvox, cin, cout)
    per_blk = 4 * (cin // 16) * 128 * cout
    for blocks in (1, 2, 9, 27):  # one partial set per block of voxels (27: one 16-voxel chunk each)
        work = torch.empty(base + (blocks - 1) * per_blk, device=DEV)
        assert L.tmn_conv3d_backward_weight(p(to_bf16_dev(x)), p(f32(g32)), p(dW), p(db), p(work), work.numel(),
                                            *DIMS, cin, cout, S()) == 0
        assert np.all(np.abs(dW.cpu().numpy() - dW_ref) <= 1e-5 * dWb + 1e-30)
        assert np.all(np.abs(db.cpu().numpy() - db_ref) <= 1e-5 * dbb + 1e-30)
    assert net_status(L) == 0
    work = torch.empty(base - 1, device=DEV)
    assert L.tmn_conv3d_backward_weight(p(to_bf16_dev(x)), p(f32(g32)), p(dW), p(db), p(work), work.numel(), *DIMS,
                                        cin, cout, S()) == -5


# rows of W = 8 .. 64 voxels take the halo-tile kernels (rows staged once per block, shared by
# the 27 taps; the weight gradient's tiles are one plane x 128 / W rows); D and H ragged
# against the tiles
HALO = [((1, 3, 17, 8), 16, 16), ((2, 3, 9, 16), 32, 64), ((1, 5, 7, 32), 96, 32), ((1, 3, 3, 64), 48, 16),
        ((1, 2, 4, 64), 16, 32), ((2, 1, 2, 16), 64, 64)]


@pytest.mark.parametrize("dims,cin,cout", HALO)
def test_conv_halo_forward_and_backward_data(L, dims, cin, cout):
    rng = np.random.default_rng(int(np.prod(dims)) + cin * 100 + cout)
    x = bf16_round(rng.normal(size=dims + (cin,)))
    W = bf16_round(rng.normal(0, 0.1, size=(27, cin, cout)))
    b = rng.normal(0, 0.1, size=cout).astype(np.float32).astype(np.float64)
    Wf, Wb = wf_wb(L, W)
    out = torch.empty(dims + (cout,), dtype=torch.bfloat16, device=DEV)
    for relu in (0, 1):
        assert L.tmn_conv3d_forward(p(to_bf16_dev(x)), p(Wf), p(f32(b)), p(out), *dims, cin, cout, relu, S()) == 0
        ref = U.conv(x, W, b)
        if relu:
            ref = np.maximum(ref, 0)
        bound = U.conv(np.abs(x), np.abs(W), np.abs(b))
        assert np.all(np.abs(out.float().cpu().numpy() - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * bound)
    g = bf16_round(rng.normal(size=dims + (cout,)))
    dx_ref = U.conv_backward(x, W, g)[0]
    bound = U.conv_backward(np.abs(x), np.abs(W), np.abs(g))[0]
    din = torch.full(dims + (cin,), 0.5, dtype=torch.float32, device=DEV)
    assert L.tmn_conv3d_backward_data(p(f32(g)), p(Wb), p(din), *dims, cin, cout, 0, S()) == 0
    assert np.all(np.abs(din.cpu().numpy() - dx_ref) <= 1e-5 * bound + 1e-30)
    assert L.tmn_conv3d_backward_data(p(f32(g)), p(Wb), p(din), *dims, cin, cout, 1, S()) == 0  # accumulate
    assert np.all(np.abs(din.cpu().numpy() - 2 * dx_ref) <= 2e-5 * bound + 1e-30)
    # weight gradient by halo tiles: one float32 partial per persistent block, 1, 3 or as many
    # blocks as the work buffer allows
    _, dW_ref, db_ref = U.conv_backward(x, W, g)
    _, dWb, dbb = U.conv_backward(np.abs(x), W, np.abs(g))
    dW = torch.empty(27, cin, cout, device=DEV)
    db = torch.empty(cout, device=DEV)
    base = L.tmn_conv3d_backward_weight_work(int(np.prod(dims)), cin, cout)
    for nblk in (1, 3, 1000):
        work = torch.empty(max(base, nblk * 27 * cin * cout), device=DEV)
        assert L.tmn_conv3d_backward_weight(p(to_bf16_dev(x)), p(f32(g)), p(dW), p(db), p(work), work.numel(),
                                            *dims, cin, cout, S()) == 0
        assert np.all(np.abs(dW.cpu().numpy() - dW_ref) <= 1e-5 * dWb + 1e-30)
        assert np.all(np.abs(db.cpu().numpy() - db_ref) <= 1e-5 * dbb + 1e-30)
    assert net_status(L) == 0


def test_argument_checks(L):
    t = torch.empty(16, device=DEV)
    assert L.tmn_conv3d_forward(p(t), p(t), None, p(t), 1, 1, 1, 1, 16, 24, 0, S()) == -1  # Cout 24
    assert L.tmn_conv3d_forward(p(t), p(t), None, p(t), 1, 1, 1, 1, 8, 16, 0, S()) == -1   # Cin 8
    assert L.tmn_conv3d_backward_data(p(t), p(t), p(t), 1, 1, 1, 1, 80, 16, 0, S()) == -1  # Cin 80
    assert L.tmn_conv3d_forward(None, p(t), None, p(t), 1, 1, 1, 1, 16, 16, 0, S()) == -1


def test_pool_upcat_relu(L):
    rng = np.random.default_rng(11)
    N, D, H, W, C = 2, 4, 6, 8, 16
    x = bf16_round(rng.normal(size=(N, D, H, W, C)))
    out = torch.empty(N, D // 2, H // 2, W // 2, C, dtype=torch.bfloat16, device=DEV)
    assert L.tmn_pool(p(to_bf16_dev(x)), p(out), N, D, H, W, C, S()) == 0
    ref = U.pool(x)
    assert np.all(np.abs(out.float().cpu().numpy() - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6 * np.abs(x).max())
    g = rng.normal(size=ref.shape).astype(np.float32)
    gin = torch.full((N, D, H, W, C), 0.25, device=DEV)
    assert L.tmn_pool_backward(p(f32(g)), p(gin), N, D, H, W, C, 1, S()) == 0
    assert np.allclose(gin.cpu().numpy(), 0.25 + U.pool_backward(g), rtol=1e-6, atol=1e-7)
    # upsample + concat: an exact copy; its backward: child sums and a slice
    C1, C2 = 32, 16
    xc = bf16_round(rng.normal(size=(N, D // 2, H // 2, W // 2, C1)))
    sk = bf16_round(rng.normal(size=(N, D, H, W, C2)))
    u = torch.empty(N, D, H, W, C1 + C2, dtype=torch.bfloat16, device=DEV)
    assert L.tmn_upcat(p(to_bf16_dev(xc)), p(to_bf16_dev(sk)), p(u), N, D, H, W, C1, C2, S()) == 0
    assert np.array_equal(u.float().cpu().numpy(), np.concatenate([U.up(xc), sk], axis=-1))
    gu = rng.normal(size=(N, D, H, W, C1 + C2)).astype(np.float32)
    gx = torch.empty(N, D // 2, H // 2, W // 2, C1, device=DEV)
    gs = torch.full((N, D, H, W, C2), 9.0, device=DEV)
    assert L.tmn_upcat_backward(p(f32(gu)), p(gx), p(gs), N, D, H, W, C1, C2, S()) == 0
    assert np.allclose(gx.cpu().numpy(), U.up_backward(gu[..., :C1].astype(np.float64)), rtol=1e-6, atol=1e-6)
    assert np.array_equal(gs.cpu().numpy(), gu[..., C1:])
    # ReLU backward through a stored activation: zero where act <= 0, bit-exact
    act = bf16_round(rng.normal(size=(3, 5, 7, 16)))
    act[0, 0, 0, :4] = 0.0
    gr = rng.normal(size=act.shape).astype(np.float32)
    gt = f32(gr)
    assert L.tmn_relu_backward(p(gt), p(to_bf16_dev(act)), gr.size, S()) == 0
    assert np.array_equal(gt.cpu().numpy(), np.where(act > 0, gr, 0.0).astype(np.float32))


def test_head_forward_backward(L):
    rng = np.random.default_rng(12)
    nvox, C = 3001, 16
    x = bf16_round(np.maximum(rng.normal(size=(nvox, C)), 0))
    w = rng.normal(0, 0.3, size=C).astype(np.float32).astype(np.float64)
    b = np.array([0.1], np.float32).astype(np.float64)
    tgt = rng.random(nvox).astype(np.float32).astype(np.float64)
    rho = torch.empty(nvox, device=DEV)
    xd = to_bf16_dev(x)
    assert L.tmn_head_forward(p(xd), p(f32(w)), p(f32(b)), p(rho), nvox, C, S()) == 0
    r_ref = U.head_forward(x, w, b)
    assert np.allclose(rho.cpu().numpy(), r_ref, rtol=1e-6, atol=1e-7)
    gx = torch.empty(nvox, C, device=DEV)
    work = torch.empty(256 * (C + 2), device=DEV)
    out = torch.empty(C + 2, device=DEV)
    assert L.tmn_head_backward(p(xd), p(f32(w)), p(rho), p(f32(tgt)), nvox, C, p(gx), p(work), p(out), S()) == 0
    r = rho.cpu().numpy().astype(np.float64)  # the backward uses the stored rho
    dz = 2 * (r - tgt) * r * (1 - r) / nvox
    o = out.cpu().numpy()
    assert np.allclose(gx.cpu().numpy(), dz[:, None] * w, rtol=1e-5, atol=1e-12)
    assert np.allclose(o[:C], x.T @ dz, rtol=1e-4, atol=1e-5 * np.abs(x).T @ np.abs(dz))
    assert np.isclose(o[C], dz.sum(), rtol=1e-4, atol=1e-5 * np.abs(dz).sum())
    assert np.isclose(o[C + 1], np.mean((r - tgt) ** 2), rtol=1e-5)


def test_adamw_and_weight_copies(L):
    rng = np.random.default_rng(13)
    cin, cout = 48, 16
    w = rng.normal(size=(27, cin, cout)).astype(np.float32)
    m = np.zeros_like(w, np.float64)
    v = np.zeros_like(w, np.float64)
    wd, md, vd = f32(w), torch.zeros(w.shape, device=DEV), torch.zeros(w.shape, device=DEV)
    wf = torch.empty(27, cout, cin, dtype=torch.bfloat16, device=DEV)
    wb = torch.empty(27, cin, cout, dtype=torch.bfloat16, device=DEV)
    ref = w.astype(np.float64)
    for step in (1, 2, 3):
        g = rng.normal(size=w.shape).astype(np.float32)
        assert L.tmn_adamw(p(wd), p(f32(g)), p(md), p(vd), w.size, 1e-2, 0.9, 0.999, 1e-8, 1e-2, step, p(wf), p(wb),
                           cin, cout, S()) == 0
        ref, m, v = U.adamw(ref, g.astype(np.float64), m, v, step, 1e-2, 0.9, 0.999, 1e-8, 1e-2)
        got = wd.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.abs(ref).max()
    # the bfloat16 copies are the round-to-nearest-even images of the masters, in both packed layouts
    rb = bf16_round(got)
    pf, pb = packed_layouts(rb)
    assert np.array_equal(wf.float().cpu().numpy().ravel(), pf)
    assert np.array_equal(wb.float().cpu().numpy().ravel(), pb)
    assert L.tmn_pack_conv_weights(p(f32(w)), p(wf), p(wb), cin, cout, S()) == 0
    pf, pb = packed_layouts(bf16_round(w))
    assert np.array_equal(wf.float().cpu().numpy().ravel(), pf)
    assert np.array_equal(wb.float().cpu().numpy().ravel(), pb)


def packed_layouts(W):
    """The tensor-core operand layouts of W [27][cin][cout], written out: per tap and 16-wide
    chunk of the reduced channels, [k-group (2)][GEMM row / 8][8 rows][8 reduced channels];
    forward rows = co (reduced ci), backward-data rows = ci (reduced co)."""
    _, cin, cout = W.shape
    tap, ci, co = np.meshgrid(np.arange(27), np.arange(cin), np.arange(cout), indexing="ij")
    f = ((tap * (cin // 16) + ci // 16) * 16 * cout + ((ci % 16) // 8) * 8 * cout + (co // 8) * 64 + (co % 8) * 8
         + ci % 8)
    b = ((tap * (cout // 16) + co // 16) * 16 * cin + ((co % 16) // 8) * 8 * cin + (ci // 8) * 64 + (ci % 8) * 8
         + co % 8)
    pf, pb = np.zeros(W.size), np.zeros(W.size)
    pf[f.ravel()] = W.ravel()
    pb[b.ravel()] = W.ravel()
    assert len(set(f.ravel())) == W.size and len(set(b.ravel())) == W.size  # both are permutations
    return pf, pb


def test_spec_input(L):
    from paper_1707_09898_gb300 import workloads as W
    from paper_1707_09898_gb300.warmstart import WarmStartNet

    net = WarmStartNet(size=(8, 12, 16))
    foot = np.zeros((2, 12, 16), np.uint8)
    foot[0, 3:7, 5:9] = 1
    foot[1, 1:2, 0:16] = 1
    x = net.spec_input(foot, [0.2, 0.05], [1, 8]).float().cpu().numpy()
    assert x.shape == (2, 8, 12, 16, 16) and not x[..., 3:].any()
    for n, (ht, h) in enumerate(((0.2, 1), (0.05, 8))):
        assert np.array_equal(x[n, :, :, :, 0], np.broadcast_to(foot[n], (8, 12, 16)).astype(np.float32))
        assert np.allclose(x[n, ..., 1], foot[n] * bf16_round(np.float32(ht)))
        assert np.all(x[n, ..., 2] == h / 8.0)
    fp, ht, h = W.config5_spec(W.config5(10000))
    assert fp.shape == (64, 64) and fp.sum() >= 64 and 1 <= h <= 8 and 0.05 <= ht <= 0.3


def _net_vs_oracle(N, D, target, q, seed=21):
    """GPU network loss, rho and parameter gradients next to the oracle's (same bfloat16
    weights; q = None: all-float64 oracle; q = bf16_round: bfloat16 product operands)."""
    from paper_1707_09898_gb300.warmstart import WarmStartNet, init_params

    params = init_params(seed=seed)
    # the oracle multiplies the same bfloat16 weights the tensor cores see
    oparams = {k: ((bf16_round(w) if k != "head" else w.astype(np.float64)), b.astype(np.float64))
               for k, (w, b) in params.items()}
    rng = np.random.default_rng(22)
    x = np.zeros((N, D, D, D, 16))
    x[..., :3] = bf16_round(rng.random((N, D, D, D, 3)))
    tgt = (rng.random((N, D, D, D)) if target == "random" else np.ones((N, D, D, D))).astype(np.float32)
    net = WarmStartNet(size=(D, D, D), params=params)
    rho = net.forward(to_bf16_dev(x)).cpu().numpy()
    loss = float(net.backward(f32(tgt)))
    got = net.grads()
    r_ref, _ = U.forward(oparams, x, q)
    l_ref, g_ref = U.loss_and_grads(oparams, x, tgt.astype(np.float64), q)
    errs = {f"{k}.{'wb'[j]}": np.linalg.norm(got[k][j] - g_ref[k][j]) / np.linalg.norm(g_ref[k][j])
            for k in g_ref for j in (0, 1)}
    print("bf16 products" if q else "float64", f"rho {np.max(np.abs(rho - r_ref)):.2e}",
          f"loss {abs(loss - l_ref) / l_ref:.2e}", {k: f"{e:.1e}" for k, e in errs.items()})
    return np.max(np.abs(rho - r_ref)), abs(loss - l_ref) / l_ref, errs


def test_network_against_oracle_with_bfloat16_products():
    """The whole network against the oracle's bfloat16-operand mode (every product of a
    convolution takes bfloat16 operands, sums exact): the GPU network is that network up
    to float32 summation order, so every parameter gradient agrees to 1e-2 even where it is
    a near-cancelling sum (random targets, 8^3, batch 2)."""
    drho, dloss, errs = _net_vs_oracle(2, 8, "random", bf16_round)
    assert drho <= 1e-4 and dloss <= 1e-4
    assert max(errs.values()) <= 1e-2, errs


def test_network_against_float64_oracle():
    """The whole network against the all-float64 oracle. With every voxel's target above
    the network's output the gradients do not cancel, so the bfloat16 operands move them by
    well under 2e-2 (about 5e-3 measured on the oracle's own two modes at this size), while
    a wrong tap, transposed weight or misrouted skip connection moves them by O(1)."""
    drho, dloss, errs = _net_vs_oracle(2, 32, "ones", None)
    assert drho <= 5e-3 and dloss <= 1e-3
    assert max(errs.values()) <= 2e-2, errs


def _random_batch(rng, N, D):
    x = np.zeros((N, D, D, D, 16))
    x[..., :3] = bf16_round(rng.random((N, D, D, D, 3)))
    return to_bf16_dev(x), f32(rng.random((N, D, D, D)))


def test_training_is_deterministic_and_resumes_bit_exactly():
    from paper_1707_09898_gb300.warmstart import WarmStartNet

    rng = np.random.default_rng(31)
    batches = [_random_batch(rng, 2, 16) for _ in range(4)]
    a = WarmStartNet(size=(16, 16, 16), seed=3)
    losses = [float(a.train_step(x, t, lr=1e-3)) for x, t in batches]
    b = WarmStartNet(size=(16, 16, 16), seed=3)
    for x, t in batches[:2]:
        b.train_step(x, t, lr=1e-3)
    st = b.state()
    c = WarmStartNet(size=(16, 16, 16), seed=99)
    c.set_state(st)
    for x, t in batches[2:]:
        c.train_step(x, t, lr=1e-3)
    pa, pc = a.params(), c.params()
    for k in pa:
        for j in (0, 1):
            assert np.array_equal(pa[k][j], pc[k][j]), k
    assert all(np.isfinite(losses))


def test_training_reduces_the_loss_on_a_fixed_batch():
    from paper_1707_09898_gb300.warmstart import WarmStartNet

    rng = np.random.default_rng(32)
    x, _ = _random_batch(rng, 2, 16)
    # a learnable target: an affine map of the first input channel (random noise is not)
    t = (0.2 + 0.6 * x[..., 0].float()).contiguous()
    net = WarmStartNet(size=(16, 16, 16), seed=4)
    l0 = float(net.train_step(x, t, lr=3e-3))
    for _ in range(40):
        last = float(net.train_step(x, t, lr=3e-3))
    assert last < 0.8 * l0


def test_trained_warm_start_needs_fewer_optimizer_steps():
    """The committed weights (trained on 2000 specs) on 20 held-out specs: the warm start
    reaches the plain run's best J (within 1%) in fewer steps for most specs, and its best
    J within 50 steps is far lower."""
    from paper_1707_09898_gb300 import workloads as W
    from paper_1707_09898_gb300.warmstart import TRAINED, WarmStartNet, evaluate, load_params, summarize

    net = WarmStartNet(params=load_params(TRAINED))
    rows = evaluate(net, list(W.CONFIG5_HELDOUT_SEEDS)[:20])
    s = summarize(rows)
    print(s)
    # the runs are chaotic (a never-shrinking step): robust summaries of 20 specs only
    assert s["specs_warm_fewer_steps"] >= 10
    assert s["median_step_ratio"] >= 1.2
    assert s["best50_warm_over_plain_median"] <= 0.5
    assert s["warm_J0_over_plain_J0_median"] <= 0.1
