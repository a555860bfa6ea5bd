"""Pins of the float64 warm-start network oracle (no GPU).

* conv, pool and upsampling against brute-force loops on tiny inputs;
* the backward-data conv is the adjoint of the forward conv (dot-product test);
* every parameter gradient of the whole network against central differences of
  the loss in float64.
"""

import numpy as np
import pytest

from oracle import unet as U


def brute_conv(x, W, b):
    N, D, H, Wd, _ = x.shape
    out = np.zeros((N, D, H, Wd, W.shape[2]))
    for n in range(N):
        for z in range(D):
            for y in range(H):
                for xx in range(Wd):
                    acc = b.astype(np.float64).copy()
                    for dz in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                zz, yy, x3 = z + dz, y + dy, xx + dx
                                if 0 <= zz < D and 0 <= yy < H and 0 <= x3 < Wd:
                                    acc += x[n, zz, yy, x3] @ W[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)]
                    out[n, z, y, xx] = acc
    return out


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 4, 5, 2))
    W = rng.normal(size=(27, 2, 3))
    b = rng.normal(size=3)
    assert np.allclose(U.conv(x, W, b), brute_conv(x, W, b), rtol=1e-12, atol=1e-12)


def test_conv_single_tap_is_a_shift():
    # only the tap (dz, dy, dx) = (1, 0, -1) set to identity: out[z, y, x] = x[z+1, y, x-1]
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 4, 4, 4, 2))
    W = np.zeros((27, 2, 2))
    W[2 * 9 + 1 * 3 + 0] = np.eye(2)
    out = U.conv(x, W, np.zeros(2))
    assert np.array_equal(out[:, :3, :, 1:], x[:, 1:, :, :3])
    assert not out[:, 3].any() and not out[:, :, :, 0].any()


def test_pool_and_up_brute_force():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 4, 2, 6, 3))
    p = U.pool(x)
    for z in range(2):
        for y in range(1):
            for xx in range(3):
                blk = x[0, 2 * z:2 * z + 2, 2 * y:2 * y + 2, 2 * xx:2 * xx + 2]
                assert np.allclose(p[0, z, y, xx], blk.reshape(-1, 3).mean(axis=0))
    u = U.up(p)
    assert u.shape == x.shape and np.array_equal(u[0, 3, 1, 5], p[0, 1, 0, 2])
    # adjoints: <pool x, g> = <x, pool_backward g>, <up y, g> = <y, up_backward g>
    g = rng.normal(size=p.shape)
    assert np.isclose(np.sum(p * g), np.sum(x * U.pool_backward(g)))
    g2 = rng.normal(size=x.shape)
    assert np.isclose(np.sum(u * g2), np.sum(p * U.up_backward(g2)))


def test_conv_backward_data_is_the_adjoint():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 3, 5, 4, 4))
    W = rng.normal(size=(27, 4, 6))
    g = rng.normal(size=(2, 3, 5, 4, 6))
    dx, dW, db = U.conv_backward(x, W, g)
    lhs = np.sum(U.conv(x, W, np.zeros(6)) * g)
    assert np.isclose(lhs, np.sum(x * dx), rtol=1e-12)
    # the conv is linear in W too: <conv(x, W), g> = <W, dW>
    assert np.isclose(lhs, np.sum(W * dW), rtol=1e-12)
    assert np.allclose(db, g.sum(axis=(0, 1, 2, 3)))


@pytest.fixture(scope="module")
def tiny():
    rng = np.random.default_rng(4)
    params = U.init_params(seed=5)
    x = np.zeros((1, 4, 8, 4, 16))
    x[..., :3] = rng.random((1, 4, 8, 4, 3))
    target = rng.random((1, 4, 8, 4))
    return params, x, target


def test_network_gradients_against_central_differences(tiny):
    params, x, target = tiny
    loss, grads = U.loss_and_grads(params, x, target)
    rng = np.random.default_rng(6)
    h = 1e-6
    # central-difference rounding: about eps * loss / h per evaluation
    atol = 100 * np.finfo(np.float64).eps * loss / h
    for name in [n for n, _, _ in U.LAYERS] + ["head"]:
        for which in (0, 1):
            arr = params[name][which]
            g = grads[name][which]
            assert g.shape == arr.shape, name
            flat = np.flatnonzero(np.abs(g) > 1e-3 * np.abs(g).max()) if np.abs(g).max() > 0 else []
            picks = rng.choice(flat, size=min(4, len(flat)), replace=False) if len(flat) else []
            for f in picks:
                idx = np.unravel_index(f, arr.shape)
                old = arr[idx]
                arr[idx] = old + h
                lp, _ = U.forward(params, x)
                arr[idx] = old - h
                lm, _ = U.forward(params, x)
                arr[idx] = old
                fd = (np.mean((lp - target) ** 2) - np.mean((lm - target) ** 2)) / (2 * h)
                assert abs(fd - g[idx]) <= 1e-5 * abs(g[idx]) + atol, (name, which, idx)
    assert loss > 0


def test_network_input_gradient_chain_reaches_the_first_layer(tiny):
    # a dropped skip or pool term would leave e1a's gradient unchanged when the
    # decoder is cut off; check that e1a's gradient depends on both paths
    params, x, target = tiny
    _, g_full = U.loss_and_grads(params, x, target)
    cut = {k: (v[0].copy(), v[1].copy()) for k, v in params.items()}
    cut["d1a"][0][:, :32, :] = 0.0  # decoder path into d1a removed, skip path kept
    _, g_cut = U.loss_and_grads(cut, x, target)
    assert not np.allclose(g_full["e1a"][0], g_cut["e1a"][0])
    assert np.abs(g_cut["e1a"][0]).max() > 0
