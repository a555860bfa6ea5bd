"""Oracle: the warm-start U-Net in float64 numpy (forward and backward).

TEST INFRASTRUCTURE ONLY -- see the package docstring. The network is not part
of the paper (its optimizer starts from rho = 1); it maps a target
specification to an initial density that the optimizer then refines.

Architecture (channels-last arrays [N][D][H][W][C]):
    x (3 used of 16 channels)
    e1 = relu(conv(relu(conv(x, 16)), 16))           skip 1, full grid
    e2 = relu(conv(relu(conv(pool(e1), 32)), 32))    skip 2, half grid
    b  = relu(conv(relu(conv(pool(e2), 64)), 64))    quarter grid
    d2 = relu(conv(relu(conv([up(b), e2], 32)), 32))
    d1 = relu(conv(relu(conv([up(d2), e1], 16)), 16))
    rho0 = sigmoid(d1 . w_head + b_head);  loss = mean (rho0 - target)^2
conv: 3x3x3, zero padding 1, weights [27][Cin][Cout] with tap = (dz+1)*9+(dy+1)*3+(dx+1);
pool: 2x2x2 mean; up: nearest 2x.

Two precisions, both from the network's definition ("bfloat16 weights, float32
accumulation"):
* q = None: every value in float64 (the exact network for the given weights);
* q = a rounding to bfloat16: every product of a convolution takes bfloat16
  operands -- the weights, the layer inputs (so the activations handed from layer
  to layer are bfloat16) and, in the backward pass, the output gradient in both
  the data-gradient and the weight-gradient product -- while every sum is exact
  and the element-wise steps (bias, ReLU and its mask, pooling, upsampling, the
  head, the bias gradient) act on unrounded values.
"""

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
LAYERS = [("e1a", 16, 16), ("e1b", 16, 16), ("e2a", 16, 32), ("e2b", 32, 32), ("b1", 32, 64), ("b2", 64, 64),
          ("d2a", 96, 32), ("d2b", 32, 32), ("d1a", 48, 16), ("d1b", 16, 16)]


def _shift(x, dz, dy, dx):
    """y[n, z, y, x] = x[n, z+dz, y+dy, x+dx] (zero outside)."""
    p = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    D, H, W = x.shape[1:4]
    return p[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]


def conv(x, W, b):
    out = np.zeros(x.shape[:4] + (W.shape[2],)) + b
    for t, (dz, dy, dx) in enumerate(TAPS):
        out += _shift(x, dz, dy, dx) @ W[t]
    return out


def conv_backward(x, W, g, q=None):
    """(dx, dW, db) of conv(x, W, b) for the output gradient g; q, if given, rounds g where
    it is an operand of a product (the data and the weight gradient), not in the sum db."""
    gq = q(g) if q is not None else g
    dW = np.stack([np.einsum("nzyxi,nzyxo->io", _shift(x, dz, dy, dx), gq) for (dz, dy, dx) in TAPS])
    db = g.sum(axis=(0, 1, 2, 3))
    dx_ = np.zeros_like(x)
    for t, (dz, dy, dx) in enumerate(TAPS):
        dx_ += _shift(gq @ W[t].T, -dz, -dy, -dx)
    return dx_, dW, db


def pool(x):
    N, D, H, W, C = x.shape
    return x.reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4, 6))


def pool_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, 1), 2, 2), 2, 3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 1), 2, 2), 2, 3)


def up_backward(g):
    N, D, H, W, C = g.shape
    return g.reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4, 6))


def relu(x):
    return np.maximum(x, 0.0)


def forward(params, x, q=None):
    """Returns (rho0, cache). params: {name: (W, b)} for LAYERS and 'head': (w[16], b[1]).
    q, if given, rounds every activation that becomes a convolution's input (conv and pool
    outputs) to the product-operand precision; without it the whole network is float64."""
    c = {"x": x}
    q = q if q is not None else (lambda a: a)

    def layer(name, inp):
        W, b = params[name]
        a = q(relu(conv(inp, W, b)))
        c[name] = a
        return a

    e1 = layer("e1b", layer("e1a", x))
    c["p1"] = q(pool(e1))
    e2 = layer("e2b", layer("e2a", c["p1"]))
    c["p2"] = q(pool(e2))
    bb = layer("b2", layer("b1", c["p2"]))
    c["u2"] = np.concatenate([up(bb), e2], axis=-1)
    d2 = layer("d2b", layer("d2a", c["u2"]))
    c["u1"] = np.concatenate([up(d2), e1], axis=-1)
    d1 = layer("d1b", layer("d1a", c["u1"]))
    w, b = params["head"]
    z = d1 @ w + b[0]
    rho = 1.0 / (1.0 + np.exp(-z))
    c["rho"] = rho
    return rho, c


def loss_and_grads(params, x, target, q=None):
    """(loss, grads) of mean (rho0 - target)^2; q as in forward(), also applied to each output
    gradient where it enters a data- or weight-gradient product."""
    rho, c = forward(params, x, q)
    n = rho.size
    loss = float(np.mean((rho - target) ** 2))
    dz = 2.0 * (rho - target) * rho * (1.0 - rho) / n
    w, _ = params["head"]
    grads = {"head": (np.einsum("nzyxc,nzyx->c", c["d1b"], dz), np.array([dz.sum()]))}

    def back(name, inp, g):
        W, _ = params[name]
        g = g * (c[name] > 0)
        gx, gW, gb = conv_backward(inp, W, g, q)
        grads[name] = (gW, gb)
        return gx

    g = dz[..., None] * w
    g = back("d1b", c["d1a"], g)
    g_u1 = back("d1a", c["u1"], g)
    g_e1 = g_u1[..., 32:].copy()
    g = up_backward(g_u1[..., :32])
    g = back("d2b", c["d2a"], g)
    g_u2 = back("d2a", c["u2"], g)
    g_e2 = g_u2[..., 64:].copy()
    g = up_backward(g_u2[..., :64])
    g = back("b2", c["b1"], g)
    g = back("b1", c["p2"], g)
    g_e2 = g_e2 + pool_backward(g)
    g = back("e2b", c["e2a"], g_e2)
    g = back("e2a", c["p1"], g)
    g_e1 = g_e1 + pool_backward(g)
    g = back("e1b", c["e1a"], g_e1)
    back("e1a", x, g)
    return loss, grads


def init_params(seed=0, scale=1.0):
    """He-normal conv weights, small biases; head weights small."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, cin, cout in LAYERS:
        p[name] = (rng.normal(0, scale * np.sqrt(2.0 / (27 * cin)), size=(27, cin, cout)),
                   rng.normal(0, 0.01, size=cout))
    p["head"] = (rng.normal(0, 0.1, size=16), np.zeros(1))
    return p


def adamw(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step (Adam moments with bias correction, decoupled weight decay
    lr * wd * w; Loshchilov and Hutter, "Decoupled Weight Decay Regularization").
    Returns (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return w - lr * (mhat / (np.sqrt(vhat) + eps) + wd * w), m, v


def head_forward(x, w, b):
    """rho0 = sigmoid(x . w + b) per voxel."""
    return 1.0 / (1.0 + np.exp(-(x @ w + b[0])))
