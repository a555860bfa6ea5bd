"""Learned warm start: a 3-level 3-D U-Net from a target specification to an
initial density, which the projected-gradient optimizer then refines.

The paper has no counterpart: its optimizer starts from a uniform density. The
network cannot change the answer, only the number of optimizer steps needed to
reach it, since the optimizer always runs on the network's output.

Network (channels-last [N][D][H][W][C] on the 64^3 design grid):
    input: footprint of the target mask, H_t,z / Ms on it, height / 8
           (3 channels, padded to 16)
    e1 = 2 x conv(16)  ->  pool  ->  e2 = 2 x conv(32)  ->  pool  ->  b = 2 x conv(64)
    d2 = 2 x conv(32) of [up(b), e2];  d1 = 2 x conv(16) of [up(d2), e1]
    rho0 = sigmoid(d1 . w + b)
Every conv is 3x3x3 with ReLU. Weights are float32 masters with bfloat16 copies
for the tensor-core convolutions (float32 accumulate); the loss is the mean
squared error against designs that the plain optimizer produced.

Every operation runs in libtopomag.so (include/topomag_net.h); this module owns
the buffers and the order of the calls.
"""

import ctypes
import os
import time

import numpy as np
import torch

from . import _lib

LAYERS = (("e1a", 16, 16), ("e1b", 16, 16), ("e2a", 16, 32), ("e2b", 32, 32), ("b1", 32, 64), ("b2", 64, 64),
          ("d2a", 96, 32), ("d2b", 32, 32), ("d1a", 48, 16), ("d1b", 16, 16))
LEVEL = {"e1a": 1, "e1b": 1, "e2a": 2, "e2b": 2, "b1": 4, "b2": 4, "d2a": 2, "d2b": 2, "d1a": 1, "d1b": 1}
C_IN = 16     # padded input channels (3 used)
C_USED = 3
BF16, F32, U8 = torch.bfloat16, torch.float32, torch.uint8


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def init_params(seed=0):
    """He-normal float32 conv weights [27][cin][cout] (input channels past the 3 used are zero),
    small biases, small head weights; numpy arrays keyed like LAYERS plus 'head'."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, cin, cout in LAYERS:
        fan = 27 * (C_USED if name == "e1a" else cin)
        w = rng.normal(0.0, np.sqrt(2.0 / fan), size=(27, cin, cout))
        if name == "e1a":
            w[:, C_USED:, :] = 0.0
        p[name] = (w.astype(np.float32), rng.normal(0.0, 0.01, size=cout).astype(np.float32))
    p["head"] = (rng.normal(0.0, 0.1, size=16).astype(np.float32), np.zeros(1, np.float32))
    return p


class WarmStartNet:
    """The U-Net on one GPU: forward (inference), backward and AdamW through the C ABI."""

    def __init__(self, size=(64, 64, 64), device=0, params=None, seed=0):
        D, H, W = size
        if D % 4 or H % 4 or W % 4:
            raise ValueError("grid sizes must be multiples of 4")
        self.size = (D, H, W)
        self.L = _lib.lib()
        self.dev = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self.step_count = 0
        self.P = {}
        for name, cin, cout in LAYERS:
            e = {"cin": cin, "cout": cout}
            e["w"] = torch.empty(27, cin, cout, dtype=F32, device=self.dev)
            e["b"] = torch.empty(cout, dtype=F32, device=self.dev)
            e["wf"] = torch.empty(27, cout, cin, dtype=BF16, device=self.dev)
            e["wb"] = torch.empty(27, cin, cout, dtype=BF16, device=self.dev)
            for k in ("gw", "mw", "vw"):
                e[k] = torch.zeros(27, cin, cout, dtype=F32, device=self.dev)
            for k in ("gb", "mb", "vb"):
                e[k] = torch.zeros(cout, dtype=F32, device=self.dev)
            self.P[name] = e
        self.head = {"w": torch.empty(16, dtype=F32, device=self.dev), "b": torch.empty(1, dtype=F32, device=self.dev),
                     "g": torch.zeros(18, dtype=F32, device=self.dev)}
        for k in ("mw", "vw"):
            self.head[k] = torch.zeros(16, dtype=F32, device=self.dev)
        for k in ("mb", "vb"):
            self.head[k] = torch.zeros(1, dtype=F32, device=self.dev)
        self.load(params if params is not None else init_params(seed))
        self._N = 0

    # -- parameters -------------------------------------------------------------
    def _ck(self, code):
        if code != 0:
            raise _lib.TopomagError(code, "warm-start network call failed")

    def load(self, params):
        s = _stream(self.dev)
        for name, e in self.P.items():
            w, b = params[name]
            e["w"].copy_(torch.from_numpy(np.ascontiguousarray(w, np.float32)))
            e["b"].copy_(torch.from_numpy(np.ascontiguousarray(b, np.float32)))
            self._ck(self.L.tmn_pack_conv_weights(_p(e["w"]), _p(e["wf"]), _p(e["wb"]), e["cin"], e["cout"], s))
        w, b = params["head"]
        self.head["w"].copy_(torch.from_numpy(np.ascontiguousarray(w, np.float32)))
        self.head["b"].copy_(torch.from_numpy(np.ascontiguousarray(b, np.float32)))

    def params(self):
        """Float32 master weights as numpy arrays (same keys as init_params)."""
        out = {name: (e["w"].cpu().numpy(), e["b"].cpu().numpy()) for name, e in self.P.items()}
        out["head"] = (self.head["w"].cpu().numpy(), self.head["b"].cpu().numpy())
        return out

    def grads(self):
        """Gradients of the last backward() as numpy arrays (same keys as init_params)."""
        out = {name: (e["gw"].cpu().numpy(), e["gb"].cpu().numpy()) for name, e in self.P.items()}
        g = self.head["g"].cpu().numpy()
        out["head"] = (g[:16].copy(), g[16:17].copy())
        return out

    def state(self):
        """Everything needed to resume training: masters, Adam moments and the step count."""
        st = {"step": self.step_count}
        for name, e in self.P.items():
            for k in ("w", "b", "mw", "vw", "mb", "vb"):
                st[f"{name}.{k}"] = e[k].cpu().numpy()
        for k in ("w", "b", "mw", "vw", "mb", "vb"):
            st[f"head.{k}"] = self.head[k].cpu().numpy()
        return st

    def set_state(self, st):
        self.step_count = int(st["step"])
        for name, e in self.P.items():
            for k in ("w", "b", "mw", "vw", "mb", "vb"):
                e[k].copy_(torch.from_numpy(np.asarray(st[f"{name}.{k}"])))
            self._ck(self.L.tmn_pack_conv_weights(_p(e["w"]), _p(e["wf"]), _p(e["wb"]), e["cin"], e["cout"],
                                                  _stream(self.dev)))
        for k in ("w", "b", "mw", "vw", "mb", "vb"):
            self.head[k].copy_(torch.from_numpy(np.asarray(st[f"head.{k}"])))

    # -- buffers ----------------------------------------------------------------
    def _alloc(self, N):
        if N == self._N:
            return
        D, H, W = self.size
        g1, g2, g3 = (N, D, H, W), (N, D // 2, H // 2, W // 2), (N, D // 4, H // 4, W // 4)

        def a(shape, c, dt=BF16):
            return torch.empty(shape + (c,), dtype=dt, device=self.dev)

        self.A = {"x": a(g1, C_IN), "e1a": a(g1, 16), "e1b": a(g1, 16), "p1": a(g2, 16), "e2a": a(g2, 32),
                  "e2b": a(g2, 32), "p2": a(g3, 32), "b1": a(g3, 64), "b2": a(g3, 64), "u2": a(g2, 96),
                  "d2a": a(g2, 32), "d2b": a(g2, 32), "u1": a(g1, 48), "d1a": a(g1, 16), "d1b": a(g1, 16)}
        self.rho = torch.empty(g1, dtype=F32, device=self.dev)
        self.G = {"d1b": a(g1, 16, F32), "d1a": a(g1, 16, F32), "u1": a(g1, 48, F32), "e1": a(g1, 16, F32),
                  "e1a": a(g1, 16, F32), "d2b": a(g2, 32, F32), "d2a": a(g2, 32, F32), "u2": a(g2, 96, F32),
                  "e2": a(g2, 32, F32), "e2a": a(g2, 32, F32), "p1": a(g2, 16, F32), "b2": a(g3, 64, F32),
                  "b1": a(g3, 64, F32), "p2": a(g3, 32, F32)}
        # weight-gradient scratch: the bfloat16 copy of the largest output gradient plus the
        # per-block partial sums of up to eight blocks per SM (8 * 160 * 128 * Cout floats)
        nwork = max(self.L.tmn_conv3d_backward_weight_work(N * (D // LEVEL[n]) * (H // LEVEL[n]) * (W // LEVEL[n]),
                                                           ci, co) for n, ci, co in LAYERS)
        self.work = torch.empty(nwork + 8 * 160 * 128 * 64, dtype=F32, device=self.dev)
        self.hwork = torch.empty(256 * 18, dtype=F32, device=self.dev)
        self._N = N

    # -- network input ------------------------------------------------------------
    def spec_input(self, foot, ht, height):
        """Input tensor [N][D][H][W][16] (bfloat16) from footprints [N][H][W] (uint8),
        H_t,z / Ms [N] and heights above the top face [N] (cells)."""
        foot = torch.as_tensor(np.ascontiguousarray(foot, np.uint8)).to(self.dev)
        N = foot.shape[0]
        self._alloc(N)
        ht = torch.as_tensor(np.asarray(ht, np.float32)).to(self.dev)
        hg = torch.as_tensor(np.asarray(height, np.float32) / 8.0).to(self.dev)
        D, H, W = self.size
        self._ck(self.L.tmn_spec_input(_p(foot), _p(ht), _p(hg), _p(self.A["x"]), N, D, H, W, C_IN,
                                       _stream(self.dev)))
        return self.A["x"]

    # -- forward ------------------------------------------------------------------
    def _conv(self, name, src, dst, dims):
        e = self.P[name]
        self._ck(self.L.tmn_conv3d_forward(_p(src), _p(e["wf"]), _p(e["b"]), _p(dst), *dims, e["cin"], e["cout"], 1,
                                           self._s))

    def forward(self, x=None):
        """rho0 [N][D][H][W] (float32) of the input in self.A['x'] (or x, copied there)."""
        if x is not None:
            self._alloc(x.shape[0])
            if x.data_ptr() != self.A["x"].data_ptr():
                self.A["x"].copy_(x)
        self._s = _stream(self.dev)
        A, L, s = self.A, self.L, self._s
        N, (D, H, W) = self._N, self.size
        f1, f2, f3 = (N, D, H, W), (N, D // 2, H // 2, W // 2), (N, D // 4, H // 4, W // 4)
        self._conv("e1a", A["x"], A["e1a"], f1)
        self._conv("e1b", A["e1a"], A["e1b"], f1)
        self._ck(L.tmn_pool(_p(A["e1b"]), _p(A["p1"]), *f1, 16, s))
        self._conv("e2a", A["p1"], A["e2a"], f2)
        self._conv("e2b", A["e2a"], A["e2b"], f2)
        self._ck(L.tmn_pool(_p(A["e2b"]), _p(A["p2"]), *f2, 32, s))
        self._conv("b1", A["p2"], A["b1"], f3)
        self._conv("b2", A["b1"], A["b2"], f3)
        self._ck(L.tmn_upcat(_p(A["b2"]), _p(A["e2b"]), _p(A["u2"]), *f2, 64, 32, s))
        self._conv("d2a", A["u2"], A["d2a"], f2)
        self._conv("d2b", A["d2a"], A["d2b"], f2)
        self._ck(L.tmn_upcat(_p(A["d2b"]), _p(A["e1b"]), _p(A["u1"]), *f1, 32, 16, s))
        self._conv("d1a", A["u1"], A["d1a"], f1)
        self._conv("d1b", A["d1a"], A["d1b"], f1)
        self._ck(L.tmn_head_forward(_p(A["d1b"]), _p(self.head["w"]), _p(self.head["b"]), _p(self.rho),
                                    N * D * H * W, 16, s))
        return self.rho

    # -- backward -----------------------------------------------------------------
    def _back(self, name, inp, g, gin, dims):
        """g: gradient at the layer's (post-ReLU) output, modified in place; gin: input gradient or None."""
        e, L, s = self.P[name], self.L, self._s
        self._ck(L.tmn_relu_backward(_p(g), _p(self.A[name]), g.numel(), s))
        self._ck(L.tmn_conv3d_backward_weight(_p(inp), _p(g), _p(e["gw"]), _p(e["gb"]), _p(self.work),
                                              self.work.numel(), *dims, e["cin"], e["cout"], s))
        if gin is not None:
            self._ck(L.tmn_conv3d_backward_data(_p(g), _p(e["wb"]), _p(gin), *dims, e["cin"], e["cout"], 0, s))

    def backward(self, target):
        """Gradients of mean (rho0 - target)^2 after forward(); returns the loss as a device scalar."""
        A, G, L, s = self.A, self.G, self.L, self._s
        N, (D, H, W) = self._N, self.size
        f1, f2, f3 = (N, D, H, W), (N, D // 2, H // 2, W // 2), (N, D // 4, H // 4, W // 4)
        self._ck(L.tmn_head_backward(_p(A["d1b"]), _p(self.head["w"]), _p(self.rho), _p(target), N * D * H * W, 16,
                                     _p(G["d1b"]), _p(self.hwork), _p(self.head["g"]), s))
        self._back("d1b", A["d1a"], G["d1b"], G["d1a"], f1)
        self._back("d1a", A["u1"], G["d1a"], G["u1"], f1)
        self._ck(L.tmn_upcat_backward(_p(G["u1"]), _p(G["d2b"]), _p(G["e1"]), *f1, 32, 16, s))
        self._back("d2b", A["d2a"], G["d2b"], G["d2a"], f2)
        self._back("d2a", A["u2"], G["d2a"], G["u2"], f2)
        self._ck(L.tmn_upcat_backward(_p(G["u2"]), _p(G["b2"]), _p(G["e2"]), *f2, 64, 32, s))
        self._back("b2", A["b1"], G["b2"], G["b1"], f3)
        self._back("b1", A["p2"], G["b1"], G["p2"], f3)
        self._ck(L.tmn_pool_backward(_p(G["p2"]), _p(G["e2"]), *f2, 32, 1, s))
        self._back("e2b", A["e2a"], G["e2"], G["e2a"], f2)
        self._back("e2a", A["p1"], G["e2a"], G["p1"], f2)
        self._ck(L.tmn_pool_backward(_p(G["p1"]), _p(G["e1"]), *f1, 16, 1, s))
        self._back("e1b", A["e1a"], G["e1"], G["e1a"], f1)
        self._back("e1a", A["x"], G["e1a"], None, f1)
        return self.head["g"][17]

    def adamw(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
        self.step_count += 1
        L, s, t = self.L, _stream(self.dev), self.step_count
        for e in self.P.values():
            self._ck(L.tmn_adamw(_p(e["w"]), _p(e["gw"]), _p(e["mw"]), _p(e["vw"]), e["w"].numel(), lr, b1, b2, eps, wd,
                                 t, _p(e["wf"]), _p(e["wb"]), e["cin"], e["cout"], s))
            self._ck(L.tmn_adamw(_p(e["b"]), _p(e["gb"]), _p(e["mb"]), _p(e["vb"]), e["b"].numel(), lr, b1, b2, eps,
                                 0.0, t, None, None, 0, 0, s))
        h, g = self.head, self.head["g"]
        gp = g.data_ptr()
        self._ck(L.tmn_adamw(_p(h["w"]), ctypes.c_void_p(gp), _p(h["mw"]), _p(h["vw"]), 16, lr, b1, b2, eps, wd, t,
                             None, None, 0, 0, s))
        self._ck(L.tmn_adamw(_p(h["b"]), ctypes.c_void_p(gp + 16 * 4), _p(h["mb"]), _p(h["vb"]), 1, lr, b1, b2, eps,
                             0.0, t, None, None, 0, 0, s))

    def train_step(self, x, target, **adam):
        self.forward(x)
        loss = self.backward(target)
        self.adamw(**adam)
        return loss


# -- plain optimizer runs on the config5 specifications ----------------------------
def run_optimizer(magnet, rho, iters, alpha, stop_below=None):
    """Projected-gradient run on a prepared Magnet from rho (modified in place).
    Returns the list of J_k (J of the density before step k); stops early once J <= stop_below."""
    G = torch.empty_like(rho)
    Js = []
    for _ in range(iters):
        J, _ = magnet.evaluate(rho, G=G)
        Js.append(J)
        if stop_below is not None and J <= stop_below:
            break
        magnet.optimize_step(rho, G, alpha, True)
    return Js


def make_magnet(wl, device=0):
    from .magnet import Magnet

    return Magnet(wl.n_out, wl.nzd, wl.cellsize, M0=wl.M0_const(), p=wl.p, device=device)


def prepare(magnet, wl):
    magnet.set_target(torch.from_numpy(wl.mask()).to(magnet.device), Ht_const=tuple(float(v) for v in
                                                                                    wl.Ht_const_vec()), w=wl.w)


def timed(fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


# -- data, training and evaluation on the config5 specifications ----------------------
def spec_arrays(seeds):
    """(workloads, footprints [n][64][64] uint8, H_t,z / Ms [n], heights [n]) of config5 seeds."""
    from . import workloads as W

    wls = [W.config5(s) for s in seeds]
    specs = [W.config5_spec(wl) for wl in wls]
    return (wls, np.stack([s[0] for s in specs]), np.array([s[1] for s in specs], np.float32),
            np.array([s[2] for s in specs], np.float32))


def plain_designs(seeds, device=0, iters=200, log=None):
    """Runs the plain optimizer from rho = 0.5 on every spec; returns (best designs [n][64][64][64]
    float32 on the device, J histories [n][iters + 1]). The best design is the iterate of lowest J."""
    wls, _, _, _ = spec_arrays(seeds)
    m = make_magnet(wls[0], device)
    out = torch.empty((len(wls),) + wls[0].design_shape, dtype=F32, device=m.device)
    hist = np.zeros((len(wls), iters + 1))
    best = torch.empty(wls[0].design_shape, dtype=F32, device=m.device)
    for i, wl in enumerate(wls):
        prepare(m, wl)
        rho = torch.from_numpy(wl.rho()).to(m.device)
        G = torch.empty_like(rho)
        jbest = np.inf
        for k in range(iters + 1):
            J, _ = m.evaluate(rho, G=G)
            hist[i, k] = J
            if J < jbest:
                jbest = J
                best.copy_(rho)
            if k < iters:
                m.optimize_step(rho, G, wl.alpha, True)
        out[i].copy_(best)
        if log and (i + 1) % 200 == 0:
            log(f"plain designs: {i + 1}/{len(wls)}")
    return out, hist


def train(net, seeds, designs, steps, batch=4, lr=1e-3, wd=1e-4, seed=0, log=None):
    """AdamW on mean (rho0 - design)^2 over random batches of the specs; cosine learning rate."""
    _, foot, ht, hgt = spec_arrays(seeds)
    rng = np.random.default_rng(seed)
    losses = []
    for t in range(steps):
        idx = rng.choice(len(foot), size=batch, replace=False)
        x = net.spec_input(foot[idx], ht[idx], hgt[idx])
        tgt = designs[torch.from_numpy(idx).to(designs.device)].contiguous()
        lr_t = lr * (0.1 + 0.9 * 0.5 * (1.0 + np.cos(np.pi * t / steps))) * min(1.0, (t + 1) / 100)
        loss = net.train_step(x, tgt, lr=lr_t, wd=wd)
        if t % 50 == 0 or t == steps - 1:
            losses.append((t, float(loss)))
            if log and t % 500 == 0:
                log(f"train step {t}: loss {losses[-1][1]:.5f}")
    return losses


def _first_below(Js, thr):
    return next((k for k, J in enumerate(Js) if J <= thr), None)


def evaluate(net, seeds, device=0, iters=200, tol=0.01, extend=2):
    """Per held-out spec, both starts run the same projected-gradient optimizer:
    plain from rho = 0.5, warm from the network's rho0. J_best = the lowest J of the plain
    run's `iters` steps; the target is J <= (1 + tol) J_best. Recorded: the first step each
    run reaches the target (the warm run may go on to extend * iters steps), the lowest J
    of each within 50 / 100 / `iters` steps, and the wall time (CUDA-synchronised) of both
    runs stopped at the target, the warm one including the network's forward pass."""
    wls, foot, ht, hgt = spec_arrays(seeds)
    m = make_magnet(wls[0], device)
    rows = []
    for i, wl in enumerate(wls):
        prepare(m, wl)
        x = net.spec_input(foot[i:i + 1], ht[i:i + 1], hgt[i:i + 1])
        Jp = run_optimizer(m, torch.from_numpy(wl.rho()).to(m.device), iters + 1, wl.alpha)
        Jw = run_optimizer(m, net.forward(x)[0].clone(), extend * iters + 1, wl.alpha)
        jbest = min(Jp)
        thr = (1.0 + tol) * jbest

        def plain():
            return run_optimizer(m, torch.from_numpy(wl.rho()).to(m.device), iters + 1, wl.alpha, stop_below=thr)

        def warm():
            r = net.forward(net.spec_input(foot[i:i + 1], ht[i:i + 1], hgt[i:i + 1]))[0].clone()
            return run_optimizer(m, r, extend * iters + 1, wl.alpha, stop_below=thr)

        _, tp = timed(plain)
        jw_t, tw = timed(warm)
        rows.append({"spec": wl.name, "J0": Jp[0], "J_best": jbest, "J_final": Jp[iters], "warm_J0": Jw[0],
                     "plain_steps": _first_below(Jp, thr), "warm_steps": _first_below(Jw, thr),
                     "plain_s": tp, "warm_s": tw if jw_t[-1] <= thr else None,
                     **{f"plain_best{k}": min(Jp[:k + 1]) for k in (50, 100, iters)},
                     **{f"warm_best{k}": min(Jw[:k + 1]) for k in (50, 100, iters)}})
    return rows


def summarize(rows, iters=200):
    inf = float("inf")
    ps = np.array([r["plain_steps"] for r in rows], float)
    ws = np.array([r["warm_steps"] if r["warm_steps"] is not None else inf for r in rows], float)
    both = [r for r in rows if r["warm_steps"] is not None and r["warm_steps"] <= iters]
    out = {"specs": len(rows),
           "warm_reached_within_budget": int(np.sum(ws <= iters)),
           "warm_reached_within_2x_budget": int(np.sum(np.isfinite(ws))),
           "plain_steps_median": float(np.median(ps)), "warm_steps_median": float(np.median(ws)),
           # a miss counts as never reaching the target: a ratio of 0
           "median_step_ratio": float(np.median(ps / np.maximum(ws, 1.0))),
           "specs_warm_fewer_steps": int(np.sum(ws < ps)),
           "warm_J0_over_plain_J0_median": float(np.median([r["warm_J0"] / r["J0"] for r in rows]))}
    for k in (50, 100, iters):
        out[f"best{k}_warm_over_plain_median"] = float(np.median([r[f"warm_best{k}"] / r[f"plain_best{k}"]
                                                                  for r in rows]))
    if both:
        out["reached_specs_plain_steps_mean"] = float(np.mean([r["plain_steps"] for r in both]))
        out["reached_specs_warm_steps_mean"] = float(np.mean([r["warm_steps"] for r in both]))
        out["reached_specs_plain_ms_mean"] = float(1e3 * np.mean([r["plain_s"] for r in both]))
        out["reached_specs_warm_ms_mean"] = float(1e3 * np.mean([r["warm_s"] for r in both]))
        out["reached_specs_time_ratio"] = out["reached_specs_plain_ms_mean"] / out["reached_specs_warm_ms_mean"]
    return out


TRAINED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "warmstart_c5.npz")
# written by: python -m paper_1707_09898_gb300.warmstart --steps 8000 (2000 training specs, batch 4)


def inference_ms(net, wl, reps=20):
    """Mean CUDA-event time of one forward pass (spec input + network) at batch 1."""
    from .workloads import config5_spec

    f, ht, h = config5_spec(wl)
    for _ in range(3):
        net.forward(net.spec_input(f[None], [ht], [h]))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        net.forward(net.spec_input(f[None], [ht], [h]))
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def conv_profile(net, N=4, reps=10):
    """CUDA-event time per launch of each layer's forward, backward-data and backward-weight
    convolution at batch N on the network's grid (activations from one forward pass), with
    the algorithmic rate 2 * voxels * 27 * Cin * Cout FLOP per launch."""
    D, H, W = net.size
    x = torch.zeros((N, D, H, W, C_IN), dtype=BF16, device=net.dev)
    net.forward(x)
    net.backward(torch.zeros((N, D, H, W), dtype=F32, device=net.dev))
    L, s = net.L, _stream(net.dev)
    dims = LEVEL
    inp = {"e1a": "x", "e1b": "e1a", "e2a": "p1", "e2b": "e2a", "b1": "p2", "b2": "b1", "d2a": "u2", "d2b": "d2a",
           "d1a": "u1", "d1b": "d1a"}
    out = []
    for name, cin, cout in LAYERS:
        f = dims[name]
        dd = (N, D // f, H // f, W // f)
        e = net.P[name]
        src, dst, g = net.A[inp[name]], net.A[name], net.G.get(name, None)
        g = torch.zeros(dd + (cout,), dtype=F32, device=net.dev) if g is None or g.shape[-1] != cout else g
        gin = torch.empty(dd + (cin,), dtype=F32, device=net.dev)
        calls = {
            "fwd": lambda: L.tmn_conv3d_forward(_p(src), _p(e["wf"]), _p(e["b"]), _p(dst), *dd, cin, cout, 1, s),
            "bwd_data": lambda: L.tmn_conv3d_backward_data(_p(g), _p(e["wb"]), _p(gin), *dd, cin, cout, 0, s),
            "bwd_weight": lambda: L.tmn_conv3d_backward_weight(_p(src), _p(g), _p(e["gw"]), _p(e["gb"]),
                                                               _p(net.work), net.work.numel(), *dd, cin, cout, s)}
        flop = 2.0 * np.prod(dd) * 27 * cin * cout
        row = {"layer": name, "cin": cin, "cout": cout, "voxels": int(np.prod(dd))}
        for kind, fn in calls.items():
            if kind == "bwd_data" and name == "e1a":
                continue
            for _ in range(2):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row[kind + "_ms"] = ms
            row[kind + "_tflops"] = flop / (ms * 1e-3) / 1e12
        out.append(row)
    return out


def save_params(path, params):
    np.savez_compressed(path, **{f"{k}.{j}": v[j] for k, v in params.items() for j in (0, 1)})


def load_params(path):
    z = np.load(path)
    names = [n for n, _, _ in LAYERS] + ["head"]
    return {n: (z[f"{n}.0"], z[f"{n}.1"]) for n in names}


def main(argv=None):
    import argparse
    import json

    from . import workloads as W

    ap = argparse.ArgumentParser(description="Train and evaluate the learned warm start on config5 specs.")
    ap.add_argument("--train-specs", type=int, default=len(W.CONFIG5_TRAIN_SEEDS))
    ap.add_argument("--eval-specs", type=int, default=len(W.CONFIG5_HELDOUT_SEEDS))
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default="warmstart_run")
    ap.add_argument("--weights", default=None, help="evaluate these trained weights (.npz) instead of training")
    ap.add_argument("--profile-convs", action="store_true", help="only time the convolutions (batch --batch)")
    a = ap.parse_args(argv)
    if a.profile_convs:
        rows = conv_profile(WarmStartNet(), N=a.batch)
        for r in rows:
            print(json.dumps(r))
        return
    os.makedirs(a.out, exist_ok=True)
    t0 = time.perf_counter()

    def log(msg):
        print(f"[{time.perf_counter() - t0:7.1f}s] {msg}", flush=True)

    losses, hist = [], np.ones((1, 1))
    if a.weights:
        net = WarmStartNet(params=load_params(a.weights))
    else:
        tr = list(W.CONFIG5_TRAIN_SEEDS)[:a.train_specs]
        designs, hist = plain_designs(tr, log=log)
        log(f"plain designs done: median J_best/J0 {np.median(hist.min(1) / hist[:, 0]):.3e}")
        net = WarmStartNet()
        losses = train(net, tr, designs, a.steps, batch=a.batch, lr=a.lr, log=log)
        torch.cuda.synchronize()
        log(f"training done: loss {losses[-1][1]:.5f}")
        del designs
    rows = evaluate(net, list(W.CONFIG5_HELDOUT_SEEDS)[:a.eval_specs])
    summ = summarize(rows)
    summ["inference_ms_batch1"] = inference_ms(net, W.config5(W.CONFIG5_HELDOUT_SEEDS[0]))
    log("evaluation: " + json.dumps(summ))
    save_params(os.path.join(a.out, "weights.npz"), net.params())
    with open(os.path.join(a.out, "result.json"), "w") as f:
        json.dump({"summary": summ, "losses": losses, "rows": rows, "args": vars(a),
                   "train_hist_best_over_J0": [float(v) for v in np.percentile(hist.min(1) / hist[:, 0],
                                                                                [5, 50, 95])]}, f, indent=1)


if __name__ == "__main__":
    main()
