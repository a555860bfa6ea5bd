"""The paper's validation problem (Sec. "Validation and Benchmarks") minimised with
L-BFGS-B on the GPU: a 39^3 unit cube magnetized along +z with two layers above it,
rho = 1 at the start, maximise the z field on a small box in those layers. Also
its field-and-gradient problem (Sec. "Optimization of field and gradient").

Reports the quantities of Table I for the finite-difference method (N_iter,
T_stray, T_iter, T_total, setup excluded), the volume fraction against the
number of objective evaluations (the quantity of Fig. 4) and the histogram of
rho (the quantity of Fig. 3).

    python -m paper_1707_09898_gb300.paper_problem [--box 5]
    python -m paper_1707_09898_gb300.paper_problem --field-gradient
"""

import json
import time

import numpy as np
import torch

from . import workloads as W
from .lbfgsb import minimize
from .magnet import Magnet

PAPER_FD_ROW = {"N_iter": 25, "T_stray_ms": 31.0, "T_iter_s": 0.196, "T_total_s": 4.9}  # Table I, "FD"


def setup(wl, device=0):
    m = Magnet(wl.n_out, wl.nzd, wl.cellsize, M0=tuple(float(v) for v in wl.M0_const()), p=wl.p, device=device)
    m.set_target(torch.from_numpy(wl.mask()).to(m.device), Ht_const=tuple(float(v) for v in wl.Ht_const_vec()),
                 w=wl.w)
    return m


def run(box=5, device=0, **lbfgsb_options):
    wl = W.paper_problem(box)
    m = setup(wl, device)
    dev = m.device
    rho0 = torch.from_numpy(wl.rho()).to(dev)
    G = torch.empty_like(rho0)

    def fg(rho):
        J, _ = m.evaluate(rho, G=G)
        return J, G

    fg(rho0)  # warm-up (module loads, first launches)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    res = minimize(fg, rho0, **lbfgsb_options)
    torch.cuda.synchronize(dev)
    t_total = time.perf_counter() - t0
    # the same run again, recording the volume fraction at every evaluation (untimed)
    vf = []

    def fg_rec(rho):
        vf.append(float(rho.double().mean()))
        return fg(rho)

    res2 = minimize(fg_rec, rho0, **lbfgsb_options)
    # one stray-field computation and one objective + gradient evaluation, CUDA events
    H = torch.empty((3,) + wl.out_shape, dtype=torch.float32, device=dev)
    x = res.x.contiguous()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(3):
        m.stray_field(x, out=H)
    ev[0].record()
    for _ in range(20):
        m.stray_field(x, out=H)
    ev[1].record()
    ev[2].record()
    for _ in range(20):
        m.evaluate(x, G=G, sync=False)
    ev[3].record()
    ev[3].synchronize()
    rho = res.x.double().cpu().numpy()
    hist, _ = np.histogram(rho, bins=10, range=(0.0, 1.0))
    return {
        "problem": wl.name, "cells": int(np.prod(wl.out_shape)), "N_iter": res.nit, "nfev": res.nfev,
        "message": res.message, "J": res.fun, "T_total_s": t_total, "T_iter_s": t_total / max(res.nit, 1),
        "T_stray_ms": ev[0].elapsed_time(ev[1]) / 20, "T_eval_ms": ev[2].elapsed_time(ev[3]) / 20,
        "volume_fraction": float(rho.mean()), "intermediate_fraction": float(np.mean((rho > 0.1) & (rho < 0.9))),
        "rho_histogram_10bins": hist.tolist(), "volume_fraction_per_evaluation": vf,
        "J_per_iteration": res.history, "rerun_identical": bool(res2.nit == res.nit and res2.fun == res.fun),
        "paper_FD_row": PAPER_FD_ROW}


def field_gradient_rows(wl, plane, field, strip, beta):
    """Stencil rows of the field-and-gradient objective (Sec. "Optimization of field and
    gradient"): J = -1/2 sum_field H_z^2 - beta/2 sum_strip (dH_z/dn)^2, with dH_z/dn at a
    strip cell c by the central difference (H_z(c+n) - H_z(c-n)) / (2 h_n) along its
    outward normal n. Returns (row_ptr, comp, cell, a, c) for Magnet.set_stencil_objective."""
    nx, ny = wl.n_out[0], wl.n_out[1]

    def cell(y, x):
        return (plane * ny + y) * nx + x

    rp, comp, cells, a, c = [0], [], [], [], []
    for y, x in zip(*np.nonzero(field)):
        comp.append(2)
        cells.append(cell(y, x))
        a.append(1.0)
        c.append(-0.5)
        rp.append(len(cells))
    for y, x, axis, sgn in strip:
        dy, dx = (sgn, 0) if axis == 0 else (0, sgn)
        h = wl.cellsize[1] if axis == 0 else wl.cellsize[0]
        comp += [2, 2]
        cells += [cell(y + dy, x + dx), cell(y - dy, x - dx)]
        a += [1.0 / (2.0 * h), -1.0 / (2.0 * h)]
        c.append(-0.5 * beta)
        rp.append(len(cells))
    return np.array(rp), np.array(comp), np.array(cells), np.array(a), np.array(c)


def run_field_gradient(device=0, **lbfgsb_options):
    """The field-and-gradient problem minimised with L-BFGS-B: iterations, times, the field
    term, the gradient term and the design."""
    wl, field, strip, beta = W.paper_field_gradient()
    m = Magnet(wl.n_out, wl.nzd, wl.cellsize, M0=tuple(float(v) for v in wl.M0_const()), p=wl.p, device=device)
    plane = wl.mask_z
    m.set_stencil_objective(*field_gradient_rows(wl, plane, field, strip, beta))
    rho0 = torch.from_numpy(wl.rho()).to(m.device)
    G = torch.empty_like(rho0)

    def fg(rho):
        J, _ = m.evaluate(rho, G=G)
        return J, G

    fg(rho0)
    torch.cuda.synchronize(m.device)
    t0 = time.perf_counter()
    res = minimize(fg, rho0, **lbfgsb_options)
    torch.cuda.synchronize(m.device)
    t_total = time.perf_counter() - t0
    Hz = m.stray_field(res.x.contiguous())[2, plane].double().cpu().numpy()
    H0 = m.stray_field(rho0)[2, plane].double().cpu().numpy()
    rho = res.x.double().cpu().numpy()

    def terms(Hp):  # mean H_z on the field region, mean |dH_z/dn| on the strip per cell
        grad = [((Hp[y + (s if ax == 0 else 0), x + (s if ax == 1 else 0)] -
                  Hp[y - (s if ax == 0 else 0), x - (s if ax == 1 else 0)]) / 2.0) for y, x, ax, s in strip]
        return float(np.mean(Hp[field])), float(np.mean(np.abs(grad)))

    return {"problem": wl.name, "N_iter": res.nit, "nfev": res.nfev, "message": res.message, "J": res.fun,
            "J0": res.history[0], "T_total_s": t_total, "T_iter_s": t_total / max(res.nit, 1),
            "mean_Hz_field_start_end": [terms(H0)[0], terms(Hz)[0]],
            "mean_abs_dHz_dn_strip_start_end": [terms(H0)[1], terms(Hz)[1]],
            "volume_fraction": float(rho.mean()), "intermediate_fraction": float(np.mean((rho > 0.1) & (rho < 0.9)))}


def main(argv=None):
    import argparse

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--box", type=int, default=5)
    ap.add_argument("--field-gradient", action="store_true", help="the field-and-gradient problem instead")
    a = ap.parse_args(argv)
    print(json.dumps(run_field_gradient() if a.field_gradient else run(box=a.box)))


if __name__ == "__main__":
    main()
