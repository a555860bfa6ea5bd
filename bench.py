#!/usr/bin/env python
"""Throughput of the adjoint-gradient evaluation on one GB300 (or N replicas).

Workload: 256^3 cells of 1 mm, design box = output grid, M0 = (0, 0, Ms),
p = 3, rho ~ U[0,1] (seed 7), objective J = sum over a centred 64 x 64 patch of
the top layer of (H_z - 0.2 Ms)^2; padded FFT grid 512^3. One step = one
projected-gradient update and one stray-field + adjoint-gradient evaluation
(forward x/y/z/y/x passes with the fused objective, adjoint passes with the fused
chain rule). The prepared path makes it one call, tm_evaluate_step: the update on
the previous gradient runs inside the first pass of the evaluation at the new rho
(--two-call-step: tm_evaluate + tm_optimize_step). The tensor setup is excluded, as
in the paper's timings.

Arms:
  native (default)  the CUDA library through its C ABI
  cufft             the same pipeline built on cuFFT (comparison baseline)
  reference         the float64 CPU oracle on the host cores

Multi-GPU: the path does not shard (a 3-D FFT convolution needs an all-to-all
transpose); N ranks run independent replicas, value = sum of their evals/s.
"""

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "adjoint-gradient evals/s at 256^3 cells, FP32 vs FP64 oracle; % of HBM peak"
UNIT = "evals/s"

# DRAM bytes (read + write) per launch of the main kernel kinds of the prepared 256^3 step,
# each from one ncu capture (profiles/traffic_c4_256cube.md; the direct z sum of the
# separate path: profiles/zdir_c4_256cube_ncu.md, forward and adjoint launch averaged);
# valid only while the kernel's source file is unchanged.
MEASURED_TRAFFIC = {
    "x_forward": {"bytes": 287.7e6, "source": "paper_1707_09898_gb300/csrc/k_xfwd.cu",  # with the fused step
                  "source_sha1": "f565c14a45fdfca0a5b06e81872532755122bc43"},
    "yz_forward": {"bytes": 219.8e6, "source": "paper_1707_09898_gb300/csrc/k_yzfused.cu",
                   "source_sha1": "a8060f1ef153b7d453354ebcd0021d119cf4472b"},
    "zy_adjoint": {"bytes": 161.7e6, "source": "paper_1707_09898_gb300/csrc/k_yzfused.cu",
                   "source_sha1": "a8060f1ef153b7d453354ebcd0021d119cf4472b"},
    "x_inverse": {"bytes": 250.3e6, "source": "paper_1707_09898_gb300/csrc/k_xinv.cu",
                  "source_sha1": "c25200c4e8f371b6b97bad7060d274435af13925"},
    "z_pass": {"bytes": 330.5e6, "source": "paper_1707_09898_gb300/csrc/k_zdir.cu",
               "source_sha1": "1e01034aaa7e24a5aeb9221956bd20b7f6d468eb"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["native", "cufft", "reference"], default="native")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-oneshot", action="store_true", help="skip timing the one-shot call")
    ap.add_argument("--two-call-step", action="store_true",
                    help="prepared path: tm_evaluate + tm_optimize_step per step instead of tm_evaluate_step")
    ap.add_argument("--separate-yz", action="store_true",
                    help="prepared path: y and direct z passes as separate kernels (default: fused)")
    ap.add_argument("--m0", choices=["const", "vmf"], default="const",
                    help="magnetization: constant (0, 0, Ms), or spatially varying (von Mises-Fisher)")
    return ap.parse_args()


def dist_setup(args):
    import torch

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        return rank, ws, local, dist
    return 0, 1, 0, None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(x, dist):
    """Slowest rank's value (the job's time); works on NCCL (cuda) and gloo (cpu) groups."""
    if dist is None:
        return x
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws, steps, ms_max):
    """Whole-job evals/s of ws independent replicas that each ran `steps` in ms_max (slowest rank)."""
    return ws * steps / (ms_max / 1e3)


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _need(v, u):
    """unique tensor components with a nonzero coefficient in v^T N u"""
    c = [v[0] * u[0], v[1] * u[1], v[2] * u[2], v[0] * u[1] + v[1] * u[0], v[0] * u[2] + v[2] * u[0],
         v[1] * u[2] + v[2] * u[1]]
    return sum(1 for x in c if x != 0)


def alg_bytes(wl, L, direct=True, fused=True, step_fused=False):
    """Algorithmic bytes per launch of each kernel kind for the objective+gradient step.

    Half spectra kx = 0..L/2 only (no padding); components actually carried: with a
    constant M0 the magnetization enters as one spectrum (rho^p, contracted with M0 in
    the z pass) and the adjoint leaves as one (contracted with M0); the forward carries
    the weighted field components, the adjoint their dJ/dH. Only the np planes that hold
    target cells carry the forward field after the z pass and the adjoint source before it.
    fused: the prepared path's y transform of the design planes fused with the direct z
    sum (forward onto one target plane with one output; adjoint always): those kinds read
    or write the x-transformed design planes, the tensor once, and the target planes.
    step_fused: the x forward pass also applies the projected-gradient step (reads G,
    writes the new rho).
    """
    nx, ny, nz = wl.n_out
    nzd = wl.nzd
    Lx, Ly, Lz = L
    K = Lx // 2 + 1
    const = wl.m0_kind == "const"
    W = [c for c in range(3) if wl.w[c] != 0]
    M0 = list(wl.M0_const()) if const else None
    e = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    fin, fout = (1, len(W)) if const else (3, 3)
    ain, aout = (len(W), 1) if const else (3, 3)
    Tcomp = (Lz // 2 + 1) * (Ly // 2 + 1) * K * 4
    if const:
        tf = sum(_need(e[c], M0) for c in W)
        ta = sum(_need(M0, e[c]) for c in W)
    else:
        tf = ta = 6
    npl = int(wl.mask().any(axis=(1, 2)).sum())  # planes holding target cells
    s8 = 8
    m0 = 0 if const else 12 * nzd * ny * nx  # the varying M0 is read by the first and last pass
    Tzc = nzd * (Ly // 2 + 1) * K * 4        # x/y-transformed tensor over nzd offsets, one component
    obj = s8 * npl * ny * K * fout * 2 + npl * ny * nx  # spectra in, adjoint spectra out, mask
    chain = s8 * aout * nzd * ny * K + 8 * nzd * ny * nx + m0
    out = {"x_forward": (12 if step_fused else 4) * nzd * ny * nx + m0 + s8 * fin * nzd * ny * K}
    if direct:  # prepared path: the objective on the target rows is its own kind
        out["objective"] = obj
        out["x_inverse"] = chain
    else:
        out["x_inverse"] = (obj + chain) / 2
    single = const and len(W) == 1 and tf == 1  # one spectrum, one tensor component
    fuse_f = direct and fused and npl == 1 and fout == 1
    fuse_a = direct and fused and npl == 1 and single
    if fuse_f:
        out["yz_forward"] = s8 * fin * nzd * ny * K + tf * Tzc + s8 * fout * npl * Ly * K
    if fuse_a:
        out["zy_adjoint"] = s8 * ain * npl * Ly * K + ta * Tzc + s8 * aout * nzd * ny * K
    # separate y passes: forward of the design planes (unless fused) and of the adjoint
    # source planes; inverse of the target planes and of the design planes (unless fused)
    yf = [s8 * ain * npl * K * (ny + Ly)] + ([] if fuse_f else [s8 * fin * nzd * K * (ny + Ly)])
    yi = [s8 * fout * npl * K * (Ly + ny)] + ([] if fuse_a else [s8 * aout * nzd * K * (Ly + ny)])
    out["y_forward"] = sum(yf) / len(yf)
    out["y_inverse"] = sum(yi) / len(yi)
    zl = []
    if not fuse_f:
        zl.append(s8 * K * Ly * (fin * nzd + fout * npl) + tf * (Tzc if direct else Tcomp))
    if not fuse_a:
        zl.append(s8 * K * Ly * (ain * npl + aout * nzd) + ta * (Tzc if direct else Tcomp))
    if zl:
        out["z_pass"] = sum(zl) / len(zl)
    return out


def m0_of(wl):
    return wl.M0_const() if wl.m0_kind == "const" else wl.M0_field()


def sha1(path):
    with open(path, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


def cpu_baseline(wl, args):
    """The float64 oracle, as it stands, on the host cores: one evaluation of the same workload."""
    import numpy as np

    from oracle import convolution as C
    from oracle import objective as O

    cores = len(os.sched_getaffinity(0))
    t0 = time.time()
    op = C.FFTOperator(C.Geometry(wl.n_out, wl.nzd, wl.cellsize), workers=cores)
    t_setup = time.time() - t0
    rho = wl.rho()
    t0 = time.perf_counter()
    J, G, _ = O.objective_and_gradient(op, rho, m0_of(wl), wl.p, wl.mask(), wl.Ht_const_vec(), wl.w)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one full float64 evaluation (objective + adjoint gradient) of the {wl.n_out[0]}^3 workload, "
                      f"scipy.fft workers={cores}; tensor setup ({t_setup:.0f} s) excluded",
            "seconds": dt, "J": J, "G_norm": float(np.linalg.norm(G))}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1707_09898_gb300 import workloads as W

    wl = W.config4(args.n, args.m0)
    from oracle import convolution as C
    from oracle import objective as O
    from oracle import optimizer as P

    cores = len(os.sched_getaffinity(0))
    op = C.FFTOperator(C.Geometry(wl.n_out, wl.nzd, wl.cellsize), workers=cores)
    rho = wl.rho().astype("float64")
    # each step: one oracle evaluation + update; the timed count is capped so the run stays within minutes
    steps = max(1, min(args.steps, 3))
    warm = min(args.warmup, 1)
    for _ in range(warm):
        J, G, _ = O.objective_and_gradient(op, rho, m0_of(wl), wl.p, wl.mask(), wl.Ht_const_vec(), wl.w)
    t0 = time.perf_counter()
    for _ in range(steps):
        J, G, _ = O.objective_and_gradient(op, rho, m0_of(wl), wl.p, wl.mask(), wl.Ht_const_vec(), wl.w)
        rho = P.projected_gradient_step(rho, G, wl.alpha, True)
    dt = time.perf_counter() - t0
    v = steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": steps,
        "warmup": warm, "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "cells": list(wl.n_out), "fft": [2 * n for n in wl.n_out]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{steps} full float64 evaluations + updates of the {args.n}^3 workload "
                                   f"(requested {args.steps}; capped at 3 to bound the run), workers={cores}"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_native(args):
    import torch

    rank, ws, local, dist = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__

    if rank == 0 or ws == 1:
        __graft_entry__.build()
    barrier(dist)
    __graft_entry__.build()
    from paper_1707_09898_gb300 import Magnet
    from paper_1707_09898_gb300 import workloads as W

    wl = W.config4(args.n, args.m0)
    if args.impl == "cufft":
        from paper_1707_09898_gb300.cufft_pipeline import CufftMagnet as Impl
    else:
        Impl = Magnet
    M0 = wl.M0_const() if wl.m0_kind == "const" else torch.from_numpy(wl.M0_field()).to(dev)
    m = Impl(wl.n_out, wl.nzd, wl.cellsize, M0=M0, p=wl.p, device=local)
    rho0 = torch.from_numpy(wl.rho()).to(dev)
    rho = rho0.clone()
    mask = torch.from_numpy(wl.mask()).to(dev)
    Htc, w = tuple(float(v) for v in wl.Ht_const_vec()), wl.w
    G = torch.empty_like(rho)

    prepared = hasattr(m, "set_target")
    reuse = {"reuse_max": True} if prepared else {}  # max|G| from the chain-rule pass
    fused = prepared and not args.separate_yz
    if prepared:
        m.set_fused(fused)
    if prepared:
        m.set_target(mask, Ht_const=Htc, w=w)

    one_call = prepared and not args.two_call_step

    def step(r=None):
        r = rho if r is None else r
        if one_call:  # the update on the previous gradient, then the evaluation at the new rho
            m.evaluate_step(r, G, wl.alpha, True, reuse_max=True, sync=False)
            return
        if prepared:
            m.evaluate(r, G=G, sync=False)
        else:
            m.objective_and_gradient(r, mask, Ht_const=Htc, w=w, G=G, sync=False)
        m.optimize_step(r, G, wl.alpha, True, **reuse)

    if one_call:
        m.evaluate(rho, G=G, sync=False)  # the gradient the first step moves along
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    J0 = m.objective()
    rho.copy_(rho0)
    launches_per_step = None
    clocks = Clocks(local)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(dist)
    torch.cuda.synchronize()
    clocks.start()
    e0.record(s)
    for _ in range(args.steps):
        step()
    e1.record(s)
    torch.cuda.synchronize()
    ck = clocks.stop()
    barrier(dist)
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, dist)
    # per-kernel times and launch counts from a separate pass with an event pair around
    # every launch (kept out of the timed loop above, where they would add gaps)
    prof = {}
    prof_steps = max(1, min(args.steps, 100))
    if hasattr(m, "profile"):
        m.profile(True)
        for _ in range(prof_steps):
            step()
        torch.cuda.synchronize()
        prof = m.profile_read()
        m.profile(False)
        launches_per_step = sum(v[1] for v in prof.values()) / prof_steps

    # end to end through the public API: pinned host rho in, J out, every step
    e2e = None
    if not args.no_e2e:
        # every step: its input rho copied from pinned host memory into one of two device
        # buffers on a copy stream, one step, and its J copied back into pinned memory.
        # The host queues step i + 1 before it waits for J(i), so the GPU never waits for
        # the host; the copy for step i + 1 is issued after J(i - 1) arrived, i.e. after
        # step i - 1, the last user of that buffer, finished.
        rho_h = torch.from_numpy(wl.rho()).pin_memory()
        bufs = [torch.empty_like(rho), torch.empty_like(rho)]
        cs = torch.cuda.Stream(dev)
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        J_h = torch.zeros(2, dtype=torch.float64).pin_memory()
        J_done = [torch.cuda.Event(), torch.cuda.Event()]
        async_J = hasattr(m, "copy_objective")
        Js = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(cs):
            bufs[0].copy_(rho_h, non_blocking=True)
            ready[0].record(cs)
        for i in range(args.steps):
            torch.cuda.current_stream(dev).wait_event(ready[i % 2])
            step(bufs[i % 2])
            if not async_J:
                Js.append(m.objective())  # 8-byte device-to-host read, synchronises
                if i + 1 < args.steps:
                    with torch.cuda.stream(cs):
                        bufs[(i + 1) % 2].copy_(rho_h, non_blocking=True)
                        ready[(i + 1) % 2].record(cs)
                continue
            m.copy_objective(J_h[i % 2])
            J_done[i % 2].record()
            if i >= 1:
                J_done[(i - 1) % 2].synchronize()
                Js.append(float(J_h[(i - 1) % 2]))
            if i + 1 < args.steps:
                with torch.cuda.stream(cs):
                    bufs[(i + 1) % 2].copy_(rho_h, non_blocking=True)
                    ready[(i + 1) % 2].record(cs)
        if async_J:
            J_done[(args.steps - 1) % 2].synchronize()
            Js.append(float(J_h[(args.steps - 1) % 2]))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, dist)
        assert len(Js) == args.steps
        e2e = {"value": ws * args.steps / dt, "unit": UNIT, "h2d_bytes_per_step": int(rho.numel() * 4),
               "d2h_bytes_per_step": 8,
               "overlap": ("host-to-device copy of step i+1 on a copy stream during step i; J(i) read back "
                           "after step i+1 is queued") if async_J else
                          "host-to-device copy of step i+1 on a copy stream during step i"}

    # the same step through the one-shot call (mask passed each time, full z transforms
    # restricted to the target planes on the device)
    oneshot = None
    if prepared and not args.no_oneshot:
        for _ in range(2):
            m.objective_and_gradient(rho, mask, Ht_const=Htc, w=w, G=G, sync=False)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(args.steps):
            m.objective_and_gradient(rho, mask, Ht_const=Htc, w=w, G=G, sync=False)
            m.optimize_step(rho, G, wl.alpha, True, **reuse)
        e1.record(s)
        torch.cuda.synchronize()
        oneshot = {"value": args.steps / (e0.elapsed_time(e1) / 1e3), "unit": UNIT,
                   "call": "tm_objective_and_gradient + tm_optimize_step"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    value = job_throughput(ws, args.steps, ms_max)
    hbm, peak_kind = peaks()
    L = m.fft_lengths()
    roof = None
    if prof:
        step_fused = one_call and L[0] == 512 and wl.m0_kind == "const"
        ab = alg_bytes(wl, L, direct=prepared, fused=fused, step_fused=step_fused)
        kind = max((k for k in prof if prof[k][1] > 0 and k in ab), key=lambda k: prof[k][0])
        t_launch = prof[kind][0] / prof[kind][1] / 1e3
        achieved = ab[kind] / t_launch / 1e9
        traffic = None
        mt = MEASURED_TRAFFIC.get(kind)
        if prepared and args.n == 256 and args.m0 == "const" and mt and \
                mt["source_sha1"] == sha1(os.path.join(ROOT, mt["source"])):
            traffic = mt["bytes"]
        roof = {"bound": "hbm", "kernel": kind, "achieved": achieved, "peak": hbm, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                "alg_bytes_per_launch": ab[kind], "ms_per_launch": t_launch * 1e3,
                "per_kernel_ms_per_step": {k: prof[k][0] / prof_steps for k in prof},
                "per_kernel_alg_gbs": {k: ab[k] / (prof[k][0] / prof[k][1] / 1e3) / 1e9
                                       for k in ab if prof.get(k, (0, 0))[1] > 0}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "impl": args.impl,
        "config": {"workload": wl.name, "cells": list(wl.n_out), "fft": list(L), "step": "update+objective+gradient",
                   "yz": "fused" if fused else "separate",
                   "parallelism": f"replicas{ws}", "l2": "working set (>2 GB) larger than L2; no flush"},
        "clocks": ck, "gpu_launches": (int(round(launches_per_step * args.steps)) if launches_per_step else None),
        "roofline": roof, "e2e": e2e, "J_first": J0, "oneshot": oneshot,
        "call": (("tm_set_target once; per step tm_evaluate_step (update on the previous gradient, "
                  "then the evaluation)") if one_call else
                 "tm_set_target once; per step tm_evaluate + tm_optimize_step") if prepared else None,
    }
    if ws == 1 and not args.no_cpu_baseline and args.impl == "native":
        try:
            line["cpu_baseline"] = cpu_baseline(wl, args)
        except Exception as ex:  # report, never fall back
            line["cpu_baseline"] = {"error": repr(ex)}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
