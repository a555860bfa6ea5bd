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

Besides the headline the native line carries, measured in the same process:
  sweep           the same step at 128^3 and 192^3 (padded 256^3, 384^3)
  cufft_baseline  the plain cuFFT pipeline on the 256^3 workload, same protocol
  general         tm_stray_field (full-grid H) and the whole-grid objective route
  e2e             pinned host rho in, host J and dJ/drho out, every step
  cpu_baseline    the float64 oracle on the host cores (all cores and one), with
                  the CUDA path's errors against it at 128^3, 192^3 and 256^3

Arms:
  native (default)  the CUDA library through its C ABI
  cufft             the same pipeline built on cuFFT (comparison baseline)
  reference         the float64 CPU oracle on the host cores

Multi-GPU: the path does not shard (a 3-D FFT convolution needs an all-to-all
transpose); N ranks run independent replicas, value = sum of their evals/s.
"""

import argparse
import ctypes
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

# Measured DRAM bytes (read + write) per launch of the main kernel kinds of the prepared
# 256^3 step, each from one ncu capture of the kernel as built from the named source file;
# a figure is reported only while that file is unchanged.
MEASURED_TRAFFIC = {
    "x_forward": {"bytes": 282.2e6, "source": "paper_1707_09898_gb300/csrc/k_xfwd.cu",  # with the fused step
                  "source_sha1": "c37b74d2d49959d1d27713fd22a6deb58ea25069"},
    "yz_forward": {"bytes": 219.1e6, "source": "paper_1707_09898_gb300/csrc/k_yzfused.cu",
                   "source_sha1": "98227a45ccd29cff2420ec2ac14ce9db3d1caf7f"},
    "y_inverse": {"bytes": 11.1e6, "source": "paper_1707_09898_gb300/csrc/k_yzfused.cu",  # the finishing kernel
                  "source_sha1": "98227a45ccd29cff2420ec2ac14ce9db3d1caf7f"},
    "zy_adjoint": {"bytes": 161.1e6, "source": "paper_1707_09898_gb300/csrc/k_yzfused.cu",
                   "source_sha1": "98227a45ccd29cff2420ec2ac14ce9db3d1caf7f"},
    "x_inverse": {"bytes": 250.6e6, "source": "paper_1707_09898_gb300/csrc/k_xinv.cu",
                  "source_sha1": "1db0b31247b968b8ac460d25b5bff05d1900e42e"},
    "objective": {"bytes": 0.66e6, "source": "paper_1707_09898_gb300/csrc/k_xobj.cu",
                  "source_sha1": "c3bd93ef1d8d2023b6f5163bbec502652dfa6488"},
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["native", "cufft", "reference"], default="native")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-oneshot", action="store_true", help="skip timing the one-shot call")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: no sweep, cuFFT baseline or general-pipeline legs")
    ap.add_argument("--two-call-step", action="store_true",
                    help="prepared path: tm_evaluate + tm_optimize_step per step instead of tm_evaluate_step")
    ap.add_argument("--separate-yz", action="store_true",
                    help="prepared path: y and direct z passes as separate kernels (default: fused)")
    ap.add_argument("--fft", type=int, default=0,
                    help="padded FFT length of every axis of the headline workload (0: the library's default)")
    ap.add_argument("--stray-field-only", action="store_true",
                    help="time tm_stray_field (full-grid H) on the workload and print only that leg")
    ap.add_argument("--m0", choices=["const", "vmf"], default="const",
                    help="magnetization: constant (0, 0, Ms), or spatially varying (von Mises-Fisher)")
    return ap.parse_args(argv)


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


# ---------------------------------------------------------------------------
# SM clocks and clock-event reasons during the timed region.

# NVML clock-event reason bits (nvml.h, nvmlClocksEventReason*)
_REASON_BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
                0x80: "hw_power_brake_slowdown"}


def summarize_clocks(samples, smax, source):
    """{sm_mhz: median of the samples, sm_max_mhz, reasons: the slowdown reasons seen, samples}."""
    sm = sorted(s for s, _ in samples)
    reasons = set()
    for _, r in samples:
        for bit, nm in _REASON_BITS.items():
            if r & bit:
                reasons.add(nm)
    return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
            "samples": len(sm), "source": source}


class NvmlClocks:
    """Polls the SM clock and the clock-event reasons through NVML (read-only queries) every
    `period` seconds on a host thread, so that even a region of a few milliseconds is seen."""

    def __init__(self, torch_device, period=2e-4):
        self.ok = False
        self.period = period
        self.samples = []
        self.smax = None
        try:
            import torch

            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            props = torch.cuda.get_device_properties(torch_device)
            found = False
            if hasattr(props, "pci_bus_id"):
                bus = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
                found = nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) == 0
            if not found:
                return
            self.nv, self.h = nv, h
            mx = ctypes.c_uint(0)
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # 1 = NVML_CLOCK_SM
                self.smax = float(mx.value)
            self._reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            self.ok = True
        except Exception:
            self.ok = False

    def _poll(self):
        clk, rs = ctypes.c_uint(0), ctypes.c_ulonglong(0)
        while not self._stop.is_set():
            if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0 and \
                    self._reasons(self.h, ctypes.byref(rs)) == 0:
                self.samples.append((float(clk.value), int(rs.value)))
            time.sleep(self.period)

    def start(self):
        if not self.ok:
            return
        self.samples = []
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._poll, daemon=True)
        self._t.start()

    def stop(self):
        if not self.ok:
            return None
        self._stop.set()
        self._t.join(timeout=5)
        return summarize_clocks(self.samples, self.smax, "nvml, every 0.2 ms during the timed region")


class SmiClocks:
    """nvidia-smi samples (every 200 ms) over a wider window: the fallback when NVML is not loadable."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    BITS = (0x8, 0x40, 0x20, 0x4)  # the order of the last four query fields

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

    def stop(self, what):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        samples, smax = [], None
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm, smax = float(f[1]), float(f[2])
            except ValueError:
                continue
            bits = sum(b for b, v in zip(self.BITS, f[5:9]) if v.lower() == "active")
            samples.append((sm, bits))
        return summarize_clocks(samples, smax, f"nvidia-smi every 200 ms over {what}")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# Algorithmic bytes.

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
        if not step_fused:  # the update as its own kernel (kind "other")
            out["other"] = 12 * nzd * ny * nx
    else:
        out["x_inverse"] = (obj + chain) / 2
    single = const and len(W) == 1 and tf == 1  # one spectrum, one tensor component
    fuse_f = direct and fused and npl == 1 and fout == 1
    fuse_a = direct and fused and npl == 1 and single
    if fuse_f:
        out["yz_forward"] = s8 * fin * nzd * ny * K + tf * Tzc + s8 * fout * npl * Ly * K
    # with L = 512 the fused adjoint transforms the source along y itself: it reads the source
    # rows (x spectra, ny rows) instead of a y-transformed source plane (Ly rows)
    yfwd_in_adjoint = fuse_a and Ly == 512 and ny <= Ly // 2
    if fuse_a:
        out["zy_adjoint"] = s8 * ain * npl * (ny if yfwd_in_adjoint else Ly) * K + ta * Tzc + s8 * aout * nzd * ny * K
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


def stray_field_bytes(wl, L):
    """Algorithmic bytes per launch of each kernel kind of tm_stray_field (H on the whole grid,
    all three components): x forward of rho^p (one spectrum, constant M0), y forward of the
    design planes, z pass (forward z transform, the tensor components M0 reaches, inverse z
    transform of three field spectra over every output plane), y and x inverse of three
    components."""
    nx, ny, nz = wl.n_out
    nzd = wl.nzd
    Lx, Ly, Lz = L
    K = Lx // 2 + 1
    M0 = list(wl.M0_const())
    e = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    tcomp = sum(_need(e[c], M0) for c in range(3))
    Tcomp = (Lz // 2 + 1) * (Ly // 2 + 1) * K * 4
    return {"x_forward": 4 * nzd * ny * nx + 8 * nzd * ny * K,
            "y_forward": 8 * nzd * K * (ny + Ly),
            "z_pass": 8 * K * Ly * (nzd + 3 * nz) + tcomp * Tcomp,
            "y_inverse": 3 * 8 * nz * K * (Ly + ny),
            "x_inverse": 3 * (8 * nz * ny * K + 4 * nz * ny * nx)}


def step_bytes(prof, ab, prof_steps):
    """Algorithmic bytes of one step: per kind, bytes per launch x launches per step."""
    return sum(ab[k] * prof[k][1] / prof_steps for k in ab if prof.get(k, (0, 0))[1] > 0)


def roofline(prof, ab, prof_steps, hbm, peak_kind, traffic_ok):
    """Roofline of the kind that takes the most time per step, and per-kind rates."""
    kind = max((k for k in prof if prof[k][1] > 0 and k in ab), key=lambda k: prof[k][0])
    t_launch = prof[kind][0] / prof[kind][1] / 1e3
    achieved = ab[kind] / t_launch / 1e9
    traffic = None
    mt = MEASURED_TRAFFIC.get(kind)
    if traffic_ok and mt and mt["source_sha1"] == sha1(os.path.join(ROOT, mt["source"])):
        traffic = mt["bytes"]
    return {"bound": "hbm", "kernel": kind, "achieved": achieved, "peak": hbm, "peak_kind": peak_kind,
            "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
            "alg_bytes_per_launch": ab[kind], "ms_per_launch": t_launch * 1e3,
            "per_kernel_ms_per_step": {k: prof[k][0] / prof_steps for k in prof if prof[k][1] > 0},
            "per_kernel_alg_gbs": {k: ab[k] / (prof[k][0] / prof[k][1] / 1e3) / 1e9
                                   for k in ab if prof.get(k, (0, 0))[1] > 0}}


def m0_of(wl):
    return wl.M0_const() if wl.m0_kind == "const" else wl.M0_field()


def sha1(path):
    with open(path, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


# ---------------------------------------------------------------------------
# The float64 oracle: the CPU baseline leg (also the only place it runs here).

def cpu_baseline(wl, gpu_results):
    """The float64 oracle, as it stands, on the host cores: one evaluation of the 256^3
    workload with every core and with one, one evaluation at each other size with every
    core, and the relative errors of the CUDA path's results at those sizes against it."""
    import numpy as np

    from oracle import convolution as C
    from oracle import objective as O

    from paper_1707_09898_gb300 import workloads as W

    cores = len(os.sched_getaffinity(0))

    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))

    out, errors, more = None, {}, []
    for n in sorted(gpu_results, reverse=True):
        w = wl if n == wl.n_out[0] else W.config4(n, wl.m0_kind)
        t0 = time.time()
        op = C.FFTOperator(C.Geometry(w.n_out, w.nzd, w.cellsize), workers=cores)
        t_setup = time.time() - t0
        rho = w.rho()
        runs = [cores] + ([1] if n == wl.n_out[0] else [])
        for k in runs:
            op.workers = k
            t0 = time.perf_counter()
            J, G, H = O.objective_and_gradient(op, rho, m0_of(w), w.p, w.mask(), w.Ht_const_vec(), w.w)
            dt = time.perf_counter() - t0
            rec = {"value": 1.0 / dt, "unit": UNIT, "cores": k, "n": n, "seconds": dt}
            if n == wl.n_out[0] and k == cores:
                out = dict(rec, kind="oracle",
                           sample=f"one full float64 evaluation (objective + adjoint gradient) of the {n}^3 "
                                  f"workload, scipy.fft workers={cores}; tensor setup ({t_setup:.0f} s) excluded")
            else:
                more.append(rec)
        g = gpu_results[n]
        errors[f"{n}^3"] = {"H_rel_l2": rel(g["H"], H), "G_rel_l2": rel(g["G"], G),
                            "J_rel": abs(g["J"] - J) / abs(J)}
        del op
    out["more"] = more
    out["error_vs_oracle"] = errors
    return out


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


# ---------------------------------------------------------------------------
# The CUDA path.

class Prepared:
    """One workload on the prepared path: tm_set_target once, then per step either one
    tm_evaluate_step call (the update on the previous gradient inside the evaluation's first
    pass) or tm_evaluate + tm_optimize_step."""

    def __init__(self, wl, dev, args, impl="native"):
        import torch

        from paper_1707_09898_gb300 import Magnet

        self.wl, self.dev = wl, dev
        if impl == "cufft":
            from paper_1707_09898_gb300.cufft_pipeline import CufftMagnet as Impl
        else:
            Impl = Magnet
        M0 = wl.M0_const() if wl.m0_kind == "const" else torch.from_numpy(wl.M0_field()).to(dev)
        kw = {"fft_lengths": (args.fft,) * 3} if impl != "cufft" and getattr(args, "fft", 0) else {}
        self.m = Impl(wl.n_out, wl.nzd, wl.cellsize, M0=M0, p=wl.p, device=dev.index or 0, **kw)
        self.rho0 = torch.from_numpy(wl.rho()).to(dev)
        self.rho = self.rho0.clone()
        self.mask = torch.from_numpy(wl.mask()).to(dev)
        self.Htc, self.w = tuple(float(v) for v in wl.Ht_const_vec()), wl.w
        self.G = torch.empty_like(self.rho)
        self.prepared = hasattr(self.m, "set_target")
        self.fused = self.prepared and not args.separate_yz
        if self.prepared:
            self.m.set_fused(self.fused)
            self.m.set_target(self.mask, Ht_const=self.Htc, w=self.w)
        self.one_call = self.prepared and not args.two_call_step
        if self.one_call:
            self.m.evaluate(self.rho, G=self.G, sync=False)  # the gradient the first step moves along

    def step(self, r=None):
        r = self.rho if r is None else r
        m, wl = self.m, self.wl
        if self.one_call:  # the update on the previous gradient, then the evaluation at the new rho
            m.evaluate_step(r, self.G, wl.alpha, True, reuse_max=True, sync=False)
            return
        if self.prepared:
            m.evaluate(r, G=self.G, sync=False)
            m.optimize_step(r, self.G, wl.alpha, True, reuse_max=True)
        else:
            m.objective_and_gradient(r, self.mask, Ht_const=self.Htc, w=self.w, G=self.G, sync=False)
            m.optimize_step(r, self.G, wl.alpha, True)

    def results_at_rho0(self):
        """(J, dJ/drho, H) of the CUDA path at the initial density, as host arrays."""
        import torch

        H = self.m.stray_field(self.rho0).cpu().numpy()
        G = torch.empty_like(self.rho0)
        J, G = self.m.evaluate(self.rho0, G=G)
        return {"J": J, "G": G.cpu().numpy(), "H": H}

    def close(self):
        self.m.close()


def time_loop(fn, steps, warmup, clocks=None, dist=None):
    """ms for `steps` calls of fn(), CUDA events on the current stream after `warmup` calls,
    a device synchronisation (and a barrier across ranks) on both sides."""
    import torch

    for _ in range(max(3, warmup)):
        fn()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(dist)
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    e0.record(s)
    for _ in range(steps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    ck = clocks.stop() if clocks is not None else None
    barrier(dist)
    return e0.elapsed_time(e1), ck


def profile_pass(m, fn, steps):
    """Per-kernel CUDA event times and launch counts over `steps` calls (a separate pass, so the
    event pairs add no gaps to the timed loop)."""
    import torch

    m.profile(True)
    for _ in range(steps):
        fn()
    torch.cuda.synchronize()
    prof = m.profile_read()
    m.profile(False)
    return prof


E2E_BUFFERS = 3  # device/host buffer sets in flight: step i computes while i + 1 uploads and i - 1 downloads
E2E_CHUNKS = 4   # each 64 MiB copy is split over this many streams per direction (several copy engines)


def e2e_loop(p, steps, full):
    """End to end through the public API, every step: that step's rho copied from pinned host
    memory, the evaluation, and its result read back into pinned host memory. full: J and the
    gradient dJ/drho come back (tm_evaluate); else J only of the one-call step
    (tm_evaluate_step). Copies in both directions run on copy streams, E2E_CHUNKS pieces each,
    and overlap the neighbouring steps' kernels; with E2E_BUFFERS buffer sets the host queues
    the upload of step i + 1 before it waits for the results of step i - 1."""
    import torch

    dev, m, NB, K = p.dev, p.m, E2E_BUFFERS, E2E_CHUNKS
    rho_h = torch.from_numpy(p.wl.rho()).pin_memory()
    nb = rho_h.numel() * 4
    bufs = [torch.empty_like(p.rho) for _ in range(NB)]
    Gs = [torch.empty_like(p.rho) for _ in range(NB)]
    G_h = [torch.empty(p.wl.design_shape, dtype=torch.float32).pin_memory() for _ in range(NB)]
    J_h = torch.zeros(NB, dtype=torch.float64).pin_memory()
    ups = [torch.cuda.Stream(dev) for _ in range(K)]
    downs = [torch.cuda.Stream(dev) for _ in range(K)]
    cs = torch.cuda.current_stream(dev)
    ready = [torch.cuda.Event() for _ in range(NB)]      # rho of step i on the device
    computed = [torch.cuda.Event() for _ in range(NB)]   # step i's kernels done
    landed = [[torch.cuda.Event() for _ in range(K)] for _ in range(NB)]  # step i's results on the host
    consumed = [torch.cuda.Event() for _ in range(NB)]   # step i's kernels no longer need bufs[i]
    flat = lambda t: t.view(-1)  # noqa: E731
    n = rho_h.numel()
    cuts = [n * k // K for k in range(K + 1)]

    def upload(i):
        b = i % NB
        for k, st in enumerate(ups):
            with torch.cuda.stream(st):
                st.wait_event(consumed[b])  # the step that used these buffers NB steps ago is done
                flat(bufs[b])[cuts[k]:cuts[k + 1]].copy_(flat(rho_h)[cuts[k]:cuts[k + 1]], non_blocking=True)
        for st in ups[1:]:
            ups[0].wait_stream(st)
        ready[b].record(ups[0])

    for b in range(NB):
        consumed[b].record(cs)
        for e in landed[b]:
            e.record(cs)
    Js = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    upload(0)
    for i in range(steps):
        b = i % NB
        if i + 1 < steps:
            upload(i + 1)
        cs.wait_event(ready[b])
        for e in landed[b]:  # the download of step i - NB has read Gs[b]
            cs.wait_event(e)
        if full:
            m.evaluate(bufs[b], G=Gs[b], sync=False)
        else:
            p.step(bufs[b])
        m.copy_objective(J_h[b])
        computed[b].record(cs)
        if full:  # gradient back on the download streams while the next step computes
            for k, st in enumerate(downs):
                with torch.cuda.stream(st):
                    st.wait_event(computed[b])
                    flat(G_h[b])[cuts[k]:cuts[k + 1]].copy_(flat(Gs[b])[cuts[k]:cuts[k + 1]], non_blocking=True)
                    landed[b][k].record(st)
            consumed[b].record(cs)
        else:
            for k in range(K):
                landed[b][k].record(cs)
            consumed[b].record(cs)
        if i >= NB - 2:  # the results of step j = i - (NB - 2) are awaited
            j = i - (NB - 2)
            for e in landed[j % NB]:
                e.synchronize()
            Js.append(float(J_h[j % NB]))
    for j in range(max(0, steps - (NB - 2)), steps):
        for e in landed[j % NB]:
            e.synchronize()
        Js.append(float(J_h[j % NB]))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert len(Js) == steps
    return dt, {"h2d_bytes_per_step": nb, "d2h_bytes_per_step": 8 + (nb if full else 0)}


def measure(p, args, dist=None, clocks=None):
    """Headline protocol on one Prepared workload: timed loop, then the profiling pass."""
    ms, ck = time_loop(p.step, args.steps, args.warmup, clocks, dist)
    prof, prof_steps = {}, max(1, min(args.steps, 100))
    if hasattr(p.m, "profile"):
        prof = profile_pass(p.m, p.step, prof_steps)
    return ms, ck, prof, prof_steps


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
    from paper_1707_09898_gb300 import workloads as W

    hbm, peak_kind = peaks()
    wl = W.config4(args.n, args.m0)
    p = Prepared(wl, dev, args, impl=args.impl)
    if args.stray_field_only:  # the general pipeline's full-grid field alone (profiling runs)
        H = torch.empty((3,) + wl.out_shape, dtype=torch.float32, device=dev)
        msg, _ = time_loop(lambda: p.m.stray_field(p.rho, out=H), args.steps, args.warmup)
        print(json.dumps({"stray_field": {"value": args.steps / (msg / 1e3), "unit": "calls/s",
                                          "ms_per_call": msg / args.steps, "workload": wl.name}}))
        p.close()
        return
    nv = NvmlClocks(dev)
    smi = None if nv.ok else SmiClocks(local)
    if smi:
        smi.start()
    ms, ck, prof, prof_steps = measure(p, args, dist, nv if nv.ok else None)
    if smi:
        ck = smi.stop("the warm-up, the timed region and the profiling pass")
    ms_max = max_over_ranks(ms, dist)
    J0 = p.m.objective()  # J of the last step
    L = p.m.fft_lengths()
    extras = rank == 0 and ws == 1 and args.impl == "native" and not args.no_extras

    e2e = e2e_J = None
    if not args.no_e2e and p.prepared:
        e2e_loop(p, min(args.steps, 20), full=True)  # warm-up: pinned buffers, streams, first copies
        dt, nbytes = e2e_loop(p, args.steps, full=True)
        dt = max_over_ranks(dt, dist)
        e2e = dict({"value": ws * args.steps / dt, "unit": UNIT, "call": "tm_evaluate (prepared target)",
                    "overlap": f"rho of step i+1 uploaded and dJ/drho of step i-1 downloaded while step i "
                               f"computes; {E2E_BUFFERS} buffer sets, each copy in {E2E_CHUNKS} pieces on "
                               f"separate streams"}, **nbytes)
        e2e_loop(p, min(args.steps, 20), full=False)
        dt, nbytes = e2e_loop(p, args.steps, full=False)
        dt = max_over_ranks(dt, dist)
        e2e_J = dict({"value": ws * args.steps / dt, "unit": UNIT,
                      "call": "tm_evaluate_step (update + evaluation), J read back, dJ/drho stays on the device"},
                     **nbytes)

    # the same step through the one-shot call (mask passed each time, full z transforms
    # restricted to the target planes on the device)
    oneshot = None
    if p.prepared and not args.no_oneshot:
        def one():
            p.m.objective_and_gradient(p.rho, p.mask, Ht_const=p.Htc, w=p.w, G=p.G, sync=False)
            p.m.optimize_step(p.rho, p.G, wl.alpha, True, reuse_max=True)
        ms1, _ = time_loop(one, args.steps, 2)
        oneshot = {"value": args.steps / (ms1 / 1e3), "unit": UNIT, "call": "tm_objective_and_gradient + tm_optimize_step"}

    gpu_results = {}
    if extras and not args.no_cpu_baseline and p.prepared:
        gpu_results[args.n] = p.results_at_rho0()

    roof, sbytes = None, None
    if prof:
        step_fused = p.one_call and L[0] == 512 and wl.m0_kind == "const"
        ab = alg_bytes(wl, L, direct=p.prepared, fused=p.fused, step_fused=step_fused)
        roof = roofline(prof, ab, prof_steps, hbm, peak_kind,
                        p.prepared and args.n == 256 and args.m0 == "const")
        sbytes = step_bytes(prof, ab, prof_steps)
    launches_per_step = sum(v[1] for v in prof.values()) / prof_steps if prof else None

    general = None
    if extras and args.m0 == "const":
        general = {}
        # tm_stray_field: the whole 3-component field on the whole grid
        H = torch.empty((3,) + wl.out_shape, dtype=torch.float32, device=dev)
        sf = lambda: p.m.stray_field(p.rho, out=H)  # noqa: E731
        msg, _ = time_loop(sf, args.steps, args.warmup)
        pg = profile_pass(p.m, sf, prof_steps)
        abg = stray_field_bytes(wl, L)
        bg = step_bytes(pg, abg, prof_steps)
        general["stray_field"] = {
            "value": args.steps / (msg / 1e3), "unit": "calls/s", "ms_per_call": msg / args.steps,
            "alg_bytes_per_call": bg, "frac": bg / (msg / args.steps / 1e3) / 1e9 / hbm,
            "roofline": roofline(pg, abg, prof_steps, hbm, peak_kind, False)}
        del H
    p.close()
    torch.cuda.empty_cache()

    if extras and args.m0 == "const":
        # the whole-grid objective route: the same patch on the top 16 layers (more than the 8
        # planes the direct z sums take), so tm_evaluate runs the z transforms
        import dataclasses

        wl16 = dataclasses.replace(wl, name=wl.name + "_16planes", mask_z=wl.n_out[2] - 16, mask_nz=16)
        q = Prepared(wl16, dev, args)
        msw, _, pw, _ = measure(q, args)
        abw = alg_bytes(wl16, L, direct=False)
        # plus the kernels of kind "other" in this route: the update (rho and G read, rho
        # written) and the mask-extent scan of the one-shot call (the mask read)
        bw = step_bytes(pw, abw, prof_steps) + 12 * wl.design_cells + wl.n_out[0] * wl.n_out[1] * wl.n_out[2]
        general["whole_grid_objective"] = {
            "value": args.steps / (msw / 1e3), "unit": UNIT, "ms_per_step": msw / args.steps,
            "target": "64 x 64 patch on each of the top 16 layers", "call": "tm_evaluate_step",
            "alg_bytes_per_step": bw, "frac": bw / (msw / args.steps / 1e3) / 1e9 / hbm,
            "roofline": roofline(pw, abw, prof_steps, hbm, peak_kind, False)}
        q.close()
        torch.cuda.empty_cache()

    sweep = None
    if extras and args.n == 256:
        sweep = []
        for n in (128, 192):
            wn = W.config4(n, args.m0)
            q = Prepared(wn, dev, argparse.Namespace(**{**vars(args), "fft": 0}))  # default padding
            msn, ckn, pn, _ = measure(q, args)
            Ln = q.m.fft_lengths()
            abn = alg_bytes(wn, Ln, direct=True, fused=q.fused,
                            step_fused=q.one_call and Ln[0] == 512 and wn.m0_kind == "const")
            bn = step_bytes(pn, abn, prof_steps)
            entry = {"workload": wn.name, "cells": list(wn.n_out), "fft": list(Ln),
                     "value": args.steps / (msn / 1e3), "unit": UNIT, "ms_per_step": msn / args.steps,
                     "alg_bytes_per_step": bn, "frac_step": bn / (msn / args.steps / 1e3) / 1e9 / hbm,
                     "roofline": roofline(pn, abn, prof_steps, hbm, peak_kind, False)}
            if not args.no_cpu_baseline:
                gpu_results[n] = q.results_at_rho0()
            q.close()
            torch.cuda.empty_cache()
            if args.m0 == "const":  # the plain cuFFT pipeline on the same workload, same protocol
                qc = Prepared(wn, dev, args, impl="cufft")
                msc_n, _ = time_loop(qc.step, args.steps, args.warmup)
                entry["cufft"] = {"value": args.steps / (msc_n / 1e3), "unit": UNIT, "ms_per_step": msc_n / args.steps}
                entry["vs_cufft"] = entry["value"] / entry["cufft"]["value"]
                qc.close()
                torch.cuda.empty_cache()
            sweep.append(entry)

    cufft = None
    if extras and args.m0 == "const":
        q = Prepared(wl, dev, args, impl="cufft")
        msc, _ = time_loop(q.step, args.steps, args.warmup)
        cufft = {"value": args.steps / (msc / 1e3), "unit": UNIT, "ms_per_step": msc / args.steps,
                 "workload": wl.name, "call": "explicit zero padding, 3-D cuFFT R2C/C2R, full complex64 tensor; "
                                              "objective_and_gradient + update per step"}
        q.close()
        torch.cuda.empty_cache()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    value = job_throughput(ws, args.steps, ms_max)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "impl": args.impl,
        "config": {"workload": wl.name, "cells": list(wl.n_out), "fft": list(L), "step": "update+objective+gradient",
                   "yz": "fused" if p.fused else "separate",
                   "parallelism": f"replicas{ws}", "l2": "working set (>2 GB) larger than L2; no flush"},
        "clocks": ck, "gpu_launches": (int(round(launches_per_step * args.steps)) if launches_per_step else None),
        "roofline": roof,
        "step_bytes": sbytes,
        "step_frac": (sbytes / (ms_max / args.steps / 1e3) / 1e9 / hbm) if sbytes else None,
        "e2e": e2e, "e2e_step_J": e2e_J, "J_first": J0, "oneshot": oneshot,
        "sweep": sweep, "cufft_baseline": cufft, "general": general,
        "vs_cufft": (value / cufft["value"]) if cufft else None,
        "call": (("tm_set_target once; per step tm_evaluate_step (update on the previous gradient, "
                  "then the evaluation)") if p.one_call else
                 "tm_set_target once; per step tm_evaluate + tm_optimize_step") if p.prepared else None,
    }
    if ws == 1 and not args.no_cpu_baseline and args.impl == "native":
        try:
            if not gpu_results:
                raise RuntimeError("no CUDA results to compare")
            line["cpu_baseline"] = cpu_baseline(wl, gpu_results)
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
