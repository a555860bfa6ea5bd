"""Many independent small optimisations on one GPU at once.

Each specification (its own grid context, target and density) runs the
projected-gradient loop of Sec. "Methodology" (box constraint) on its own CUDA
stream; a block of its steps (evaluate + update) is captured once as a CUDA graph
and replayed, so one Python call submits many steps, and the graphs of different
specifications overlap on the GPU. A 64^3 step is a few short kernels; run alone it
leaves most of the GPU idle between launches, run side by side it does not.
Independent specifications share nothing, so there is no exchange between them;
results equal the specifications' own sequential runs bit for bit (every kernel
of the path is deterministic).

    runs = BatchedRuns([workloads.config5(s) for s in seeds])
    runs.run(200)        # 200 steps of every specification
    runs.rho[i]          # the densities
"""

import time

import torch

from .warmstart import make_magnet, prepare


class BatchedRuns:
    def __init__(self, workloads, device=0, steps_per_graph=10, rho0=None):
        self.wls = list(workloads)
        self.k = int(steps_per_graph)
        self.dev = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self.mags, self.rho, self.G, self.streams, self.graphs = [], [], [], [], []
        for i, wl in enumerate(self.wls):
            m = make_magnet(wl, self.dev)
            prepare(m, wl)
            r0 = rho0[i] if rho0 is not None else torch.from_numpy(wl.rho()).to(self.dev)
            rho = r0.clone().contiguous()
            G = torch.empty_like(rho)
            s = torch.cuda.Stream(self.dev)
            with torch.cuda.stream(s):
                # one eager step first: lazily created buffers and kernel attributes
                # are set up outside the capture; then the density is put back
                m.evaluate(rho, G=G, sync=False)
                m.optimize_step(rho, G, wl.alpha, True, reuse_max=True)
                rho.copy_(r0)
            s.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                for _ in range(self.k):
                    m.evaluate(rho, G=G, sync=False)
                    m.optimize_step(rho, G, wl.alpha, True, reuse_max=True)
            self.mags.append(m)
            self.rho.append(rho)
            self.G.append(G)
            self.streams.append(s)
            self.graphs.append(g)
        torch.cuda.synchronize(self.dev)

    def run(self, steps):
        """Advance every specification by `steps` (a multiple of steps_per_graph)."""
        if steps % self.k:
            raise ValueError("steps must be a multiple of steps_per_graph")
        main = torch.cuda.current_stream(self.dev)
        for s in self.streams:
            s.wait_stream(main)
        for _ in range(steps // self.k):
            for g, s in zip(self.graphs, self.streams):
                with torch.cuda.stream(s):
                    g.replay()
        for s in self.streams:
            main.wait_stream(s)

    def objectives(self):
        """J of every specification's last evaluation (synchronises)."""
        return [m.objective() for m in self.mags]


def sequential(wl, steps, device=0):
    """The same loop, one specification, eager launches (the reference for BatchedRuns)."""
    m = make_magnet(wl, device)
    prepare(m, wl)
    rho = torch.from_numpy(wl.rho()).to(m.device)
    G = torch.empty_like(rho)
    for _ in range(steps):
        m.evaluate(rho, G=G, sync=False)
        m.optimize_step(rho, G, wl.alpha, True, reuse_max=True)
    return rho


def throughput(workloads, steps=200, device=0, steps_per_graph=10):
    """Steps per second summed over specifications: eager one at a time, graphs one at a
    time, and all graphs side by side (CUDA-synchronised wall time; construction and
    capture excluded)."""
    out = {"specs": len(workloads), "steps": steps}
    dev = torch.device("cuda", device)
    t0 = time.perf_counter()
    for wl in workloads:
        sequential(wl, steps, device)
    torch.cuda.synchronize(dev)
    out["eager_sequential_steps_per_s"] = len(workloads) * steps / (time.perf_counter() - t0)
    runs = BatchedRuns(workloads, device, steps_per_graph)
    runs.run(steps_per_graph)  # warm replay
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for g, s in zip(runs.graphs, runs.streams):
        with torch.cuda.stream(s):
            for _ in range(steps // steps_per_graph):
                g.replay()
        s.synchronize()
    out["graph_sequential_steps_per_s"] = len(workloads) * steps / (time.perf_counter() - t0)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    runs.run(steps)
    torch.cuda.synchronize(dev)
    out["graph_concurrent_steps_per_s"] = len(workloads) * steps / (time.perf_counter() - t0)
    return out


def main(argv=None):
    import argparse
    import json

    from . import workloads as W

    ap = argparse.ArgumentParser(description="Throughput of independent 64^3 optimisations run side by side.")
    ap.add_argument("--specs", type=int, default=32)
    ap.add_argument("--steps", type=int, default=200)
    a = ap.parse_args(argv)
    wls = [W.config5(s) for s in list(W.CONFIG5_HELDOUT_SEEDS)[:a.specs]]
    print(json.dumps(throughput(wls, a.steps)))


if __name__ == "__main__":
    main()
