"""Projected-gradient optimisation runs: per-iteration log and checkpoint / resume.

The loop minimises J(rho) on the box 0 <= rho <= 1 (Sec. "Methodology", the box
constraint after Eq. 1) with the normalised projected-gradient step
rho <- clip(rho - alpha G / max|G|, 0, 1). One evaluation at the start gives the
first gradient; every iteration is then one tm_evaluate_step call: the step on the
gradient of the previous evaluation, then the objective and its adjoint gradient
at the new density (Eqs. (adjoint1)-(adjoint2)). All arithmetic runs in the CUDA
library; this module keeps the loop state and writes files.

Log: one JSON line per evaluation with k, J, max|dJ/drho|, the volume fraction
sum(rho)/N (the quantity of Fig. 4, Sec. "Validation and Benchmarks") and the share
of intermediate densities 0.1 < rho < 0.9 (the quality measure of Fig. 3).

Checkpoint (.npz): rho and the last gradient (the next step moves along it), k,
alpha, the J history and the caller's configuration with its hash. A run of k + m
iterations and a run of k iterations, saved, resumed in a fresh context and run m
more, give the same densities and objectives bit for bit.
"""

import hashlib
import json

import numpy as np
import torch


def config_hash(config):
    return hashlib.sha256(json.dumps(config, sort_keys=True).encode()).hexdigest()


class Run:
    """State of one projected-gradient run on a Magnet whose target is set (set_target)."""

    def __init__(self, magnet, rho0, alpha=0.1, config=None, log=None, _state=None):
        self.m = magnet
        self.alpha = float(alpha)
        self.config = dict(config or {})
        self.log_path = log
        if _state is not None:
            self.rho, self.G, self.k, self.history = _state
            self.m.check_design(self.rho)
            return
        if not isinstance(rho0, torch.Tensor):
            rho0 = torch.from_numpy(np.ascontiguousarray(rho0, dtype=np.float32))
        self.rho = rho0.to(magnet.device, torch.float32).contiguous().clone()
        self.m.check_design(self.rho)
        self.G = torch.empty_like(self.rho)
        J, _ = self.m.evaluate(self.rho, G=self.G)
        self.k = 0
        self.history = [J]
        self._log(J)

    def _log(self, J):
        if not self.log_path:
            return
        gmax, vf, inter = self.m.iteration_stats(self.rho, self.G)
        with open(self.log_path, "a") as f:
            f.write(json.dumps({"k": self.k, "J": J, "grad_max": gmax, "volume_fraction": vf,
                                "intermediate_fraction": inter}) + "\n")

    def step(self, n=1):
        """n iterations; returns the J of the last evaluation."""
        for _ in range(n):
            J, _ = self.m.evaluate_step(self.rho, self.G, self.alpha, True, reuse_max=True, sync=True)
            self.k += 1
            self.history.append(J)
            self._log(J)
        return self.history[-1]

    def save(self, path):
        np.savez(path, rho=self.rho.cpu().numpy(), G=self.G.cpu().numpy(), k=np.int64(self.k),
                 alpha=np.float64(self.alpha), history=np.asarray(self.history, np.float64),
                 config=np.asarray(json.dumps(self.config, sort_keys=True)),
                 config_hash=np.asarray(config_hash(self.config)))

    @classmethod
    def resume(cls, magnet, path, config=None, log=None):
        """Continue a saved run in `magnet` (same grid and target). If config is given it
        must hash to the saved configuration."""
        d = np.load(path, allow_pickle=False)
        saved = json.loads(str(d["config"]))
        if config is not None and config_hash(dict(config)) != str(d["config_hash"]):
            raise ValueError("checkpoint was written for another configuration")
        if config_hash(saved) != str(d["config_hash"]):
            raise ValueError("checkpoint configuration does not match its hash")
        rho = torch.from_numpy(d["rho"]).to(magnet.device).contiguous()
        G = torch.from_numpy(d["G"]).to(magnet.device).contiguous()
        if tuple(rho.shape) != magnet.design_shape or tuple(G.shape) != magnet.design_shape:
            raise ValueError("checkpoint arrays do not fit this grid")
        state = (rho, G, int(d["k"]), [float(v) for v in d["history"]])
        return cls(magnet, None, alpha=float(d["alpha"]), config=saved, log=log, _state=state)
