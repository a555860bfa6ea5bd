"""Oracle: box-constrained projected-gradient update on the density (float64).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

The paper minimises J over 0 <= rho <= 1 with a bound-constrained quasi-Newton
method (Sec. "Methodology", the box constraint after Eq. 1; Sec.
"Discretization", last paragraph). The update used here is the simpler
projected gradient step on the same box:
    rho <- clip(rho - alpha * G / max|G|, 0, 1)      (normalize = True)
    rho <- clip(rho - alpha * G, 0, 1)               (normalize = False)
with no update when max|G| = 0.
"""

import numpy as np

from .objective import objective_and_gradient


def projected_gradient_step(rho, G, alpha, normalize=True):
    rho = np.asarray(rho, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    if normalize:
        gmax = float(np.max(np.abs(G))) if G.size else 0.0
        if gmax == 0.0:
            return rho.copy()
        step = alpha * G / gmax
    else:
        step = alpha * G
    return np.clip(rho - step, 0.0, 1.0)


def optimize(op, rho0, M0, p, mask, Ht, w, iters, alpha, normalize=True, callback=None):
    """Plain loop of (J, G) evaluations and projected steps. Returns (rho, [J_k])."""
    rho = np.asarray(rho0, dtype=np.float64).copy()
    history = []
    for k in range(iters):
        J, G, _ = objective_and_gradient(op, rho, M0, p, mask, Ht, w)
        history.append(J)
        if callback is not None:
            callback(k, rho, J, G)
        rho = projected_gradient_step(rho, G, alpha, normalize)
    return rho, history
