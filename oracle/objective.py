"""Oracle: density model, least-squares objective and adjoint gradient (float64).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Sec. "Methodology":
* density rho in [0, 1] per design cell (Eq. 1 and the relaxation after it);
* penalised magnetization M = rho^p M0, M0 constant or varying (Eq. 2);
* objective J(H(rho), rho) (Eq. (objective_function)); here the weighted
  least-squares form summed over target cells Omega (mask):
      J = sum_{i in Omega} sum_c w_c (H_{i,c} - Ht_{i,c})^2 ;
  its partial derivative g = dJ/dH = 2 w_c (H_c - Ht_c) on Omega, 0 elsewhere;
  dJ/drho at fixed H is zero for this J.
* the field-and-gradient objective of Sec. "Optimization of field and gradient"
  and, generally, quadratic forms in linear combinations of field values
  (stencil_objective), with their exact partial derivatives dJ/dH.
* gradient by the adjoint method (Eqs. (adjoint1)-(adjoint2) and the
  operator form after them): with H = D M and D self-adjoint, the chain rule
  gives dJ/drho_j = p rho_j^(p-1) M0_j . (D g)_j. The paper's operator form
  prints a leading minus that its own benchmark gradient (Sec. "Validation and
  Benchmarks") does not carry; the plain chain rule, checked here against
  central finite differences, is the reading used.
"""

import numpy as np


def magnetization(rho, M0, p):
    """M = rho^p M0 on the design box: (3, nzd, ny, nx). M0 is (3,) or (3, nzd, ny, nx)."""
    rho = np.asarray(rho, dtype=np.float64)
    M0 = np.asarray(M0, dtype=np.float64)
    if M0.ndim == 1:
        M0 = M0[:, None, None, None]
    return (rho ** p)[None] * M0


def objective(H, mask, Ht, w):
    """J = sum over mask of sum_c w_c (H_c - Ht_c)^2 (float64)."""
    H = np.asarray(H, dtype=np.float64)
    m = np.asarray(mask).astype(bool)
    Ht = np.asarray(Ht, dtype=np.float64)
    if Ht.ndim == 1:
        Ht = Ht.reshape(3, 1, 1, 1)
    r = (H - np.broadcast_to(Ht, H.shape))[:, m]
    w = np.asarray(w, dtype=np.float64)
    return float(np.sum(w[:, None] * r * r))


def dJ_dH(H, mask, Ht, w):
    """g = 2 w_c (H_c - Ht_c) on the mask, zero elsewhere: (3, nz, ny, nx)."""
    H = np.asarray(H, dtype=np.float64)
    m = np.asarray(mask).astype(bool)
    Ht = np.asarray(Ht, dtype=np.float64)
    if Ht.ndim == 1:
        Ht = Ht.reshape(3, 1, 1, 1)
    w = np.asarray(w, dtype=np.float64).reshape(3, 1, 1, 1)
    return 2.0 * w * (H - Ht) * m[None]


def chain_rule(rho, M0, p, DgH):
    """dJ/drho_j = p rho_j^(p-1) M0_j . (D g)_j on the design box."""
    rho = np.asarray(rho, dtype=np.float64)
    M0 = np.asarray(M0, dtype=np.float64)
    if M0.ndim == 1:
        M0 = M0[:, None, None, None]
    return p * rho ** (p - 1) * np.sum(M0 * DgH, axis=0)


def objective_and_gradient(op, rho, M0, p, mask, Ht, w):
    """(J, dJ/drho, H) for operator op (forward/adjoint of oracle.convolution)."""
    H = op.forward(magnetization(rho, M0, p))
    J = objective(H, mask, Ht, w)
    g = dJ_dH(H, mask, Ht, w)
    G = chain_rule(rho, M0, p, op.adjoint(g))
    return J, G, H


def stencil_objective(H, rows):
    """J = sum_k c_k r_k^2 with r_k = sum_e a_e H[comp_e, z_e, y_e, x_e] (a quadratic form in
    linear combinations of field values), and g = dJ/dH. rows: sequence of
    (c_k, [(comp, z, y, x, a), ...]). Plain loops, float64."""
    H = np.asarray(H, dtype=np.float64)
    g = np.zeros_like(H)
    J = 0.0
    for c, ents in rows:
        r = 0.0
        for comp, z, y, x, a in ents:
            r += a * H[comp, z, y, x]
        J += c * r * r
        for comp, z, y, x, a in ents:
            g[comp, z, y, x] += 2.0 * c * r * a
    return float(J), g


def field_gradient_objective(H, plane, field, strip, h, beta):
    """Sec. "Optimization of field and gradient": maximise the z field on a region and its
    normal derivative on a strip around three of its sides,
        J = -1/2 sum_{field} H_z^2 - beta/2 sum_{strip} (dH_z/dn)^2 ,
    on the plane z = plane (cell sums stand for the integrals). dH_z/dn at strip cell
    (y, x) with outward normal n: the central difference (H_z(c+n) - H_z(c-n)) / (2 h).
    field: (ny, nx) bool; strip: (y, x, axis, sign) with axis 0 = y, 1 = x. Returns (J, g)."""
    H = np.asarray(H, dtype=np.float64)
    Hz = H[2, plane]
    f = np.asarray(field, dtype=bool)
    g = np.zeros_like(H)
    J = -0.5 * float(np.sum(Hz[f] ** 2))
    g[2, plane][f] = -Hz[f]
    for y, x, axis, sgn in strip:
        dy, dx = (sgn, 0) if axis == 0 else (0, sgn)
        D = (Hz[y + dy, x + dx] - Hz[y - dy, x - dx]) / (2.0 * h)
        J += -0.5 * beta * D * D
        g[2, plane, y + dy, x + dx] += -beta * D / (2.0 * h)
        g[2, plane, y - dy, x - dx] += beta * D / (2.0 * h)
    return float(J), g


def general_objective_and_gradient(op, rho, M0, p, obj):
    """(J, dJ/drho, H) for any objective obj(H) -> (J, dJ/dH) of the field alone."""
    H = op.forward(magnetization(rho, M0, p))
    J, g = obj(H)
    return J, chain_rule(rho, M0, p, op.adjoint(g)), H
