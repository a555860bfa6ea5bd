"""L-BFGS-B on the GPU against SciPy's L-BFGS-B, the minimiser the paper uses.

With a float64 objective both run the same algorithm in float64, so the iterates
agree to rounding; only the order of the length-n sums differs (block partials
here, numpy's pairwise sums there), and that difference grows along a run by the
problem's sensitivity. On the topology objective the GPU evaluates J and G in
float32 while SciPy drives the float64 oracle, so iterates agree to the float32
evaluation error.
"""

import numpy as np
import pytest
import torch
from scipy.optimize import minimize as sp_minimize
from scipy.optimize import rosen, rosen_der

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


def scipy_run(fg_np, x0, lo, hi, **opts):
    xs = []
    res = sp_minimize(fg_np, x0, jac=True, method="L-BFGS-B", bounds=[(lo, hi)] * len(x0),
                      callback=lambda xk: xs.append(xk.copy()), options=opts)
    return res, xs


def gpu_run(fg_t, x0, lo, hi, **kw):
    from paper_1707_09898_gb300.lbfgsb import minimize

    xs = []
    res = minimize(fg_t, torch.from_numpy(np.asarray(x0, np.float64)).to(DEV), lo, hi,
                   callback=lambda x, f: xs.append(x.cpu().numpy().copy()), **kw)
    return res, xs


def quad_problem(n, seed, rank=None):
    rng = np.random.default_rng(seed)
    if rank is None:
        A = rng.normal(size=(n, n))
        A = A @ A.T / n + 0.1 * np.eye(n)
        b = rng.normal(size=n) * 2
        At, bt = torch.from_numpy(A).to(DEV), torch.from_numpy(b).to(DEV)
        return (lambda x: (0.5 * x @ A @ x + b @ x, A @ x + b),
                lambda x: (float(0.5 * x @ (At @ x) + bt @ x), At @ x + bt))
    # diagonal plus low-rank coupling, large n
    a = rng.uniform(0.5, 2.0, n)
    b = rng.normal(size=n)
    U = rng.normal(size=(rank, n)) / np.sqrt(n)
    at, bt, Ut = (torch.from_numpy(v).to(DEV) for v in (a, b, U))

    def fnp(x):
        ux = U @ x
        return 0.5 * np.sum(a * x * x) + b @ x + 0.5 * ux @ ux, a * x + b + U.T @ ux

    def ft(x):
        ux = Ut @ x
        return float(0.5 * torch.sum(at * x * x) + bt @ x + 0.5 * ux @ ux), at * x + bt + Ut.T @ ux

    return fnp, ft


@pytest.mark.parametrize("seed", range(4))
def test_dense_quadratic_matches_scipy(seed):
    fnp, ft = quad_problem(40, seed)
    x0 = np.full(40, 0.5)
    rs, xs = scipy_run(fnp, x0, 0.0, 1.0)
    rg, xg = gpu_run(ft, x0, 0.0, 1.0)
    assert (rg.nit, rg.nfev) == (rs.nit, rs.nfev)
    assert rg.message == rs.message
    for a, b in zip(xg, xs):
        assert np.max(np.abs(a - b)) <= 1e-12
    assert abs(rg.fun - rs.fun) <= 1e-13 * abs(rs.fun)


@pytest.mark.parametrize("n", [1, 2047, 300001])
def test_large_coupled_quadratic_matches_scipy(n):
    """Many breakpoints over many sort tiles and scan chunks, ragged sizes."""
    fnp, ft = quad_problem(n, 7 + n % 5, rank=3)
    x0 = np.random.default_rng(n).random(n) * 1.4 - 0.2  # partly outside the box: projected first
    rs, xs = scipy_run(fnp, x0, 0.0, 1.0)
    rg, xg = gpu_run(ft, x0, 0.0, 1.0)
    assert abs(rg.nit - rs.nit) <= 1
    for k, (a, b) in enumerate(zip(xg[:5], xs[:5])):
        assert np.max(np.abs(a - b)) <= 1e-10, k
    assert abs(rg.fun - rs.fun) <= 1e-10 * max(1.0, abs(rs.fun))
    assert np.all((xg[-1] >= 0) & (xg[-1] <= 1))


def test_rosenbrock_line_search_matches_scipy():
    n = 30
    x0 = np.full(n, -0.5) + 0.1 * np.arange(n) / n

    def ft(x):
        xn = x.cpu().numpy()
        return float(rosen(xn)), torch.from_numpy(rosen_der(xn)).to(DEV)

    rs, xs = scipy_run(lambda x: (rosen(x), rosen_der(x)), x0, -1.0, 0.8)
    rg, xg = gpu_run(ft, x0, -1.0, 0.8)
    # the run is chaotic: rounding differences of 1e-16 grow about tenfold per 4 iterations
    for k in range(20):
        assert np.max(np.abs(xg[k] - xs[k])) <= 1e-9, k
    assert rs.nfev > rs.nit + 5  # the line search backtracked along the way
    assert abs(rg.fun - rs.fun) <= 1e-6 * abs(rs.fun)


def test_edge_cases():
    from paper_1707_09898_gb300.lbfgsb import CONV_PGTOL, minimize

    # every variable at a bound with the gradient pushing outward: converged at x0
    x0 = torch.tensor([0.0, 1.0, 0.0], dtype=torch.float64, device=DEV)
    g = torch.tensor([1.0, -1.0, 2.0], dtype=torch.float64, device=DEV)
    r = minimize(lambda x: (float(g @ x), g), x0)
    assert r.status == CONV_PGTOL and r.nit == 0 and r.nfev == 1
    # float32 evaluation point and gradient
    c = torch.tensor([0.25, 2.0, -1.0, 0.5], dtype=torch.float32, device=DEV)
    r = minimize(lambda x: (float(((x - c) ** 2).sum()), 2 * (x - c)), torch.zeros(4, device=DEV))
    assert np.allclose(r.x.cpu().numpy(), [0.25, 1.0, 0.0, 0.5], atol=1e-6)


def test_topology_objective_against_scipy_on_the_oracle():
    """The paper's objective (maximise the z field on a target box, J = -1/2 sum H_z^2 over
    its cells), 16^3 design, rho0 = 1, M0 = (0, 0, 1): GPU L-BFGS-B on the float32 CUDA
    objective vs SciPy's L-BFGS-B on the float64 oracle. (With the cell volume as a factor,
    |G| starts below SciPy's pgtol = 1e-5 at this size and both stop at once.)"""
    from oracle import convolution as C
    from oracle import objective as O
    from paper_1707_09898_gb300.lbfgsb import optimize_magnet
    from paper_1707_09898_gb300.magnet import Magnet

    n, cs = 16, 1.0 / 16
    n_out = (n, n, n + 2)
    mask = np.zeros((n + 2, n, n), np.uint8)
    mask[n:n + 2, 6:10, 6:10] = 1
    w = (0.0, 0.0, -0.5)
    op = C.Geometry(n_out, n, (cs, cs, cs))
    op = C.FFTOperator(op)
    M0 = np.array([0.0, 0.0, 1.0])

    def fnp(x):
        J, G, _ = O.objective_and_gradient(op, x.reshape(n, n, n), M0, 3.0, mask, np.zeros(3, np.float32), w)
        return J, G.ravel()

    rs, xs = scipy_run(fnp, np.ones(n ** 3), 0.0, 1.0)
    m = Magnet(n_out, n, (cs, cs, cs), M0=(0.0, 0.0, 1.0), p=3.0, device=0)
    m.set_target(torch.from_numpy(mask).to(DEV), Ht_const=(0.0, 0.0, 0.0), w=w)
    xg = []
    rg = optimize_magnet(m, torch.ones((n, n, n), device=DEV),
                         callback=lambda x, f: xg.append(x.cpu().numpy().ravel().copy()))
    print("scipy", rs.nit, rs.nfev, rs.fun, rs.message, "| gpu", rg.nit, rg.nfev, rg.fun, rg.message)
    assert rs.nit >= 5 and abs(rg.nit - rs.nit) <= max(2, rs.nit // 5)
    assert abs(rg.fun - rs.fun) <= 1e-3 * abs(rs.fun)
    for k in range(min(3, len(xs), len(xg))):
        assert np.max(np.abs(xg[k] - xs[k])) <= 1e-3, k
    # the final designs agree on most cells
    assert np.mean(np.abs(xg[-1] - rs.x) > 0.05) <= 0.02


def test_paper_validation_problem_against_scipy_on_the_oracle():
    """The paper's benchmark geometry (39^3 cube + 2 layers, maximise H_z on a 5 x 5 box,
    rho0 = 1): the GPU run (float32 objective, GPU L-BFGS-B) and SciPy's L-BFGS-B on the
    float64 oracle reach the same design."""
    from oracle import convolution as C
    from oracle import objective as O
    from paper_1707_09898_gb300 import paper_problem as PP
    from paper_1707_09898_gb300 import workloads as W

    wl = W.paper_problem(5)
    op = C.FFTOperator(C.Geometry(wl.n_out, wl.nzd, wl.cellsize))
    mask, M0, Ht = wl.mask(), wl.M0_const(), wl.Ht_const_vec()

    def fnp(x):
        J, G, _ = O.objective_and_gradient(op, x.reshape(wl.design_shape), M0, wl.p, mask, Ht, wl.w)
        return J, G.ravel()

    rs, _ = scipy_run(fnp, wl.rho().astype(np.float64).ravel(), 0.0, 1.0)
    out = PP.run(box=5)
    print({k: v for k, v in out.items() if not isinstance(v, list)}, "| scipy", rs.nit, rs.nfev, rs.fun)
    assert abs(out["N_iter"] - rs.nit) <= 3
    assert abs(out["J"] - rs.fun) <= 1e-3 * abs(rs.fun)
    assert abs(out["volume_fraction"] - rs.x.mean()) <= 0.01
    assert out["rerun_identical"]
    assert out["intermediate_fraction"] <= 0.05
    assert len(out["volume_fraction_per_evaluation"]) == out["nfev"]
