"""FP64 CPU oracle for the finite-difference magnet topology optimizer.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports, calls or links
this package: only the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it. It shares no code with the CUDA path
(``paper_1707_09898_gb300``) and imports nothing from it.

It is a plain, slow, obviously-correct restatement of what the method of
Abert et al., "A fast finite-difference algorithm for topology optimization of
permanent magnets" (arXiv:1707.09898) computes, in float64:

* ``tensor``      -- the cell-averaged demagnetization tensor of
  Eq. (demag_tensor) (Sec. "Discretization") by the Newell f/g second
  differences, with a far-field quadrature beyond a fixed integer distance.
* ``convolution`` -- the discrete convolution of Eq. (convolution), once by a
  zero-padded float64 FFT and once by direct O(N^2) summation, and its adjoint.
* ``objective``   -- the least-squares objective J(H(rho), rho) of
  Eq. (objective_function) and its adjoint gradient (Sec. "Methodology",
  Eqs. (adjoint1)-(adjoint2) and the operator form that follows them).
* ``optimizer``   -- the box-constrained projected-gradient update on rho.

Parity status: every function here is pinned by the CPU tests in
``tests/test_oracle_*.py`` against closed forms (cube self-term 1/3, the
Aharoni prism formula, trace identities), an independent Gauss-Legendre
quadrature of the six-fold integral, the point-dipole limit, direct summation,
the box identity, the adjoint dot-product identity and central finite
differences. The paper itself prints no numeric field, tensor or density
values, so no function is pinned to a number printed in the paper.
"""

from . import tensor, convolution, objective, optimizer  # noqa: F401
