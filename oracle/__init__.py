"""Plain FP64 CPU oracle of the multigrid-FFT free-space Poisson solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or runs
this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` do.  It shares no code, table or constant
generator with the CUDA library; both sides receive the same seeded inputs
from the synthetic generator module.

Each function follows the paper (arXiv 2512.08555) step by step and cites the
passage it implements.  Every numeric choice the paper leaves open is stated
in the docstring of the function that makes it.

Modules
-------
stencils      Eq. cross_discr2, Eq. mehrstellen_discr4/6, Sec. 2.1 interpolation,
              Sec. 3.1 transfer operators.
lgf           Sec. 2.2 / 3.3 lattice Green's function of the multigrid operator,
              free-space convolution on the uniform level, brute-force sum.
forest        Sec. 2.1 block forest, 2:1 and unbounded-boundary constraints.
multigrid     Alg. 1 adaptive FAS V-cycle with Gauss-Seidel smoothing.
composite     Independent route to the converged composite solution (GMRES).
closed_forms  Analytic free-space potentials used as pins.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py``; none is "parity unpinned".  The pins per module:

stencils      polynomial exactness, h^M truncation order, transfer weights;
lgf           Watson's constant (M = 2), L G = delta, symmetries, far field,
              direct summation, the Gaussian erf potential at order M;
forest        rejection of each violated constraint;
multigrid     single-level solve = brute-force direct sum; V-cycle limit =
              GMRES composite solution; O(h^M) E_inf order against the
              manufactured u_unb product (M = 2, 4, 6) and against the C4 bump's
              closed-form potential (M = 4, 6); stall with a non-LGF kernel;
              the Cauchy stop rule's limit = the GMRES composite solution;
composite     zero residual at the V-cycle fixed point;
closed_forms  Gaussian: order-M convergence of the discrete solution; bump:
              Gauss's-law quadrature and order-M convergence; u_unb: its
              Laplacian by finite differences;
adjoint       dot-product identity, finite differences, GMRES on the transpose.
"""
